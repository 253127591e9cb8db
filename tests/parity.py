"""Comparison of the CUDA path's neighbour lists and scores with the FP64 oracle.

Rules (per trajectory row t):
  * every returned index is a valid candidate (0 <= j < M, |t - j| > e, distinct);
  * the returned distances are non-decreasing, and each equals the oracle's D(t, j)
    for that index within the relative tolerance;
  * the sorted distance profile matches the oracle's k smallest within tolerance;
  * the index set equals the oracle's, except that indices whose true distance is
    within tolerance of the oracle's k-th distance may be exchanged (near ties);
  * the score matches the oracle's within tolerance.
"""
import numpy as np

import oracle


def check_rows(rows, gidx, gdist, gscore, Drows, oidx, odist, oscore, M, k, e, tol):
    """All arrays are per sampled row; Drows[r] is the oracle's full D(t, .) row."""
    fails = []
    for r, t in enumerate(rows):
        gi = np.asarray(gidx[r], dtype=np.int64)
        gd = np.asarray(gdist[r], dtype=np.float64)
        Dr = Drows[r]
        dk = odist[r, k - 1]
        scale = max(float(np.median(odist[r, :k])), 1e-30)
        atol = tol * 1e-3 * scale
        if np.any(gi < 0) or np.any(gi >= M):
            fails.append((t, "index out of range", gi))
            continue
        if len(set(gi.tolist())) != k:
            fails.append((t, "duplicate indices", gi))
            continue
        if np.any(np.abs(gi - t) <= e):
            fails.append((t, "excluded index returned", gi))
            continue
        if np.any(np.diff(gd) < -tol * np.abs(gd[1:]) - atol):
            fails.append((t, "distances not sorted", gd))
        true_d = Dr[gi]
        if np.any(np.abs(gd - true_d) > tol * np.abs(true_d) + atol):
            fails.append((t, "reported distance differs from D(t,j)",
                          float(np.max(np.abs(gd - true_d) / np.maximum(true_d, 1e-30)))))
        if np.any(np.abs(gd - odist[r, :k]) > tol * np.abs(odist[r, :k]) + atol):
            fails.append((t, "distance profile differs",
                          float(np.max(np.abs(gd - odist[r, :k]) / odist[r, :k]))))
        oi = set(np.asarray(oidx[r, :k]).tolist())
        gs = set(gi.tolist())
        if oi != gs:
            extra = gs - oi
            missing = oi - gs
            near = all(abs(Dr[j] - dk) <= tol * dk + atol for j in extra | missing)
            if not near:
                fails.append((t, "neighbour set differs beyond a near tie",
                              sorted(extra), sorted(missing)))
        if abs(gscore[r] - oscore[r]) > tol * abs(oscore[r]) + atol:
            fails.append((t, "score differs", float(gscore[r]), float(oscore[r])))
    assert not fails, f"{len(fails)} rows fail, first: {fails[:3]}"


def check_full(X, L, k, e, gidx, gdist, gscore, tol):
    """Compare all rows against the full oracle (small N)."""
    oidx, odist, oscore, Dt = oracle.knn_scores(X, L, k, e, kk=k + 1, return_D=True)
    M = Dt.shape[0]
    rows = np.arange(M)
    check_rows(rows, gidx, gdist, gscore, Dt, oidx, odist, oscore, M, k, e, tol)
    return oscore


def check_sampled(X, L, k, e, rows, gidx, gdist, gscore, tol):
    """Compare sampled rows (GPU outputs for all rows; oracle rows computed one by one)."""
    rows = np.asarray(rows, dtype=np.int64)
    oidx, odist, oscore, Drows = oracle.knn_rows(X, L, k, e, rows, kk=k + 1)
    M = X.shape[0] - L + 1
    check_rows(rows, gidx[rows], gdist[rows], gscore[rows], Drows, oidx, odist, oscore, M, k,
               e, tol)


def structural_rows(M, L, *, n_random=500, seed=0, strip_every=1, col_bounds=(),
                    extra=(), rows_per_strip=None):
    """Trajectory rows that exercise the kernels' work split at full size.

    Output rows are cut into strips of 128 - (L-1) rows (one Gram tile height minus
    the window halo): the first and last row of every `strip_every`-th strip; the
    rows on both sides of each column boundary in `col_bounds` (work-unit and chunk
    edges); the first two and last two rows; `extra` rows; and `n_random` seeded
    random rows. `rows_per_strip` overrides the strip height (128 with
    trajectory-embedded operands, which have no window halo)."""
    R = rows_per_strip or 128 - (L - 1)
    rows = [0, 1, M - 2, M - 1]
    for s in range(0, (M + R - 1) // R, strip_every):
        rows += [s * R, min(M - 1, s * R + R - 1)]
    for c in col_bounds:
        rows += [c - 1, c]
    rows += list(extra)
    rng = np.random.default_rng(seed)
    rows += rng.integers(0, M, n_random).tolist()
    rows = np.unique(np.asarray(rows, dtype=np.int64))
    return rows[(rows >= 0) & (rows < M)]


def tc_unit_bounds(M, L, tiles=8):
    """Column edges of the tensor-core path's work units (tiles consecutive Gram tiles
    of 256 columns, tiles * 256 - (L-1) output columns; L = 1 with trajectory-embedded
    operands) and of the tiles inside the first unit (the first yields 256 - (L-1)
    output columns, the later ones 256 each, the last L-1 Gram columns carried)."""
    cols = tiles * 256 - (L - 1)
    inner = range(256 - (L - 1), min(M, cols), 256)
    return sorted(set(list(range(cols, M, cols)) + list(inner)))


def fp32_chunk_bounds(M, chunks=8):
    """Column edges of the FP32 path's column chunks."""
    cc = -(-M // chunks)
    return list(range(cc, M, cc))
