"""FP64 CPU oracle for the TRAKNN trajectory-kNN rarity score (arXiv 2603.02059).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the CUDA library or its binding.

The arithmetic lives in ``traknn_oracle.c`` (plain C, double precision, written
from Sec. 3.2 Eq. 2-3 and Algorithm 1's kNN step); this module compiles it with
gcc on first use and wraps it with ctypes.

Parity status of each function (pins in tests/test_oracle_pins.py):

* ``snapshot_matrix``  pinned: symmetry, zero diagonal, closed forms (linear
  and circular day sequences), numpy brute force on tiny inputs.
* ``traj_rows`` / ``traj_matrix``  pinned: Eq. 2 tensor form by brute force,
  the Eq. 5 recurrence, L=1 reduction, constant-offset invariance.
* ``knn_scores`` / ``knn_from_rows``  pinned: scipy/argsort brute force, the
  k-prefix property, the k=1 matrix-profile case, closed-form neighbour sets,
  a planted anomaly ranking first.
* ``score_grad``  pinned: exact central finite differences of an independent
  numpy score, and torch float64 autograd through the Eq. 2 definition.
* grid-point weights (``weights=`` of the functions above)  pinned: all-ones
  weights reproduce the unweighted results bit for bit, constant weights scale
  every distance exactly, 0/1 weights equal the unweighted oracle on the selected
  grid points.
* ``prefix_scores``  pinned: numpy brute force on tiny inputs, nesting of the
  neighbour sets over k (Sec. 6).
* ``local_id``  pinned: a hand-computed closed form, invariance to scaling X,
  and points spread uniformly over a 3-dimensional cube embedded in 30 dimensions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "traknn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARGS, ERR_FEW_CANDIDATES, ERR_NOMEM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            lib.oracle_snapshot_matrix.argtypes = [P, I64, I64, P, I]
            lib.oracle_traj_matrix.argtypes = [P, I64, I, P]
            lib.oracle_traj_rows.argtypes = [P, I64, I64, I, P, I64, P, I]
            lib.oracle_knn_from_rows.argtypes = [P, P, I64, I64, I, I, I, P, P, P]
            lib.oracle_knn_scores.argtypes = [P, I64, I64, I, I, I, I, P, P, P, P, I]
            lib.oracle_score_grad.argtypes = [P, I64, I64, I, I, P, P, P]
            lib.oracle_snapshot_matrix_w.argtypes = [P, I64, I64, P, P, I]
            lib.oracle_traj_rows_w.argtypes = [P, I64, I64, I, P, P, I64, P, I]
            lib.oracle_knn_scores_w.argtypes = [P, I64, I64, I, P, I, I, I, P, P, P, P, I]
            lib.oracle_score_grad_w.argtypes = [P, I64, I64, I, P, I, P, P, P]
            lib.oracle_num_threads.argtypes = [I]
            for f in (lib.oracle_snapshot_matrix, lib.oracle_traj_matrix, lib.oracle_traj_rows,
                      lib.oracle_knn_from_rows, lib.oracle_knn_scores, lib.oracle_score_grad,
                      lib.oracle_snapshot_matrix_w, lib.oracle_traj_rows_w,
                      lib.oracle_knn_scores_w, lib.oracle_score_grad_w,
                      lib.oracle_num_threads):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X must be 2-D (days x grid points)")
    return X


def _weights(w, D):
    """Grid-point weights as a contiguous float64 array (None: unweighted)."""
    if w is None:
        return None, None
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.shape != (D,) or np.any(w < 0):
        raise ValueError("weights must be D non-negative values")
    return w, _ptr(w)


def _check(rc):
    if rc != OK:
        raise RuntimeError({ERR_ARGS: "invalid arguments",
                            ERR_FEW_CANDIDATES: "fewer than k candidates",
                            ERR_NOMEM: "out of memory"}.get(rc, f"oracle error {rc}"))


def num_threads(nthreads: int = 0) -> int:
    return int(_load().oracle_num_threads(nthreads))


def snapshot_matrix(X, nthreads: int = 0, weights=None) -> np.ndarray:
    """S[a, b] = sum_p w_p (X[a,p] - X[b,p])^2 (Eq. 2 inner term; w = 1 unless
    grid-point weights are given), N x N float64."""
    X = _f32(X)
    N, D = X.shape
    w, wp = _weights(weights, D)
    S = np.empty((N, N), dtype=np.float64)
    _check(_load().oracle_snapshot_matrix_w(_ptr(X), N, D, wp, _ptr(S), nthreads))
    return S


def traj_matrix(S: np.ndarray, L: int) -> np.ndarray:
    """D[t, j] = sum_{m<L} S[t+m, j+m] (Eq. 2), M x M float64."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    N = S.shape[0]
    M = N - L + 1
    Dt = np.empty((M, M), dtype=np.float64)
    _check(_load().oracle_traj_matrix(_ptr(S), N, L, _ptr(Dt)))
    return Dt


def traj_rows(X, L: int, rows, nthreads: int = 0, weights=None) -> np.ndarray:
    """Rows of D computed directly from X: out[r, j] = D(rows[r], j)."""
    X = _f32(X)
    N, D = X.shape
    w, wp = _weights(weights, D)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    M = N - L + 1
    out = np.empty((rows.size, M), dtype=np.float64)
    _check(_load().oracle_traj_rows_w(_ptr(X), N, D, L, wp, _ptr(rows), rows.size, _ptr(out),
                                      nthreads))
    return out


def knn_from_rows(Drows, rows, k: int, e: int, kk: int | None = None):
    """Neighbour sets and scores of the given rows from their full D rows.

    Returns (idx int32 [n, kk], dist float64 [n, kk], score float64 [n]); the
    first k columns are the neighbour set sorted by (D, index), columns k..kk
    continue the sorted candidate order (for near-tie checks)."""
    Drows = np.ascontiguousarray(Drows, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    kk = k if kk is None else kk
    n, M = Drows.shape
    idx = np.empty((n, kk), dtype=np.int32)
    dist = np.empty((n, kk), dtype=np.float64)
    score = np.empty(n, dtype=np.float64)
    _check(_load().oracle_knn_from_rows(_ptr(Drows), _ptr(rows), n, M, k, kk, e, _ptr(idx),
                                        _ptr(dist), _ptr(score)))
    return idx, dist, score


def knn_scores(X, L: int, k: int, e: int, kk: int | None = None, nthreads: int = 0,
               return_D: bool = False, weights=None):
    """Full oracle over all M = N-L+1 trajectories (stores S and D: small N only)."""
    X = _f32(X)
    N, D = X.shape
    w, wp = _weights(weights, D)
    kk = k if kk is None else kk
    M = N - L + 1
    idx = np.empty((M, kk), dtype=np.int32)
    dist = np.empty((M, kk), dtype=np.float64)
    score = np.empty(M, dtype=np.float64)
    Dt = np.empty((M, M), dtype=np.float64) if return_D else None
    _check(_load().oracle_knn_scores_w(_ptr(X), N, D, L, wp, k, kk, e, _ptr(idx), _ptr(dist),
                                       _ptr(score), _ptr(Dt) if return_D else None, nthreads))
    if return_D:
        return idx, dist, score, Dt
    return idx, dist, score


def knn_rows(X, L: int, k: int, e: int, rows, kk: int | None = None, nthreads: int = 0,
             weights=None):
    """Neighbour sets/scores for sampled rows at any size; also returns the D rows."""
    Drows = traj_rows(X, L, rows, nthreads, weights=weights)
    idx, dist, score = knn_from_rows(Drows, rows, k, e, kk)
    return idx, dist, score, Drows


def score_grad(X, L: int, k: int, idx, g, weights=None) -> np.ndarray:
    """d(sum_t g_t s_t)/dX with the neighbour sets idx (M x k) held fixed, float64."""
    X = _f32(X)
    N, D = X.shape
    w, wp = _weights(weights, D)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    g = np.ascontiguousarray(g, dtype=np.float64)
    dX = np.empty((N, D), dtype=np.float64)
    _check(_load().oracle_score_grad_w(_ptr(X), N, D, L, wp, k, _ptr(idx), _ptr(g), _ptr(dX)))
    return dX


def prefix_scores(X, L: int, k: int, e: int, weights=None) -> np.ndarray:
    """Scores for every neighbour count k' = 1..k: out[t, k'-1] = s_t with k' neighbours
    (Eq. 3 at k'), each from its own full kNN selection (the definition; the paper notes
    in Sec. 6 that the k' sets are nested in the k set). Small N only (stores D)."""
    _, _, _, Dt = knn_scores(X, L, 1, e, return_D=True, weights=weights)
    M = Dt.shape[0]
    rows = np.arange(M)
    out = np.empty((M, k), dtype=np.float64)
    for kp in range(1, k + 1):
        out[:, kp - 1] = knn_from_rows(Dt, rows, kp, e)[2]
    return out


def local_id(dist, k: int) -> np.ndarray:
    """Local intrinsic dimension of every row by the maximum-likelihood kNN estimator of
    Levina and Bickel (2004), as applied to the trajectories in Sec. 4 (intrinsic
    dimension study): with T_j the distance to the j-th nearest neighbour,
        m(t) = [ (1/(k-1)) sum_{j=1}^{k-1} log(T_k / T_j) ]^(-1).
    `dist` holds squared distances sorted ascending per row (as the kNN search returns
    them), so log(T_k / T_j) = log(d_k / d_j) / 2. Rows with a zero distance among the
    first k, or with all k distances equal, have no finite estimate: NaN."""
    d = np.asarray(dist, dtype=np.float64)[:, :k]
    out = np.full(d.shape[0], np.nan)
    for t in range(d.shape[0]):
        row = d[t]
        if row[0] <= 0.0:
            continue
        s = 0.0
        for j in range(k - 1):
            s += 0.5 * np.log(row[k - 1] / row[j])
        if s > 0.0:
            out[t] = (k - 1) / s
    return out
