"""Parity of the tensor-core (tcgen05) paths with the FP64 oracle, through the C ABI,
and the bounded-wait failure path."""
import numpy as np
import pytest

from conftest import load_golden
from parity import check_full, check_sampled, structural_rows, tc_unit_bounds
from synth import config_inputs, make_slp_like

pytestmark = pytest.mark.gpu
TOL = {"split_bf16": 2e-4, "bf16": 2e-2}


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _run(tk, X, L, k, e, prec="split_bf16", **kw):
    import torch
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, precision=prec, **kw)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    return idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy()


@pytest.mark.parametrize("embed", ["never", "always"])
@pytest.mark.parametrize("prec", ["split_bf16", "bf16"])
def test_hand_example_exact(tk, prec, embed):
    """Small integers are exact in BF16, so both tensor-core forms are exact here, with
    diagonal window sums and with trajectory-embedded operands."""
    Xrows, cases = load_golden("hand_example_6days.txt")
    X = np.array(Xrows, dtype=np.float32)
    for name, (p, rows) in cases.items():
        idx, dist, score = _run(tk, X, p["L"], p["k"], p["e"], prec, center=False, embed=embed)
        for t, (gi, gd, gs) in rows.items():
            assert list(idx[t]) == gi, (name, t)
            assert list(dist[t]) == gd, (name, t)
            assert score[t] == gs, (name, t)


def test_small_5y_config_split(tk):
    X, meta, cfg = config_inputs("small_5y_16x32")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    idx, dist, score = _run(tk, X, L, k, e)
    check_full(X, L, k, e, idx, dist, score, TOL["split_bf16"])


@pytest.mark.parametrize("N,h,w,L,k,e", [
    (517, 7, 11, 5, 7, 4),
    (300, 4, 5, 1, 1, 0),
    (420, 6, 6, 17, 64, 16),
    (20, 1, 3, 2, 2, 1),
    (1000, 3, 3, 2, 9, 0),
    (777, 9, 15, 10, 20, 9),
    (1300, 16, 20, 7, 33, 6),
    (900, 8, 10, 4, 45, 3),
])
@pytest.mark.parametrize("embed", ["never", "always"])
def test_shapes_split(tk, N, h, w, L, k, e, embed):
    X, _ = make_slp_like(N, h, w, seed=N + L)
    idx, dist, score = _run(tk, X, L, k, e, embed=embed)
    check_full(X, L, k, e, idx, dist, score, TOL["split_bf16"])


@pytest.mark.parametrize("epi_groups", [0, 1])
def test_single_day_trajectories_on_long_rows(tk, epi_groups):
    """L = 1 with long operand rows (D = 1,200: 1,280 K entries, one accumulation
    segment): by default two epilogue groups with the split band pre-pass; with one
    group the band pre-pass runs in one BF16 product and raises its distances by their
    error bound before they become row bounds. Full parity with the oracle either way."""
    import torch
    X, _ = make_slp_like(1500, 30, 40, seed=1201)
    L, k, e = 1, 10, 0
    h = tk.Handle()
    h.set_option("epi_groups", epi_groups)
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, handle=h)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    h.close()
    check_full(X, L, k, e, idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(),
               TOL["split_bf16"])


def test_bf16_error_is_bounded(tk):
    X, meta, cfg = config_inputs("small_5y_16x32")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    idx, dist, score = _run(tk, X, L, k, e, "bf16")
    check_full(X, L, k, e, idx, dist, score, TOL["bf16"])


@pytest.mark.parametrize("cols", [256, 300, 700, 5000])
def test_work_unit_size_is_bitwise_invariant(tk, cols):
    X, _ = make_slp_like(1500, 8, 12, seed=6)
    ref = _run(tk, X, 5, 10, 4, embed="never")
    got = _run(tk, X, 5, 10, 4, unit_cols=cols, embed="never")
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("N,h,w,L,k,e", [(1500, 8, 12, 5, 10, 4), (777, 9, 15, 10, 20, 9),
                                         (420, 6, 6, 17, 64, 16), (300, 4, 5, 1, 1, 0),
                                         (1000, 3, 3, 2, 9, 0)])
@pytest.mark.parametrize("embed", ["never", "always"])
def test_symmetric_split_equals_full_evaluation(tk, N, h, w, L, k, e, embed):
    """Evaluating each unordered pair once (upper triangle with column-side lists)
    gives the neighbour lists and scores of evaluating both triangles. D(t,j) and
    D(j,t) come from Gram tiles with the operand roles swapped, so they may differ
    in the last bit: distances agree to 1e-6 and index sets may differ only at
    near ties."""
    X, _ = make_slp_like(N, h, w, seed=N + 2 * L)
    full = _run(tk, X, L, k, e, symmetric=False, embed=embed)
    half = _run(tk, X, L, k, e, symmetric=True, embed=embed)
    rel = np.abs(full[1] - half[1]) / np.maximum(np.abs(full[1]), 1e-30)
    assert rel.max() <= 1e-6
    assert np.allclose(full[2], half[2], rtol=1e-6)
    same = (full[0] == half[0]).all(axis=1)
    for t in np.nonzero(~same)[0]:
        # rows that differ exchange only neighbours tied (to 1e-6) with the k-th distance
        dk = full[1][t][-1]
        fd = dict(zip(full[0][t].tolist(), full[1][t].tolist()))
        hd = dict(zip(half[0][t].tolist(), half[1][t].tolist()))
        for j in set(fd) - set(hd):
            assert abs(fd[j] - dk) <= 1e-6 * dk, (t, j)
        for j in set(hd) - set(fd):
            assert abs(hd[j] - dk) <= 1e-6 * dk, (t, j)


def test_constant_offset_invariance(tk):
    X, _ = make_slp_like(700, 8, 8, seed=19)
    F = np.linspace(950.0, 1050.0, X.shape[1], dtype=np.float32)[None, :]
    idx, dist, score = _run(tk, (X + F).astype(np.float32), 4, 6, 3)
    check_full(X, 4, 6, 3, idx, dist, score, TOL["split_bf16"])


def test_euro_75y_sampled_rows_split(tk):
    """The headline workload at full size: the first and last row of every row strip,
    the rows at every work-unit and first-unit tile edge, the planted anomalies and
    500 seeded random rows against the oracle; the planted anomalies rank first."""
    X, meta, cfg = config_inputs("euro_75y_46x81")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    idx, dist, score = _run(tk, X, L, k, e)
    M = X.shape[0] - L + 1
    rows = structural_rows(M, L, n_random=500, seed=1, col_bounds=tc_unit_bounds(M, L),
                           extra=meta.planted_starts)
    assert len(rows) >= 900
    check_sampled(X, L, k, e, rows, idx, dist, score, TOL["split_bf16"])
    order = np.argsort(-score)
    top, taken = [], np.zeros(M, bool)
    for t in order:
        if not taken[max(0, t - L):t + L].any():
            top.append(t)
            taken[t] = True
        if len(top) == len(meta.planted_starts):
            break
    for s0 in meta.planted_starts:
        assert min(abs(t - s0) for t in top) <= L - 1


@pytest.mark.parametrize("L,k", [(17, 64), (10, 48), (10, 20), (2, 1)])
def test_euro_75y_sampled_rows_extreme_settings(tk, L, k):
    """The 75-year workload at the largest (and the smallest) supported trajectory
    length and neighbour count: every third strip's boundary rows, the unit edges and
    100 random rows against the oracle."""
    X, meta, cfg = config_inputs("euro_75y_46x81")
    e = L - 1
    idx, dist, score = _run(tk, X, L, k, e)
    M = X.shape[0] - L + 1
    rows = structural_rows(M, L, n_random=100, seed=L * 100 + k, strip_every=3,
                           col_bounds=tc_unit_bounds(M, L)[::2])
    check_sampled(X, L, k, e, rows, idx, dist, score, TOL["split_bf16"])


def test_bounded_wait_reports_timeout(tk):
    """The producer withholds one stage (test hook): the consumer's bounded wait runs out,
    the kernel records TRAKNN_ERR_TIMEOUT and returns; the next call is correct again."""
    import torch
    h = tk.Handle()
    X, _ = make_slp_like(400, 6, 6, seed=3)
    Xd = torch.from_numpy(X).cuda()
    h.set_option("wait_limit_ms", 300)
    h.set_option("debug_withhold", 1)
    tk.knn_scores(Xd, 3, 4, 2, handle=h)
    assert h.sync_status() == 5
    h.set_option("debug_withhold", 0)
    idx, dist, score = tk.knn_scores(Xd, 3, 4, 2, handle=h)
    assert h.sync_status() == 0
    check_full(X, 3, 4, 2, idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(),
               TOL["split_bf16"])
    h.close()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_constant_series_ties_go_to_smaller_indices(tk, prec):
    """Every distance is zero: each row's neighbours are its k smallest candidate
    indices (Algorithm 1's kNN step with the smaller-index tie rule)."""
    N, L, k, e = 700, 3, 12, 2
    X = np.full((N, 10), 3.25, dtype=np.float32)
    idx, dist, score = _run(tk, X, L, k, e, prec)
    M = N - L + 1
    for t in range(M):
        exp = [j for j in range(M) if abs(j - t) > e][:k]
        assert list(idx[t]) == exp, t
    assert np.all(dist == 0) and np.all(score == 0)


@pytest.mark.parametrize("seg", [64, 1024])
def test_segmented_accumulation(tk, seg):
    """Gram entries accumulated on the tensor cores in segments of `seg` grid points,
    the segments added in FP32: parity with the oracle, and agreement with the
    default accumulation."""
    h = tk.get_handle()
    X, _ = make_slp_like(1500, 46, 81, seed=77)
    try:
        h.set_option("segment_k", seg)
        idx, dist, score = _run(tk, X, 5, 10, 4)
    finally:
        h.set_option("segment_k", 0)
    check_full(X, 5, 10, 4, idx, dist, score, TOL["split_bf16"])
    ref = _run(tk, X, 5, 10, 4)
    assert np.allclose(score, ref[2], rtol=1e-4, atol=0)
