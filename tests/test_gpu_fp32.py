"""Parity of the FP32 CUDA path with the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

from conftest import load_golden
from parity import check_full, check_sampled, fp32_chunk_bounds, structural_rows
from synth import config_inputs, make_slp_like

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _run(tk, X, L, k, e, **kw):
    import torch
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, precision="fp32", **kw)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    return idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy()


def test_hand_example_exact(tk):
    Xrows, cases = load_golden("hand_example_6days.txt")
    X = np.array(Xrows, dtype=np.float32)
    for name, (p, rows) in cases.items():
        idx, dist, score = _run(tk, X, p["L"], p["k"], p["e"], center=False)
        for t, (gi, gd, gs) in rows.items():
            assert list(idx[t]) == gi, (name, t)
            assert list(dist[t]) == gd, (name, t)
            assert score[t] == gs, (name, t)


def test_small_5y_config_full_parity(tk):
    X, meta, cfg = config_inputs("small_5y_16x32")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    idx, dist, score = _run(tk, X, L, k, e)
    check_full(X, L, k, e, idx, dist, score, TOL)


@pytest.mark.parametrize("N,h,w,L,k,e", [
    (517, 7, 11, 5, 7, 4),      # D=77: ragged K, several strips and chunks, ragged tails
    (300, 4, 5, 1, 1, 0),       # L=1, k=1: snapshot matrix profile
    (420, 6, 6, 17, 64, 16),    # largest L and k
    (20, 1, 3, 2, 2, 1),        # a single partial strip
    (1000, 3, 3, 2, 9, 0),      # tiny D, zero exclusion
    (777, 9, 15, 10, 20, 9),
])
def test_shapes_full_parity(tk, N, h, w, L, k, e):
    X, _ = make_slp_like(N, h, w, seed=N + L)
    idx, dist, score = _run(tk, X, L, k, e)
    check_full(X, L, k, e, idx, dist, score, TOL)


@pytest.mark.parametrize("chunks", [1, 3, 32])
def test_column_chunking_is_bitwise_invariant(tk, chunks):
    X, _ = make_slp_like(900, 8, 10, seed=5)
    ref = _run(tk, X, 4, 6, 3)
    got = _run(tk, X, 4, 6, 3, col_chunks=chunks)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_constant_offset_invariance(tk):
    X, _ = make_slp_like(600, 8, 8, seed=9)
    F = np.linspace(900.0, 1100.0, X.shape[1], dtype=np.float32)[None, :]
    idx, dist, score = _run(tk, (X + F).astype(np.float32), 3, 5, 2)
    check_full(X, 3, 5, 2, idx, dist, score, TOL)


def test_euro_75y_sampled_rows(tk):
    X, meta, cfg = config_inputs("euro_75y_46x81")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    idx, dist, score = _run(tk, X, L, k, e)
    M = X.shape[0] - L + 1
    # first and last row of every strip, the column-chunk edges, the planted
    # anomalies and 500 seeded random rows
    rows = structural_rows(M, L, n_random=500, seed=0, col_bounds=fp32_chunk_bounds(M),
                           extra=meta.planted_starts)
    assert len(rows) >= 900
    check_sampled(X, L, k, e, rows, idx, dist, score, TOL)
    # the planted multi-day anomalies are the rarest trajectories
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
