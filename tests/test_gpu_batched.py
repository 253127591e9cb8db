"""Batched forward pass (several series of one grid size in one launch sequence):
every series equals its own single call, graph replays follow the inputs, and
parity with the FP64 oracle holds series by series."""
import numpy as np
import pytest

from parity import check_full, check_sampled, structural_rows, tc_unit_bounds
from synth import make_slp_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


# uneven lengths, trajectory lengths, neighbour counts and exclusions on a 9 x 14 grid
SHAPES = [(1400, 5, 20, 4), (333, 2, 5, 1), (901, 10, 10, 9), (260, 3, 7, 2),
          (1777, 7, 12, 6), (129, 1, 3, 0)]


def _series(shapes, h=9, w=14, seed0=100):
    return [make_slp_like(N, h, w, seed=seed0 + i)[0] for i, (N, _, _, _) in enumerate(shapes)]


def _single(tk, Xd, L, k, e, prec):
    """The single-series call on the batched path's operands (trajectory-embedded
    operands off: the batched form never embeds)."""
    import torch
    idx, dist, score = tk.knn_scores(Xd, L, k, e, precision=prec, embed="never")
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy()


def _batched(tk, Xds, shapes, prec, **kw):
    import torch
    outs = tk.knn_scores_batched([(X, L, k, e) for X, (_, L, k, e) in zip(Xds, shapes)],
                                 precision=prec, **kw)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    return [tuple(t.cpu().numpy() for t in o) for o in outs]


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_each_series_equals_its_single_call(tk, prec):
    import torch
    Xs = _series(SHAPES)
    Xds = [torch.from_numpy(X).cuda() for X in Xs]
    got = _batched(tk, Xds, SHAPES, prec)
    for X, (N, L, k, e), g in zip(Xds, SHAPES, got):
        ref = _single(tk, X, L, k, e, prec)
        for a, b in zip(ref, g):
            assert np.array_equal(a, b), (N, L, k, e)


def test_batched_parity_with_oracle(tk):
    import torch
    Xs = _series(SHAPES, seed0=300)
    Xds = [torch.from_numpy(X).cuda() for X in Xs]
    got = _batched(tk, Xds, SHAPES, "split_bf16")
    for X, (N, L, k, e), (idx, dist, score) in zip(Xs, SHAPES, got):
        check_full(X, L, k, e, idx, dist, score, 2e-4)


def test_graph_replay_follows_new_inputs(tk):
    """The second call with the same shapes and pointers replays the captured graph;
    new data written into the same input buffers must give the new results."""
    import torch
    shapes = SHAPES[:4]
    Xds = [torch.from_numpy(X).cuda() for X in _series(shapes, seed0=500)]
    outs = [(torch.empty((N - L + 1, k), dtype=torch.int32, device="cuda"),
             torch.empty((N - L + 1, k), dtype=torch.float32, device="cuda"),
             torch.empty((N - L + 1,), dtype=torch.float32, device="cuda"))
            for N, L, k, _ in shapes]
    first = _batched(tk, Xds, shapes, "split_bf16", outs=outs)
    again = _batched(tk, Xds, shapes, "split_bf16", outs=outs)
    for a, b in zip(first, again):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    for X, Xn in zip(Xds, _series(shapes, seed0=700)):
        X.copy_(torch.from_numpy(Xn))
    replay = _batched(tk, Xds, shapes, "split_bf16", outs=outs)
    for X, (N, L, k, e), g in zip(Xds, shapes, replay):
        ref = _single(tk, X, L, k, e, "split_bf16")
        for a, b in zip(ref, g):
            assert np.array_equal(a, b)


def test_more_series_than_one_launch_holds(tk):
    """70 short series: split into launch groups of at most 64."""
    import torch
    rng = np.random.default_rng(9)
    shapes = [(int(rng.integers(60, 200)), int(rng.integers(1, 6)), int(rng.integers(1, 9)), 0)
              for _ in range(70)]
    shapes = [(N, L, k, L - 1) for N, L, k, _ in shapes]
    Xs = [make_slp_like(N, 4, 6, seed=900 + i)[0] for i, (N, _, _, _) in enumerate(shapes)]
    Xds = [torch.from_numpy(X).cuda() for X in Xs]
    got = _batched(tk, Xds, shapes, "split_bf16")
    for X, (N, L, k, e), g in zip(Xds, shapes, got):
        ref = _single(tk, X, L, k, e, "split_bf16")
        for a, b in zip(ref, g):
            assert np.array_equal(a, b)


def test_autotuned_unit_size_gives_the_same_results(tk):
    import torch
    Xs = _series(SHAPES[:3], seed0=1100)
    Xds = [torch.from_numpy(X).cuda() for X in Xs]
    ref = _batched(tk, Xds, SHAPES[:3], "split_bf16")
    got = _batched(tk, Xds, SHAPES[:3], "split_bf16", autotune=True)
    tiles, group = tk.get_handle().work_shape()
    assert tiles in (4, 8, 16) and group in (10, 19, 38)
    tk.get_handle().set_option("autotune", 0)
    for a, b in zip(ref, got):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_invalid_series_is_rejected_before_launch(tk):
    import torch
    Xds = [torch.from_numpy(X).cuda() for X in _series([(1400, 5, 20, 4), (40, 2, 40, 1)],
                                                        seed0=1300)]
    bad = [(Xds[0], 5, 20, 4), (Xds[1], 2, 40, 1)]  # second: 36 candidates for k = 40
    n0 = tk.get_handle().launch_count()
    with pytest.raises(tk.TrakNNError) as ei:
        tk.knn_scores_batched(bad)
    assert ei.value.status == 2
    assert tk.get_handle().launch_count() == n0


def test_graph_cache_stays_bounded(tk):
    """New output buffers on every call create new graph signatures; the cache keeps
    only the most recent ones and every call stays correct."""
    import torch
    shapes = SHAPES[:2]
    Xds = [torch.from_numpy(X).cuda() for X in _series(shapes, seed0=1500)]
    ref = [_single(tk, X, L, k, e, "split_bf16") for X, (N, L, k, e) in zip(Xds, shapes)]
    for _ in range(20):
        got = _batched(tk, Xds, shapes, "split_bf16")  # fresh outputs each time
        for a, b in zip(ref, got):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_batched_with_k_segments_equals_single_calls(tk):
    """Several series whose Gram entries are accumulated in K segments (folded through
    the per-CTA scratch): each equals its single call under the same segmenting."""
    import torch
    shapes = [(700, 5, 10, 4), (450, 3, 6, 2), (820, 8, 12, 7)]
    Xds = [torch.from_numpy(make_slp_like(N, 30, 40, seed=1700 + i)[0]).cuda()
           for i, (N, _, _, _) in enumerate(shapes)]  # D = 1,200
    h = tk.get_handle()
    try:
        h.set_option("segment_k", 256)
        got = _batched(tk, Xds, shapes, "split_bf16", handle=h)
        ref = [_single(tk, X, L, k, e, "split_bf16") for X, (N, L, k, e) in zip(Xds, shapes)]
    finally:
        h.set_option("segment_k", 0)
    for r, g in zip(ref, got):
        for a, b in zip(r, g):
            assert np.array_equal(a, b)


def test_batched_full_grid_series_parity_with_oracle(tk):
    """Series shaped like the batched workload (1-degree European grid, D = 3,726;
    N drawn from [3,650, 27,394]; per-series L in 2..10 and k in {5, 10, 20}, exclusion
    L - 1) in one batched call: every series' sampled rows (boundary rows of every
    fourth strip, unit edges, 40 random rows) against the oracle, and bitwise
    equality with the series' own single call for two of them."""
    import torch
    rng = np.random.default_rng(20260305)
    shapes = []
    for _ in range(7):
        L = int(rng.integers(2, 11))
        shapes.append((int(rng.integers(3650, 27395)), L, int(rng.choice([5, 10, 20])), L - 1))
    shapes.append((27394, 5, 20, 4))  # the longest series of the workload's range
    Xs = [make_slp_like(N, 46, 81, seed=20260400 + b)[0] for b, (N, _, _, _) in enumerate(shapes)]
    Xds = [torch.from_numpy(X).cuda() for X in Xs]
    got = _batched(tk, Xds, shapes, "split_bf16")
    for b, (X, (N, L, k, e), (idx, dist, score)) in enumerate(zip(Xs, shapes, got)):
        M = N - L + 1
        rows = structural_rows(M, L, n_random=40, seed=b, strip_every=4,
                               col_bounds=tc_unit_bounds(M, L)[::3])
        check_sampled(X, L, k, e, rows, idx, dist, score, 2e-4)
    for b in (0, len(shapes) - 1):
        N, L, k, e = shapes[b]
        ref = _single(tk, Xds[b], L, k, e, "split_bf16")
        for x, y in zip(ref, got[b]):
            assert np.array_equal(x, y), shapes[b]
