"""Grid-point weights (forward paths and adjoint) and the statistics of sorted
neighbour lists (scores for every k' <= k, local intrinsic dimension) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from parity import check_rows
from synth import config_inputs, make_slp_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _coslat(h, w):
    lat = np.deg2rad(np.linspace(35.0, 72.0, h))
    return np.repeat(np.cos(lat), w).astype(np.float32)


@pytest.mark.parametrize("prec,tol", [("split_bf16", 2e-4), ("fp32", 1e-5)])
def test_weighted_forward_matches_oracle(tk, prec, tol):
    import torch
    X, meta, cfg = config_inputs("small_5y_16x32")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    w = _coslat(16, 32)
    h = tk.Handle()
    h.set_grid_weights(torch.from_numpy(w).cuda())
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, precision=prec, handle=h)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    oidx, odist, oscore, Dt = oracle.knn_scores(X, L, k, e, kk=k + 1, return_D=True, weights=w)
    M = Dt.shape[0]
    check_rows(np.arange(M), idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(), Dt,
               oidx, odist, oscore, M, k, e, tol)
    # weights change the answer (the test is not vacuous)
    _, _, s0 = oracle.knn_scores(X, L, k, e)
    assert np.max(np.abs(s0 - oscore) / oscore) > 1e-2
    h.close()


def test_weights_with_another_grid_size_are_refused(tk):
    import torch
    h = tk.Handle()
    h.set_grid_weights(torch.ones(100, device="cuda"))
    X, _ = make_slp_like(200, 4, 5, seed=1)
    with pytest.raises(tk.TrakNNError) as ei:
        tk.knn_scores(torch.from_numpy(X).cuda(), 3, 4, 2, handle=h)
    assert ei.value.status == 1
    h.set_grid_weights(None)
    tk.knn_scores(torch.from_numpy(X).cuda(), 3, 4, 2, handle=h)
    h.close()


def test_weighted_adjoint_matches_oracle(tk):
    import torch
    X, _ = make_slp_like(400, 16, 32, seed=21)
    w = _coslat(16, 32)
    L, k = 5, 6
    h = tk.Handle()
    h.set_grid_weights(torch.from_numpy(w).cuda())
    Xd = torch.from_numpy(X).cuda()
    idx, _, _ = tk.knn_scores(Xd, L, k, L - 1, handle=h)
    g = torch.linspace(0.5, 1.5, idx.shape[0], device="cuda")
    dX = tk.score_backward(Xd, L, k, idx, g, handle=h)
    torch.cuda.synchronize()
    ref = oracle.score_grad(X, L, k, idx.cpu().numpy(), g.cpu().numpy().astype(np.float64),
                            weights=w)
    got = dX.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-4 * scale
    h.close()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_knn_stats_match_oracle(tk, prec):
    import torch
    X, _ = make_slp_like(700, 9, 14, seed=33)
    L, k, e = 4, 20, 3
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, precision=prec)
    pre, lid = tk.knn_stats(dist, k_id=20)
    torch.cuda.synchronize()
    pre, lid, gd = pre.cpu().numpy(), lid.cpu().numpy(), dist.cpu().numpy()
    # the kernel's arithmetic on its own input lists: FP64 prefix means, FP64 logs
    ref_pre = np.cumsum(gd.astype(np.float64), axis=1) / np.arange(1, k + 1)
    assert np.allclose(pre, ref_pre, rtol=1e-6, atol=0)
    assert np.allclose(lid, oracle.local_id(gd, 20), rtol=1e-5, equal_nan=True)
    assert np.allclose(pre[:, -1], score.cpu().numpy(), rtol=1e-6)
    # against the oracle's own neighbour search
    tol = 2e-4 if prec == "split_bf16" else 1e-5
    opre = oracle.prefix_scores(X, L, k, e)
    assert np.max(np.abs(pre - opre) / opre) <= tol
    _, odist, _ = oracle.knn_scores(X, L, k, e)
    olid = oracle.local_id(odist, 20)
    assert np.max(np.abs(lid - olid) / olid) <= 50 * tol


def test_knn_stats_local_id_for_smaller_k_and_errors(tk):
    import torch
    d = torch.tensor([[1.0, 4.0, 9.0, 16.0], [0.0, 1.0, 2.0, 3.0], [2.0, 2.0, 2.0, 2.0]],
                     device="cuda")
    _, lid = tk.knn_stats(d, k_id=3, prefix=False)
    lid = lid.cpu().numpy()
    assert lid[0] == pytest.approx(2.0 / np.log(4.5), rel=1e-6)
    assert np.isnan(lid[1]) and np.isnan(lid[2])
    with pytest.raises(tk.TrakNNError):
        tk.knn_stats(d, k_id=5)
    with pytest.raises(tk.TrakNNError):
        tk.knn_stats(d, k_id=None, prefix=False)


def test_weights_apply_to_batched_and_multi_calls(tk):
    """Grid weights set on a handle act on every forward entry point: the batched and
    the several-settings calls agree with weighted single calls."""
    import torch
    w = _coslat(9, 14)
    h = tk.Handle()
    h.set_grid_weights(torch.from_numpy(w).cuda())
    Xs = [torch.from_numpy(make_slp_like(n, 9, 14, seed=70 + n)[0]).cuda() for n in (600, 900)]
    singles = [tk.knn_scores(X, 4, 8, 3, handle=h, embed="never") for X in Xs]
    batched = tk.knn_scores_batched([(X, 4, 8, 3) for X in Xs], handle=h)
    multi = tk.knn_scores_multi(Xs[1], [(4, 8, 3), (2, 6, 1)], handle=h)
    single_l2 = tk.knn_scores(Xs[1], 2, 6, 1, handle=h, embed="never")
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    for ref, got in zip(singles, batched):
        for a, b in zip(ref, got):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    for ref, got in ((singles[1], multi[0]), (single_l2, multi[1])):
        rd, gd = ref[1].cpu().numpy(), got[1].cpu().numpy()
        assert np.max(np.abs(rd - gd) / rd) <= 1e-6
        assert np.allclose(ref[2].cpu().numpy(), got[2].cpu().numpy(), rtol=1e-6)
    # and the weights matter
    h.set_grid_weights(None)
    plain = tk.knn_scores(Xs[0], 4, 8, 3, handle=h)
    torch.cuda.synchronize()
    assert not np.allclose(plain[2].cpu().numpy(), singles[0][2].cpu().numpy(), rtol=1e-3)
    h.close()
