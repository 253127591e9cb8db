"""The adjoint d(sum_t g_t s_t)/dX with the neighbour sets held fixed (CUDA kernel,
through the C ABI) against the FP64 oracle, central finite differences and torch
FP64 autograd through the definition (Eq. 1-3)."""
import numpy as np
import pytest

import oracle
from synth import config_inputs, make_slp_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _forward_backward(tk, X, L, k, e, g, prec="split_bf16"):
    import torch
    Xd = torch.from_numpy(X).cuda()
    idx, dist, score = tk.knn_scores(Xd, L, k, e, precision=prec)
    dX = tk.score_backward(Xd, L, k, idx, torch.from_numpy(g.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    return idx.cpu().numpy(), dist.cpu().numpy(), dX.cpu().numpy()


def _assert_close(got, ref, rtol):
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= rtol * scale
    big = np.abs(ref) > 1e-2 * scale
    assert (np.abs(got[big] - ref[big]) / np.abs(ref[big])).max() <= 50 * rtol


@pytest.mark.parametrize("N,h,w,L,k,e", [(60, 1, 7, 3, 4, 2), (400, 6, 9, 5, 10, 4),
                                         (333, 3, 5, 1, 3, 0), (250, 4, 4, 8, 6, 0)])
def test_matches_oracle_closed_form(tk, N, h, w, L, k, e):
    X, _ = make_slp_like(N, h, w, seed=N * 3 + L)
    M = N - L + 1
    g = np.random.default_rng(N).uniform(0.2, 2.0, M)
    idx, _, dX = _forward_backward(tk, X, L, k, e, g)
    ref = oracle.score_grad(X, L, k, idx, g)
    _assert_close(dX, ref, 1e-5)


def test_matches_torch_autograd_N500_D512(tk):
    torch = pytest.importorskip("torch")
    X, _ = make_slp_like(500, 16, 32, seed=500)
    L, k, e = 5, 10, 4
    M = 500 - L + 1
    g = np.ones(M)
    idx, _, dX = _forward_backward(tk, X, L, k, e, g)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    T = torch.stack([Xt[t:t + L].reshape(-1) for t in range(M)])
    Dm = ((T[:, None, :] - T[torch.tensor(idx, dtype=torch.long)]) ** 2).sum(-1)
    Dm.mean(1).sum().backward()
    _assert_close(dX, Xt.grad.numpy(), 1e-5)


def test_finite_differences_30y(tk):
    """200 random entries of the 30-year workload, away from ties: central FD
    (h = 1e-3 hPa) of the summed score, evaluated in FP64 over the pair terms that
    contain the perturbed day only. The summed score is quadratic in X when the
    neighbour sets are fixed, so FD is exact up to rounding."""
    import torch
    X, meta, cfg = config_inputs("euro_30y_46x81")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    N, D = X.shape
    M = N - L + 1
    Xd = torch.from_numpy(X).cuda()
    idx1, dist1, _ = tk.knn_scores(Xd, L, k + 1, e)
    idx1, dist1 = idx1.cpu().numpy(), dist1.cpu().numpy()
    idx = np.ascontiguousarray(idx1[:, :k])
    g = np.ones(M)
    dX = tk.score_backward(Xd, L, k, torch.from_numpy(idx).cuda(),
                           torch.ones(M, device="cuda")).cpu().numpy()
    gap = dist1[:, k] - dist1[:, k - 1]
    rev = [[] for _ in range(M)]
    for t in range(M):
        for j in idx[t]:
            rev[j].append(t)
    X64 = X.astype(np.float64)
    hstep = 1e-3
    rng = np.random.default_rng(2024)
    checked = 0
    while checked < 200:
        a, p = int(rng.integers(0, N)), int(rng.integers(0, D))
        pairs = set()
        for t in range(max(0, a - L + 1), min(a, M - 1) + 1):
            pairs.update((t, int(j)) for j in idx[t])
        for j in range(max(0, a - L + 1), min(a, M - 1) + 1):
            pairs.update((t, j) for t in rev[j])
        rows = {t for t, _ in pairs}
        # away from ties: no row's k-th/(k+1)-th gap is within reach of the perturbation
        bound = 4 * hstep * np.abs(X64[:, p] - X64[a, p]).max() + 1e-4 * dist1[:, k - 1].max()
        if any(gap[t] <= bound for t in rows):
            continue

        def F(delta):
            old = X64[a, p]
            X64[a, p] = old + delta
            s = 0.0
            for t, j in pairs:
                s += g[t] / k * ((X64[t:t + L] - X64[j:j + L]) ** 2).sum()
            X64[a, p] = old
            return s

        fd = (F(hstep) - F(-hstep)) / (2 * hstep)
        assert abs(dX[a, p] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(dX).max()), (a, p)
        checked += 1


def test_autograd_function_and_determinism(tk):
    import torch
    X, _ = make_slp_like(300, 5, 6, seed=31)
    Xd = torch.from_numpy(X).cuda().requires_grad_(True)
    s = tk.TrakNNScore.apply(Xd, 4, 5, 3)
    (s * torch.linspace(0.5, 1.5, s.numel(), device="cuda")).sum().backward()
    idx, _, _ = tk.knn_scores(Xd.detach(), 4, 5, 3)
    g = torch.linspace(0.5, 1.5, s.numel(), device="cuda")
    d1 = tk.score_backward(Xd.detach(), 4, 5, idx, g)
    d2 = tk.score_backward(Xd.detach(), 4, 5, idx, g)
    assert torch.equal(d1, d2)
    assert torch.equal(Xd.grad, d1)


def test_invalid_neighbour_index_is_reported(tk):
    import torch
    X = torch.randn(50, 4, device="cuda")
    idx = torch.zeros((48, 2), dtype=torch.int32, device="cuda")
    idx[3, 1] = 10_000
    h = tk.get_handle()
    tk.score_backward(X, 3, 2, idx, torch.ones(48, device="cuda"))
    assert h.sync_status() == 1


def test_days_with_many_incidences(tk):
    """Neighbour lists with hub trajectories: the days near trajectory 500 (chosen by
    1,500 trajectories) have between 512 and 4,096 incidences and are merged by a whole
    CTA; the days after 2,000 and 2,001 (chosen by every trajectory) have more than
    4,096 and list their incidences unmerged. Both against the oracle, and bitwise
    reproducible."""
    import torch
    N, L, k = 3000, 5, 4
    M = N - L + 1
    X, _ = make_slp_like(N, 4, 5, seed=7)
    t = np.arange(M)
    idx = np.stack([np.where(t < 1500, 500, (t + 11) % M), np.full(M, 2000), np.full(M, 2001),
                    (t + 5) % M], axis=1).astype(np.int32)
    g = np.random.default_rng(3).uniform(0.5, 1.5, M)
    Xd = torch.from_numpy(X).cuda()
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    idd = torch.from_numpy(idx).cuda()
    d1 = tk.score_backward(Xd, L, k, idd, gd)
    d2 = tk.score_backward(Xd, L, k, idd, gd)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    assert torch.equal(d1, d2)
    ref = oracle.score_grad(X, L, k, idx, g.astype(np.float32).astype(np.float64))
    _assert_close(d1.cpu().numpy(), ref, 1e-5)


@pytest.mark.parametrize("D", [64, 54])
def test_load_forms_agree_bitwise(tk, D):
    """The gather loads four grid points per thread as one 16-byte load (D a multiple
    of 4, aligned rows), as two 8-byte loads, or one point per thread, depending on D
    and the alignment of X: a copy of X placed 4 or 8 bytes past an aligned address
    takes the other forms, with the same arithmetic and so the same bits."""
    import torch
    N, L, k, e = 400, 5, 8, 4
    X, _ = make_slp_like(N, 8, D // 8, seed=D) if D % 8 == 0 else make_slp_like(N, 6, 9, seed=D)
    assert X.shape[1] == D
    Xd = torch.from_numpy(X).cuda()
    idx, _, _ = tk.knn_scores(Xd, L, k, e)
    g = torch.linspace(0.5, 1.5, N - L + 1, device="cuda")
    ref = tk.score_backward(Xd, L, k, idx, g)
    for shift in (1, 2):
        buf = torch.empty(N * D + shift, device="cuda")
        Xs = buf[shift:].view(N, D)
        Xs.copy_(Xd)
        got = tk.score_backward(Xs, L, k, idx, g)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), shift
    assert tk.get_handle().sync_status() == 0
