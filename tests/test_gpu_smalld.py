"""The small-grid form (fields reduced to a few dozen values, as the paper's case
study reduces sea-level pressure to its leading principal components, Sec. 5):
trajectory-embedded operands, whose Gram entries are whole window sums of Eq. 2,
against the FP64 oracle at full length and against the diagonal-sum form."""
import numpy as np
import pytest

from parity import check_full, check_sampled, structural_rows, tc_unit_bounds
from synth import make_slp_like

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _run(tk, X, L, k, e, **kw):
    import torch
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, **kw)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    return idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy()


@pytest.fixture(scope="module")
def small_d_75y():
    # 75 years of 32-value fields (4 x 8 grid), the annual cycle removed
    X, meta = make_slp_like(27394, 4, 8, seed=20260310, annual_amp=5.0)
    return X, meta


@pytest.mark.parametrize("embed", ["auto", "never"])
def test_small_d_75y_sampled_rows(tk, small_d_75y, embed):
    """N = 27,394 days of D = 32 values, L = 5, k = 20: the first and last row of every
    strip (128 rows with embedded operands, 124 without), the unit edges and 500
    random rows against the oracle."""
    X, meta = small_d_75y
    L, k, e = 5, 20, 4
    idx, dist, score = _run(tk, X, L, k, e, embed=embed)
    M = X.shape[0] - L + 1
    Lg = 1 if embed == "auto" else L  # strip geometry of the form that ran
    rows = structural_rows(M, L, n_random=500, seed=5, col_bounds=tc_unit_bounds(M, Lg),
                           rows_per_strip=128 - (Lg - 1))
    check_sampled(X, L, k, e, rows, idx, dist, score, TOL)


@pytest.mark.parametrize("N,h,w,L,k,e", [(2000, 2, 4, 5, 20, 4), (1500, 4, 8, 10, 10, 9),
                                         (900, 3, 3, 17, 32, 16), (700, 1, 13, 2, 5, 1),
                                         (1100, 8, 16, 3, 64, 2)])
def test_embedded_full_parity(tk, N, h, w, L, k, e):
    X, _ = make_slp_like(N, h, w, seed=3 * N + L)
    idx, dist, score = _run(tk, X, L, k, e, embed="always")
    check_full(X, L, k, e, idx, dist, score, TOL)


def test_embedded_with_grid_weights(tk):
    import torch
    import oracle
    from parity import check_rows
    X, _ = make_slp_like(800, 4, 8, seed=91)
    w = np.linspace(0.3, 1.0, 32).astype(np.float32)
    h = tk.Handle()
    h.set_grid_weights(torch.from_numpy(w).cuda())
    L, k, e = 5, 10, 4
    idx, dist, score = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, handle=h,
                                     embed="always")
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    oidx, odist, oscore, Dt = oracle.knn_scores(X, L, k, e, kk=k + 1, return_D=True, weights=w)
    M = Dt.shape[0]
    check_rows(np.arange(M), idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(), Dt,
               oidx, odist, oscore, M, k, e, TOL)
    h.close()


def test_embedded_and_window_forms_agree(tk, small_d_75y):
    """Both forms evaluate the same distances: within the tolerance, with neighbour
    sets equal except at near ties."""
    X, meta = small_d_75y
    X = X[:6000]
    a = _run(tk, X, 5, 20, 4, embed="always")
    b = _run(tk, X, 5, 20, 4, embed="never")
    rel = np.abs(a[1] - b[1]) / np.maximum(b[1], 1e-30)
    assert rel.max() <= 2 * TOL
    assert np.allclose(a[2], b[2], rtol=2 * TOL)


@pytest.mark.parametrize("N,h,w,L,k,e,embed", [(2000, 4, 8, 5, 20, 4, "always"),
                                               (1500, 3, 5, 1, 10, 0, "never"),
                                               (900, 2, 4, 10, 32, 9, "always"),
                                               (700, 6, 6, 3, 4, 2, "always")])
def test_two_epilogue_groups_equal_one(tk, N, h, w, L, k, e, embed):
    """At L = 1 (embedded operands included) two epilogue groups split every tile's
    columns; the neighbour lists, distances and scores are those of one group."""
    import torch
    X, _ = make_slp_like(N, h, w, seed=7 * N + L)
    Xd = torch.from_numpy(X).cuda()
    hd = tk.Handle()
    two = [t.cpu().numpy() for t in tk.knn_scores(Xd, L, k, e, embed=embed, handle=hd)]
    hd.set_option("epi_groups", 1)
    one = [t.cpu().numpy() for t in tk.knn_scores(Xd, L, k, e, embed=embed, handle=hd)]
    torch.cuda.synchronize()
    assert hd.sync_status() == 0
    for a, b in zip(one, two):
        assert np.array_equal(a, b)
    check_full(X, L, k, e, *two, TOL)
    hd.close()
