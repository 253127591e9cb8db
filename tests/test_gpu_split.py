"""One series split into parts (traknn_knn_partial), run one after another on one GPU,
and merged (traknn_merge_partials): the result equals the single call on the whole
series and passes parity with the FP64 oracle. (Processes that each own a GPU run
the same calls with an all-gather between them; that exchange is tested on the CPU
with gloo ranks.)"""
import numpy as np
import pytest

from parity import check_full, check_sampled, structural_rows
from synth import config_inputs, make_slp_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _split(tk, Xd, L, k, e, P):
    import torch
    parts = [tk.knn_partial(Xd, L, k, e, p, P) for p in range(P)]
    ip = torch.stack([a for a, _ in parts])
    dp = torch.stack([b for _, b in parts])
    idx, dist, score = tk.merge_partials(ip, dp)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    return idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(), ip.cpu().numpy()


def test_one_part_is_the_single_call(tk):
    import torch
    X, _ = make_slp_like(1500, 9, 14, seed=61)
    Xd = torch.from_numpy(X).cuda()
    got = _split(tk, Xd, 5, 10, 4, 1)
    ref = [t.cpu().numpy() for t in tk.knn_scores(Xd, 5, 10, 4, embed="never")]
    for a, b in zip(ref, got[:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("P", [2, 3, 5, 32])
@pytest.mark.parametrize("N,h,w,L,k,e", [(1500, 9, 14, 5, 10, 4), (900, 6, 8, 17, 20, 16),
                                         (700, 4, 5, 1, 3, 0)])
def test_parts_merge_to_oracle(tk, P, N, h, w, L, k, e):
    import torch
    X, _ = make_slp_like(N, h, w, seed=N + P)
    Xd = torch.from_numpy(X).cuda()
    idx, dist, score, ip = _split(tk, Xd, L, k, e, P)
    check_full(X, L, k, e, idx, dist, score, 2e-4)
    # every listed candidate pair belongs to its part: min(t, j) in the part's rows
    M = N - L + 1
    for p in range(P):
        lo, hi = tk.partition(M, L, P, p)
        t, i = np.nonzero(ip[p] >= 0)
        j = ip[p][t, i]
        assert np.all((np.minimum(t, j) >= lo) & (np.minimum(t, j) < hi)), p


def test_four_parts_euro_75y(tk):
    """The headline workload split into four parts: sampled rows against the oracle
    (strip boundaries, the parts' row edges, random rows)."""
    import torch
    X, meta, cfg = config_inputs("euro_75y_46x81")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    Xd = torch.from_numpy(X).cuda()
    idx, dist, score, _ = _split(tk, Xd, L, k, e, 4)
    M = X.shape[0] - L + 1
    edges = [tk.partition(M, L, 4, p)[0] for p in range(1, 4)]
    rows = structural_rows(M, L, n_random=150, seed=9, strip_every=6, col_bounds=edges)
    check_sampled(X, L, k, e, rows, idx, dist, score, 2e-4)
    ref = tk.knn_scores(Xd, L, k, e, embed="never")
    rd = ref[1].cpu().numpy()
    assert np.max(np.abs(rd - dist) / rd) <= 1e-6
