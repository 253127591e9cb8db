"""Several (L, k, exclusion) settings of one record in one Gram sweep: every setting
agrees with its own single call and passes parity with the FP64 oracle.

The shared sweep sizes strips and tiles for the largest L, so a pair (t, j) may be
evaluated from the other operand order than in the single call (D(t,j) from the
Gram tile of j's rows); the split-BF16 products are then accumulated in another
order, and distances may differ in the last bits. Distances therefore agree to
1e-6 and neighbour sets may differ only at near ties, as between the symmetric
and the full evaluation."""
import ctypes

import numpy as np
import pytest

from parity import check_full
from synth import make_slp_like

pytestmark = pytest.mark.gpu

SETTINGS = [(3, 10, 2), (5, 20, 4), (10, 5, 9), (2, 8, 1), (7, 12, 6)]


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _agree(ref, got, k):
    ri, rd, rs = (x.cpu().numpy() for x in ref)
    gi, gd, gs = (x.cpu().numpy() for x in got)
    rel = np.abs(rd - gd) / np.maximum(np.abs(rd), 1e-30)
    assert rel.max() <= 1e-6
    assert np.allclose(rs, gs, rtol=1e-6, atol=0)
    for t in np.nonzero(~(ri == gi).all(axis=1))[0]:
        # a differing row must be a near tie at the k-th distance
        assert abs(gd[t][-1] - rd[t][-1]) <= 1e-6 * rd[t][-1], t
        assert len(set(ri[t]) ^ set(gi[t])) <= 2 * k


@pytest.mark.parametrize("symmetric", [True, False])
def test_each_setting_agrees_with_its_single_call(tk, symmetric):
    import torch
    X, _ = make_slp_like(1500, 9, 14, seed=41)
    Xd = torch.from_numpy(X).cuda()
    got = tk.knn_scores_multi(Xd, SETTINGS, symmetric=symmetric)
    torch.cuda.synchronize()
    assert tk.get_handle().sync_status() == 0
    for (L, k, e), g in zip(SETTINGS, got):
        ref = tk.knn_scores(Xd, L, k, e, symmetric=symmetric, embed="never")
        torch.cuda.synchronize()
        _agree(ref, g, k)


def test_multi_parity_with_oracle(tk):
    import torch
    X, _ = make_slp_like(900, 16, 32, seed=43)
    got = tk.knn_scores_multi(torch.from_numpy(X).cuda(), SETTINGS[:3])
    torch.cuda.synchronize()
    for (L, k, e), (idx, dist, score) in zip(SETTINGS[:3], got):
        check_full(X, L, k, e, idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(), 2e-4)


def test_multi_with_segments(tk):
    """K segments folded through the scratch while every tile is scanned once per
    setting: agreement with the single calls and parity with the oracle."""
    import torch
    X, _ = make_slp_like(700, 40, 60, seed=45)  # D = 2,400
    Xd = torch.from_numpy(X).cuda()
    h = tk.get_handle()
    try:
        h.set_option("segment_k", 512)
        got = tk.knn_scores_multi(Xd, SETTINGS[:4], handle=h)
        refs = [tk.knn_scores(Xd, L, k, e, handle=h, embed="never") for L, k, e in SETTINGS[:4]]
        torch.cuda.synchronize()
        assert h.sync_status() == 0
    finally:
        h.set_option("segment_k", 0)
    for (L, k, e), ref, g in zip(SETTINGS[:4], refs, got):
        _agree(ref, g, k)
    L, k, e = SETTINGS[1]
    idx, dist, score = got[1]
    check_full(X, L, k, e, idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy(), 2e-4)


def test_settings_of_different_records_are_refused(tk):
    import torch
    X1 = torch.from_numpy(make_slp_like(300, 4, 5, seed=1)[0]).cuda()
    X2 = torch.from_numpy(make_slp_like(300, 4, 5, seed=2)[0]).cuda()
    out = [(torch.empty((298, 4), dtype=torch.int32, device="cuda"),
            torch.empty((298, 4), device="cuda"), torch.empty((298,), device="cuda"))
           for _ in range(2)]
    arr = (tk.Series * 2)()
    for b, X in enumerate((X1, X2)):
        arr[b] = tk.Series(X.data_ptr(), 300, 3, 4, 2, out[b][0].data_ptr(),
                           out[b][1].data_ptr(), out[b][2].data_ptr())
    rc = tk.lib().traknn_knn_scores_multi(tk.get_handle()._h, ctypes.cast(arr, ctypes.c_void_p),
                                          2, 20, None)
    assert rc == 1


def test_multi_single_product_bf16(tk):
    """The single-product BF16 form through the several-settings call agrees with its
    single calls."""
    import torch
    X, _ = make_slp_like(800, 9, 14, seed=47)
    Xd = torch.from_numpy(X).cuda()
    got = tk.knn_scores_multi(Xd, SETTINGS[:3], precision="bf16")
    refs = [tk.knn_scores(Xd, L, k, e, precision="bf16", embed="never")
            for L, k, e in SETTINGS[:3]]
    torch.cuda.synchronize()
    for (L, k, e), ref, g in zip(SETTINGS[:3], refs, got):
        _agree(ref, g, k)
