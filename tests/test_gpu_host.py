"""The host-buffer entry point (copies X in, computes, copies the results out and
synchronises): its results equal the device-buffer entry point's and pass parity
with the FP64 oracle, for pinned and for pageable host buffers."""
import numpy as np
import pytest

from parity import check_full
from synth import config_inputs, make_slp_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_host_entry_equals_device_entry(tk, pinned, prec):
    import torch
    X, _ = make_slp_like(1200, 12, 20, seed=61)
    L, k, e = 5, 12, 4
    Xh = torch.from_numpy(X)
    if pinned:
        Xh = Xh.pin_memory()
    hidx, hdist, hscore = tk.knn_scores_host(Xh, L, k, e, precision=prec)
    didx, ddist, dscore = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, precision=prec)
    torch.cuda.synchronize()
    assert not hidx.is_cuda and not hscore.is_cuda
    assert np.array_equal(hidx.numpy(), didx.cpu().numpy())
    assert np.array_equal(hdist.numpy(), ddist.cpu().numpy())
    assert np.array_equal(hscore.numpy(), dscore.cpu().numpy())


def test_host_entry_parity_with_oracle(tk):
    import torch
    X, meta, cfg = config_inputs("small_5y_16x32")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    idx, dist, score = tk.knn_scores_host(torch.from_numpy(X).pin_memory(), L, k, e)
    check_full(X, L, k, e, idx.numpy(), dist.numpy(), score.numpy(), 2e-4)


def test_host_entry_rejects_bad_shapes_without_work(tk):
    import torch
    h = tk.get_handle()
    n0 = h.launch_count()
    X = torch.zeros((10, 4))
    with pytest.raises(tk.TrakNNError) as ei:
        tk.knn_scores_host(X, 3, 9, 2, handle=h)  # 8 trajectories cannot have 9 neighbours
    assert ei.value.status == 2
    assert h.launch_count() == n0


def test_host_entry_equals_device_entry_75y(tk):
    """The 75-year workload through host buffers takes the phased sequence (the strips of
    the last 35 % of the days run while the earlier days are copied in): its results
    equal the device entry point's bit for bit."""
    import torch
    X, meta, cfg = config_inputs("euro_75y_46x81")
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    hidx, hdist, hscore = tk.knn_scores_host(torch.from_numpy(X).pin_memory(), L, k, e)
    didx, ddist, dscore = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e)
    torch.cuda.synchronize()
    assert np.array_equal(hidx.numpy(), didx.cpu().numpy())
    assert np.array_equal(hdist.numpy(), ddist.cpu().numpy())
    assert np.array_equal(hscore.numpy(), dscore.cpu().numpy())


def test_host_entry_with_grid_weights(tk):
    import torch
    X, _ = make_slp_like(2500, 12, 20, seed=63)
    w = torch.linspace(0.2, 1.0, 240, device="cuda")
    h = tk.Handle()
    h.set_grid_weights(w)
    hres = tk.knn_scores_host(torch.from_numpy(X).pin_memory(), 5, 10, 4, handle=h)
    dres = tk.knn_scores(torch.from_numpy(X).cuda(), 5, 10, 4, handle=h)
    torch.cuda.synchronize()
    for a, b in zip(hres, dres):
        assert np.array_equal(a.numpy(), b.cpu().numpy())
    h.close()


@pytest.mark.parametrize("N,h,w,L,k,e,weights", [(9000, 12, 20, 5, 10, 4, False),
                                                  (8000, 8, 12, 17, 32, 16, False),
                                                  (12000, 10, 16, 3, 20, 2, True)])
def test_host_entry_phases_equal_device_entry(tk, N, h, w, L, k, e, weights):
    """Series long enough to be split into phases (first phase: the strips of the last
    35 % of the days, at least the 4,096 days the centring mean reads): bitwise equal to
    the device entry point, with and without grid-point weights and at the longest L."""
    import torch
    X, _ = make_slp_like(N, h, w, seed=N + L)
    hd = tk.Handle()
    if weights:
        hd.set_grid_weights(torch.linspace(0.3, 1.0, h * w, device="cuda"))
    hres = tk.knn_scores_host(torch.from_numpy(X).pin_memory(), L, k, e, handle=hd)
    dres = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, handle=hd)
    torch.cuda.synchronize()
    assert hd.sync_status() == 0
    for a, b in zip(hres, dres):
        assert np.array_equal(a.numpy(), b.cpu().numpy())
    hd.close()
