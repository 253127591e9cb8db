"""The entry point for callers that cannot allocate device memory.

traknn_knn_scores_static keeps its scratch in one fixed device array inside the
library instead of a cudaMalloc'd workspace, so that code whose device memory is
owned by another allocator, or which must avoid the synchronisation of a
cudaMalloc, can still run the forward pass. These checks call it through the C
ABI twice in a row on different problems (so the second call runs on the first
call's leftover scratch) and compare each result with the handle-based entry
point; check that a repeated call leaves the device's free memory unchanged; run
a problem sized just under the documented scratch limit and refuse one just over
it. This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

from synth import make_slp_like

pytestmark = pytest.mark.gpu
TOL = 1e-5
LIMIT = 32 << 20  # bytes of the library's fixed scratch array


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _a(x):
    return (x + 255) // 256 * 256


def static_bytes(N, D, L, k):
    """Scratch bytes of a problem, by the formula documented in include/traknn.h."""
    M = N - L + 1
    Dp = (D + 31) // 32 * 32
    c = min(8, M)
    C = -(-M // -(-M // c))
    return (_a(256 * D) + _a(4 * D) + _a(8 * N) + _a(4 * M) + _a(4 * N * Dp)
            + 2 * _a(4 * M * C * k) + 256)


def _outs(N, L, k):
    import torch
    M = N - L + 1
    return (torch.empty((M, k), dtype=torch.int32, device="cuda"),
            torch.empty((M, k), dtype=torch.float32, device="cuda"),
            torch.empty((M,), dtype=torch.float32, device="cuda"))


def _static_call(tk, Xd, L, k, e, outs=None):
    import torch
    N, D = Xd.shape
    idx, dist, score = outs if outs is not None else _outs(N, L, k)
    rc = tk.lib().traknn_knn_scores_static(
        Xd.data_ptr(), N, D, L, k, e, idx.data_ptr(), dist.data_ptr(), score.data_ptr(),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, idx, dist, score


def _matches_handle_path(tk, Xd, L, k, e, idx, dist, score):
    import torch
    ridx, rdist, rscore = tk.knn_scores(Xd, L, k, e, precision="fp32")
    torch.cuda.synchronize()
    assert (torch.abs(score - rscore) / torch.abs(rscore)).max().item() <= TOL
    assert (torch.abs(dist - rdist) / torch.abs(rdist)).max().item() <= TOL
    same = (idx == ridx).all(dim=1)
    near = (torch.abs(rdist[:, -1] - dist[:, -1]) <= TOL * rdist[:, -1])
    assert bool((same | near).all())


def test_static_scratch_matches_handle_entry_point_twice(tk):
    import torch
    problems = [(make_slp_like(1826, 16, 32, seed=41)[0], 3, 10, 2),
                (make_slp_like(1100, 9, 13, seed=42)[0], 6, 7, 5)]
    Xds = [torch.from_numpy(X).cuda() for X, _, _, _ in problems]
    outs = []
    # two calls in a row on different problems: the first through the C ABI, the
    # second through the Python wrapper (which calls the same entry point)
    rc, idx, dist, score = _static_call(tk, Xds[0], *problems[0][1:])
    assert rc == 0
    outs.append((idx, dist, score))
    outs.append(tk.knn_scores_static(Xds[1], *problems[1][1:]))
    torch.cuda.synchronize()
    for Xd, (X, L, k, e), (idx, dist, score) in zip(Xds, problems, outs):
        _matches_handle_path(tk, Xd, L, k, e, idx, dist, score)


def test_static_call_allocates_no_device_memory(tk):
    """After a warm-up call (which may load the library's device code and its array),
    a further call leaves the device's free memory exactly as it was."""
    import torch
    X, _ = make_slp_like(1500, 12, 20, seed=43)
    Xd = torch.from_numpy(X).cuda()
    outs = _outs(1500, 4, 8)
    assert _static_call(tk, Xd, 4, 8, 3, outs)[0] == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _static_call(tk, Xd, 4, 8, 3, outs)[0] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _matches_handle_path(tk, Xd, 4, 8, 3, *outs)


def _largest_fitting_N(D, L, k):
    N = 64
    while static_bytes(N + 1, D, L, k) <= LIMIT:
        N += 1
    return N


def test_static_scratch_limit_is_exact(tk):
    """A problem sized by the documented formula to sit just under the limit runs and
    matches the handle path; one more day is refused before any work."""
    import torch
    D, L, k, e = 512, 3, 10, 2
    N = _largest_fitting_N(D, L, k)
    assert LIMIT - static_bytes(N, D, L, k) < 4096
    X, _ = make_slp_like(N + 1, 16, 32, seed=44)
    Xd = torch.from_numpy(X).cuda()
    rc, idx, dist, score = _static_call(tk, Xd[:N], L, k, e)
    assert rc == 0
    torch.cuda.synchronize()
    _matches_handle_path(tk, Xd[:N].contiguous(), L, k, e, idx, dist, score)
    assert static_bytes(N + 1, D, L, k) > LIMIT
    rc, *_ = _static_call(tk, Xd, L, k, e)
    assert rc == 8


def test_static_scratch_refuses_oversized_problem(tk):
    import torch
    Xd = torch.zeros((6000, 2048), dtype=torch.float32, device="cuda")
    rc, *_ = _static_call(tk, Xd, 5, 10, 4)
    assert rc == 8
    assert tk.lib().traknn_status_string(8).startswith(b"problem exceeds")
