"""The entry point for callers that cannot allocate device memory.

traknn_knn_scores_static keeps its scratch in one fixed device array inside the
library instead of a cudaMalloc'd workspace, so that code whose device memory is
owned by another allocator, or which must avoid the synchronisation of a
cudaMalloc, can still run the forward pass. These checks call it through the C
ABI twice in a row on different problems (so the second call runs on the first
call's leftover scratch) and compare each result with the handle-based entry
point, then check that an oversized problem is refused. This file is named to
be collected last."""
import ctypes

import numpy as np
import pytest

from synth import make_slp_like

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_02059_gb300 as m
    return m


def _static_call(tk, Xd, L, k, e):
    import torch
    N, D = Xd.shape
    M = N - L + 1
    idx = torch.empty((M, k), dtype=torch.int32, device="cuda")
    dist = torch.empty((M, k), dtype=torch.float32, device="cuda")
    score = torch.empty((M,), dtype=torch.float32, device="cuda")
    rc = tk.lib().traknn_knn_scores_static(
        Xd.data_ptr(), N, D, L, k, e, idx.data_ptr(), dist.data_ptr(), score.data_ptr(),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, idx, dist, score


def test_static_scratch_matches_handle_entry_point_twice(tk):
    import torch
    problems = [(make_slp_like(1826, 16, 32, seed=41)[0], 3, 10, 2),
                (make_slp_like(1100, 9, 13, seed=42)[0], 6, 7, 5)]
    outs = []
    for X, L, k, e in problems:     # two calls in a row on different problems
        rc, idx, dist, score = _static_call(tk, torch.from_numpy(X).cuda(), L, k, e)
        assert rc == 0
        outs.append((idx, dist, score))
    torch.cuda.synchronize()
    for (X, L, k, e), (idx, dist, score) in zip(problems, outs):
        ridx, rdist, rscore = tk.knn_scores(torch.from_numpy(X).cuda(), L, k, e, precision="fp32")
        torch.cuda.synchronize()
        rel = (torch.abs(score - rscore) / torch.abs(rscore)).max().item()
        assert rel <= TOL
        assert (torch.abs(dist - rdist) / torch.abs(rdist)).max().item() <= TOL
        same = (idx == ridx).all(dim=1)
        near = (torch.abs(rdist[:, -1] - dist[:, -1]) <= TOL * rdist[:, -1])
        assert bool((same | near).all())


def test_static_scratch_refuses_oversized_problem(tk):
    import torch
    Xd = torch.zeros((6000, 2048), dtype=torch.float32, device="cuda")
    rc, *_ = _static_call(tk, Xd, 5, 10, 4)
    assert rc == 8
    assert tk.lib().traknn_status_string(8).startswith(b"problem exceeds")
