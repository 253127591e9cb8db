"""Error of each precision form against the FP64 oracle, per trajectory length, on
the 0.25-degree grid (D = 58,101): the first 2,000 days of the 75-year series,
L in {3, 5, 7, 10}, k = 20, exclusion L - 1; and on the 1-degree grid (D = 3,726),
first 2,000 days of its 75-year series, L in {2, 3, 5, 10}, for one and two
tensor-core accumulation segments per Gram entry.

Prints one line per (form, L): the largest relative error of a reported distance
against the oracle's D(t, j) for the same pair, the largest relative error of a
score, and the fraction of rows whose neighbour set equals the oracle's exactly.
The split-BF16 and FP32 forms must also pass the parity rules at 2e-4 and 1e-5."""
import numpy as np
import pytest

import oracle
from parity import check_rows
from synth import config_inputs

pytestmark = pytest.mark.gpu

N_SUB = 2000
LS = (3, 5, 7, 10)
TOL = {"fp32": 1e-5, "split_bf16": 2e-4}


@pytest.fixture(scope="module")
def sub():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, meta, cfg = config_inputs("euro_75y_181x321")
    Xs = np.ascontiguousarray(X[:N_SUB])
    del X
    S = oracle.snapshot_matrix(Xs)
    return Xs, S, cfg["k"]


def _errors(gidx, gdist, gscore, D, oscore, oidx, k):
    rows = np.arange(D.shape[0])[:, None]
    true_d = D[rows, gidx.astype(np.int64)]
    derr = float(np.max(np.abs(gdist - true_d) / np.maximum(true_d, 1e-30)))
    serr = float(np.max(np.abs(gscore - oscore) / np.maximum(oscore, 1e-30)))
    same = np.mean([set(a.tolist()) == set(b[:k].tolist()) for a, b in zip(gidx, oidx)])
    return derr, serr, float(same)


@pytest.mark.parametrize("L", LS)
def test_error_per_L(sub, L):
    import torch

    import paper_2603_02059_gb300 as tk
    Xs, S, k = sub
    e = L - 1
    D = oracle.traj_matrix(S, L)
    M = D.shape[0]
    rows = np.arange(M)
    oidx, odist, oscore = oracle.knn_from_rows(D, rows, k, e, kk=k + 1)
    Xd = torch.from_numpy(Xs).cuda()
    got = {}
    h = tk.get_handle()
    try:
        for prec, seg in (("split_bf16", 65536), ("split_bf16", 8192), ("split_bf16", 0),
                          ("bf16", 0), ("fp32", 0)):
            h.set_option("segment_k", seg)
            idx, dist, score = tk.knn_scores(Xd, L, k, e, precision=prec, handle=h)
            torch.cuda.synchronize()
            assert h.sync_status() == 0
            r = (idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy())
            if seg == 0:
                got[prec] = r
            derr, serr, same = _errors(*r, D, oscore, oidx, k)
            print(f"\nprecision L={L:2d} {prec:10s} segment_k={seg or 'default'} max rel err "
                  f"dist {derr:.3e} score {serr:.3e} identical sets {same:.4f}")
    finally:
        h.set_option("segment_k", 0)
    for prec, tol in TOL.items():
        gidx, gdist, gscore = got[prec]
        check_rows(rows, gidx, gdist, gscore, D, oidx, odist, oscore, M, k, e, tol)


@pytest.fixture(scope="module")
def sub_1deg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, meta, cfg = config_inputs("euro_75y_46x81")
    Xs = np.ascontiguousarray(X[:N_SUB])
    return Xs, oracle.snapshot_matrix(Xs), cfg["k"]


@pytest.mark.parametrize("L", (2, 3, 5, 10))
def test_error_per_L_1deg(sub_1deg, L):
    import torch

    import paper_2603_02059_gb300 as tk
    Xs, S, k = sub_1deg
    e = L - 1
    D = oracle.traj_matrix(S, L)
    M = D.shape[0]
    rows = np.arange(M)
    oidx, odist, oscore = oracle.knn_from_rows(D, rows, k, e, kk=k + 1)
    Xd = torch.from_numpy(Xs).cuda()
    h = tk.get_handle()
    got = {}
    try:
        for seg in (65536, 4096, 0):
            h.set_option("segment_k", seg)
            idx, dist, score = tk.knn_scores(Xd, L, k, e, handle=h)
            torch.cuda.synchronize()
            assert h.sync_status() == 0
            got[seg] = (idx.cpu().numpy(), dist.cpu().numpy(), score.cpu().numpy())
            derr, serr, same = _errors(*got[seg], D, oscore, oidx, k)
            print(f"\nprecision D=3726 L={L:2d} split_bf16 segment_k={seg or 'default'} "
                  f"max rel err dist {derr:.3e} score {serr:.3e} identical sets {same:.4f}")
    finally:
        h.set_option("segment_k", 0)
    gidx, gdist, gscore = got[0]
    check_rows(rows, gidx, gdist, gscore, D, oidx, odist, oscore, M, k, e, TOL["split_bf16"])
