"""One series split across processes (the upper-triangle pair space of Sec. 3.3 cut
into contiguous strip ranges by traknn_partition), run as gloo ranks on the CPU.

Each rank builds its part's candidate lists from the FP64 oracle's distances (the
pairs {t, j} whose smaller index lies in its rows, the k best per row), the ranks
exchange them with the binding's gather_partials, and the union of the gathered
lists, merged by (distance, index), must give the oracle's neighbour sets. The
parts must also cover every pair exactly once."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

L, K, E = 3, 6, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from synth import make_slp_like
    X, _ = make_slp_like(300, 3, 4, seed=7)
    return X


def _part_lists(Dt, lo, hi):
    """The part's candidate lists: for every row t, the K best j with |t - j| > E and
    min(t, j) in [lo, hi), sorted by (distance, index); -1 / inf beyond."""
    M = Dt.shape[0]
    idx = np.full((M, K), -1, dtype=np.int32)
    dist = np.full((M, K), np.inf, dtype=np.float32)
    for t in range(M):
        js = [j for j in range(M) if abs(t - j) > E and lo <= min(t, j) < hi]
        js.sort(key=lambda j: (Dt[t, j], j))
        for i, j in enumerate(js[:K]):
            idx[t, i] = j
            dist[t, i] = Dt[t, j]
    return idx, dist


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    import paper_2603_02059_gb300 as tk
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        X = _problem()
        _, _, _, Dt = oracle.knn_scores(X, L, K, E, return_D=True)
        M = Dt.shape[0]
        lo, hi = tk.partition(M, L, ws, rank)
        idx, dst = _part_lists(Dt, lo, hi)
        ip, dp = tk.gather_partials(torch.from_numpy(idx), torch.from_numpy(dst))
        out[rank] = (lo, hi, ip.numpy(), dp.numpy())
    finally:
        dist.destroy_process_group()


def _merge(ip, dp):
    """Per row: the K smallest (distance, index) entries of the union of the lists."""
    P, M, k = ip.shape
    idx = np.empty((M, k), dtype=np.int64)
    for t in range(M):
        c = sorted((float(dp[p, t, i]), int(ip[p, t, i])) for p in range(P) for i in range(k)
                   if ip[p, t, i] >= 0)
        idx[t] = [j for _, j in c[:k]]
    return idx


@pytest.mark.parametrize("ws", [2, 3])
def test_split_exchange_and_merge_matches_oracle(ws):
    import oracle
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == list(range(ws))
    X = _problem()
    oidx, odist, _ = oracle.knn_scores(X, L, K, E)
    M = oidx.shape[0]
    # the parts' rows are contiguous and cover [0, M)
    bounds = [res[r][:2] for r in range(ws)]
    assert bounds[0][0] == 0 and bounds[-1][1] == M
    assert all(bounds[r][1] == bounds[r + 1][0] for r in range(ws - 1))
    # every rank gathered the same lists, in rank order
    for r in range(1, ws):
        assert np.array_equal(res[r][2], res[0][2]) and np.array_equal(res[r][3], res[0][3])
    ip, dp = res[0][2], res[0][3]
    # a candidate of row t appears in exactly one part's list
    for t in range(M):
        seen = [j for p in range(ws) for j in ip[p, t] if j >= 0]
        assert len(seen) == len(set(seen))
    got = _merge(ip, dp)
    assert np.array_equal(got, oidx.astype(np.int64))


def test_partition_covers_and_balances():
    import paper_2603_02059_gb300 as tk
    for M, L in ((27390, 5), (1000, 17), (300, 1), (130, 3)):
        R = 128 - (L - 1)
        for P in (1, 2, 3, 4, 8, 32):
            parts = [tk.partition(M, L, P, p) for p in range(P)]
            assert parts[0][0] == 0 and parts[-1][1] == M
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            work = [sum(M - t for t in range(a, b)) for a, b in parts]
            # each part is within one strip's work of an equal share
            share = M * (M + 1) / 2 / P
            assert all(abs(w - share) <= R * M for w in work), (M, L, P, work)
            for a, b in parts:  # parts start on strip boundaries
                assert a % R == 0 or a == M
    with pytest.raises(tk.TrakNNError):
        tk.partition(100, 3, 2, 2)
