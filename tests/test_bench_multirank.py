"""Host-side logic of the multi-process benchmark (weak scaling: every rank solves its
own series, no collective on the data path): max-over-ranks timing, whole-job
aggregation and per-rank inputs, run as two `gloo` ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    from synth import config_inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        bench.barrier(ws)
        ms = 10.0 + 5.0 * rank  # this rank's step time
        slowest = bench.reduce_max(ms, ws)
        value = bench.aggregate(1e9, slowest, ws)
        X, _, _ = config_inputs("small_5y_16x32", seed_offset=rank)
        out[rank] = (slowest, value, float(X[:4, :4].sum()))
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ws = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    # every rank sees the slowest rank's time, and the value counts both ranks' pairs
    for r in range(ws):
        assert res[r][0] == pytest.approx(15.0)
        assert res[r][1] == pytest.approx(2 * 1e9 / 15e-3)
    # the ranks solve different series
    assert res[0][2] != res[1][2]


def test_single_process_helpers():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(2e8, 4.0, 1) == pytest.approx(5e10)
    clocks = bench.parse_clocks("0, 1800, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, "
                                "Active\n0, 1900, 2070, 950, 0x4, Not Active, Not Active, "
                                "Not Active, Not Active\n")
    assert clocks["sm_max_mhz"] == 2070.0
    assert clocks["reasons"] == ["sw_power_cap"]
    assert clocks["sm_mhz"] == pytest.approx(np.median([1800.0, 1900.0]))
