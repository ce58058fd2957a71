"""The multi-GPU path is replicas only: each rank decodes its own frames (no
collective in the data path) and the job time is the slowest rank's.  These
host-side pieces run here as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2507_03509_gb300 import gen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        code = gen.workload_code(1)
        F = 3
        fr = gen.workload_frames(1, code, frames=F, first=bench.shard_first_frame(rank, F))
        local_ms = 10.0 + 5.0 * rank
        job = bench.job_time_ms(local_ms, dist, "cpu")
        out.put((rank, fr.llr[:, :8].copy(), job,
                 bench.job_value_mbit_s(code.n, F, 2, world, job)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    code = gen.workload_code(1)
    whole = gen.workload_frames(1, code, frames=6)
    # rank r decodes frames 3r .. 3r+2 of the workload, disjoint and complete
    assert np.array_equal(res[0][1], whole.llr[0:3, :8]) and np.array_equal(res[1][1], whole.llr[3:6, :8])
    # both ranks report the slowest rank's time (15 ms) and the whole job's bits
    assert res[0][2] == res[1][2] == 15.0
    assert res[0][3] == pytest.approx(code.n * 3 * 2 * 2 / 15e-3 / 1e6)
