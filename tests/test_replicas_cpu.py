"""The multi-GPU path of bench.py is replicas only (codewords are independent; no data-path
collective).  Its host logic, run here as two gloo ranks on the CPU: every rank decodes
distinct seeded inputs of the same shape, the job's time is the slowest rank's, and the
reported value counts the work of all ranks."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # distinct inputs per rank, same shapes
        w, B, Z, frames = bench.workload_frames("flood_n648_b128", rank)
        digest = torch.tensor([float(np.abs(frames[0][2]).sum()), float(frames[0][1].sum())], dtype=torch.float64)
        got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(got, digest)
        # the job's time is the slowest rank's
        t = bench.reduce_max(dist, 1.0 + rank, None)
        out.put((rank, [g.tolist() for g in got], t, frames[0][2].shape))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    digests = res[0][1]
    assert digests[0] != digests[1]                      # rank-offset seeds: different LLRs and codewords
    assert all(r[2] == float(world) for r in res)        # every rank sees the slowest rank's time
    assert res[0][3] == res[1][3]                        # the same per-rank workload shape


def test_whole_job_value_counts_all_ranks():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    one = bench.whole_job_gbps(1, 57344, 972, 0.01)
    assert abs(bench.whole_job_gbps(4, 57344, 972, 0.01) - 4 * one) < 1e-9
    assert bench.reduce_max(None, 3.5) == 3.5
