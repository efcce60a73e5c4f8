"""The benchmark's multi-rank logic on CPU: world size 2 over gloo.  Each rank
is an independent replica; the job's time is the maximum over ranks and the
value is every rank's bytes over that time."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) ms for its step and 10 - r s end to end
        got = bench.max_over_ranks(dist, [rank + 1.0, 10.0 - rank], torch.device("cpu"))
        out[rank] = got
    finally:
        dist.destroy_process_group()


def _combine_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthgraphs as sg

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank: the oracle's moments of the same graph with its own probes (seed 100 + rank)
        s, d, n = sg.erdos_renyi(300, 0.03, 4)
        ref = oracle.build_csr(s, d, n)
        z = oracle.probes(100 + rank, ref.old_id, 6)
        mine = oracle.kpm_doubled(ref, z, 20) / (ref.n * 6)
        out[rank] = bench.combine_moments(dist, mine, torch.device("cpu")).numpy().tolist()
    finally:
        dist.destroy_process_group()


def test_probe_sharded_moments_world_2():
    """Two ranks with independent probes combine into the estimate of all 12
    probes: the single-process oracle run on the two probe blocks side by side."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import oracle
    import synthgraphs as sg

    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_combine_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    s, d, n = sg.erdos_renyi(300, 0.03, 4)
    ref = oracle.build_csr(s, d, n)
    z = np.concatenate([oracle.probes(100, ref.old_id, 6), oracle.probes(101, ref.old_id, 6)], axis=1)
    want = oracle.kpm_doubled(ref, z, 20) / (ref.n * 12)
    assert res[0] == res[1]
    assert np.abs(np.array(res[0]) - want).max() < 1e-14


def test_max_over_ranks_world_2():
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == [2.0, 10.0]


def test_whole_job_value_and_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, [3.0, 4.0], torch.device("cpu")) == [3.0, 4.0]
    # two replicas each moving 1 GB in the slowest rank's 0.5 s: 4 GB/s whole-job
    assert bench.whole_job_gbs(2, 1e9, 0.5) == 4.0
