"""The N > 1 path of bench.py on the CPU: world size 2 over gloo.

The path does not shard (every rank runs one replica of the step; there is no
data-path collective), so what multi-rank code exists is host logic: the
job's time is the maximum over ranks (one all-reduce of a scalar), the value
is the whole job's throughput, and the reference arm runs on rank 0 alone.

The arithmetic a sharded form would rest on is checked too: chi0 summed
over k-point shards by one all-reduce equals chi0 over all k (the oracle's
chi0 on each rank's shard).
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank            # rank 1 is the slower replica
        got = bench.max_over_ranks(ms, dist, "cpu")
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 125.0, 1: 125.0}


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle as O
    from synth import cfg_tiny, make_system
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = make_system(cfg_tiny(seed=51, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(12, 12, 12), ng=9,
                                 n_occ=3, n_bands=6, npw_target=20, a=6.0, freqs=(0.3j, 2.0j), eta=0.0))
        G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
        mine = O.chi0_tr(s, 0, G, s.freqs, s.eta, ks=range(rank, s.nk, world))   # k points rank, rank+world, ...
        t = torch.from_numpy(np.ascontiguousarray(mine))
        parts = torch.view_as_real(t).contiguous()
        dist.all_reduce(parts, op=dist.ReduceOp.SUM)
        if rank == 0:
            full = O.chi0_tr(s, 0, G, s.freqs, s.eta)
            summed = torch.view_as_complex(parts).numpy()
            q.put(float(np.abs(summed - full).max() / np.abs(full).max()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_k_shards_summed_by_all_reduce_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert q.get(timeout=10) < 1e-13


def test_single_rank_and_whole_job_value():
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    f = bench.chi0_flops(1000, 1507328, 32)
    one = bench.whole_job_tflops(1, f, 1000.0)
    assert bench.whole_job_tflops(2, f, 1000.0) == pytest.approx(2 * one)
    assert one == pytest.approx(f / 1.0 / 1e12)


def test_reference_arm_runs_on_rank_0_only():
    import argparse
    import bench
    args = argparse.Namespace(kgrid=None, nw=32, steps=1, warmup=0, real_axis=False, ppa=0, bg_terminator=None)
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(args, 1, 2)       # a rank other than 0: no work, no output
    assert out.getvalue() == ""
