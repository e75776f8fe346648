"""Splitting one evaluation's uv points over ranks: world_size-2 gloo ranks on
the CPU, each evaluating its share with the oracle; the exchanged total must
equal the oracle's chi-square of the whole observation."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1709_06999_gb300 import shard, synth


def test_shard_bounds_cover_exactly():
    for M in (0, 1, 5, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(M, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == M
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)


def test_combine_is_order_independent_and_exact():
    rng = np.random.default_rng(0)
    parts = list(rng.standard_normal(7) * 10.0 ** rng.integers(-8, 8, 7))
    assert shard.combine(parts) == math.fsum(parts)
    assert shard.combine(parts[::-1]) == shard.combine(parts)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = synth.small_image_problem(nxy=64, M=5_001, seed=4)
    vis = oracle.sample_image(p.image, p.dxy, p.u, p.v, p.dRA, p.dDec, p.PA)
    re, im = vis.real + p.noise_re, vis.imag + p.noise_im
    scale = 1.0 + 0.01 * np.cos(np.arange(p.u.size))   # observed != model

    def local(lo, hi):
        return oracle.chi2_image(p.image * 1.01, p.dxy, p.u[lo:hi], p.v[lo:hi],
                                 (re * scale)[lo:hi], im[lo:hi], p.w[lo:hi], p.dRA, p.dDec, p.PA)

    total = shard.sharded_chi2(local, p.u.size)
    q.put((rank, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_the_whole_sum():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = synth.small_image_problem(nxy=64, M=5_001, seed=4)
    vis = oracle.sample_image(p.image, p.dxy, p.u, p.v, p.dRA, p.dDec, p.PA)
    re, im = vis.real + p.noise_re, vis.imag + p.noise_im
    scale = 1.0 + 0.01 * np.cos(np.arange(p.u.size))
    whole = oracle.chi2_image(p.image * 1.01, p.dxy, p.u, p.v, re * scale, im, p.w, p.dRA,
                              p.dDec, p.PA)
    assert got[0] == got[1]                              # every rank gets the same total
    assert abs(got[0] - whole) <= 1e-12 * abs(whole)


def _bench_rank(rank, world, port, q):
    """bench.shard_loop, the timed loop of `bench.py --mode shard`, on a gloo
    rank: each step evaluates this rank's share with the oracle (another
    model amplitude per step) and the partials go through the loop's exchange."""
    import sys
    import torch
    import torch.distributed as dist
    import oracle
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = synth.small_image_problem(nxy=64, M=4_003, seed=8)
    lo, hi = shard.shard_bounds(p.u.size, world, rank)
    flushed = []

    def local(i):
        c = oracle.chi2_image(p.image * (1.0 + 0.1 * i), p.dxy, p.u[lo:hi], p.v[lo:hi],
                              p.noise_re[lo:hi], p.noise_im[lo:hi], p.w[lo:hi], p.dRA, p.dDec,
                              p.PA)
        return torch.tensor(c, dtype=torch.float64)

    totals = bench.shard_loop(local, 3, world, torch.device("cpu"), before=flushed.append)
    q.put((rank, totals, flushed))
    dist.destroy_process_group()


def test_bench_shard_loop_two_gloo_ranks():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = {r: (t, f) for r, t, f in (q.get(timeout=120) for _ in procs)}
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = synth.small_image_problem(nxy=64, M=4_003, seed=8)
    assert got[0][0] == got[1][0]                        # the same totals on both ranks
    assert got[0][1] == got[1][1] == [0, 1, 2]           # the flush hook ran before each step
    for i, total in enumerate(got[0][0]):
        whole = oracle.chi2_image(p.image * (1.0 + 0.1 * i), p.dxy, p.u, p.v, p.noise_re,
                                  p.noise_im, p.w, p.dRA, p.dDec, p.PA)
        assert abs(total - whole) <= 1e-12 * abs(whole)


@pytest.mark.gpu
def test_sharded_observation_on_one_gpu_rank():
    """World size 1 on the GPU: the sharded call equals the plain call."""
    import torch
    import torch.distributed as dist
    from paper_1709_06999_gb300 import Context
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        ctx = Context(0)
        p = synth.small_image_problem(nxy=128, M=20_000, seed=6)
        d = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
        t = [d(a) for a in (p.u, p.v, p.noise_re, p.noise_im, p.w)]
        so = shard.ShardedObservation(ctx, *t)
        img = d(p.image)
        got = so.chi2_image(img, p.dxy, p.dRA, p.dDec, p.PA)
        want = ctx.chi2_image(img, p.dxy, ctx.register(*t), p.dRA, p.dDec, p.PA).item()
        assert got == want
    finally:
        dist.destroy_process_group()
