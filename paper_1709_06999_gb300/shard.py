"""One chi-square evaluation split over ranks (one GPU per rank).

The chi-square is a sum over uv points (Eq. chap6.eq:def.chi.square), so a
large observation can be divided into contiguous shares, one per rank.  Every
rank transforms the full model image (the FFT costs the same on each) and
evaluates the chi-square of its own share; the partial sums are then
exchanged once -- one double per rank -- and added in rank order, so every
rank obtains the same, reproducible total.

The exchange uses torch.distributed (NCCL on GPUs, gloo on CPU); the per-rank
evaluation is the library's chi2 call on a registered slice.
"""
from __future__ import annotations

import math

import torch


def shard_bounds(M: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of M points; shares differ by at most one."""
    if world < 1 or not 0 <= rank < world or M < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, M >= 0")
    return rank * M // world, (rank + 1) * M // world


def combine(partials) -> float:
    """Sum of the per-rank partial chi-squares in rank order, exactly rounded
    (Shewchuk's summation via math.fsum): independent of how the ranks'
    values arrived."""
    return math.fsum(float(p) for p in partials)


def exchange(partial: float, group=None) -> float:
    """All ranks contribute one double; all receive the rank-ordered total."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([partial], dtype=torch.float64, device=dev)
    parts = [torch.empty(1, dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    return combine(p.item() for p in parts)


def sharded_chi2(local_chi2, M: int, group=None) -> float:
    """Total chi-square of M points over the ranks of `group`:
    local_chi2(lo, hi) evaluates this rank's share [lo, hi)."""
    import torch.distributed as dist
    lo, hi = shard_bounds(M, dist.get_world_size(group), dist.get_rank(group))
    return exchange(float(local_chi2(lo, hi)), group)


class ShardedObservation:
    """This rank's share of an observation, registered on a Context."""

    def __init__(self, ctx, u, v, re, im, w, group=None):
        import torch.distributed as dist
        self.M = u.numel()
        self.group = group
        self.lo, self.hi = shard_bounds(self.M, dist.get_world_size(group), dist.get_rank(group))
        sl = slice(self.lo, self.hi)
        self.obs = ctx.register(u[sl], v[sl], re[sl], im[sl], w[sl])
        self.ctx = ctx

    def chi2_image(self, image, dxy, dRA=0.0, dDec=0.0, PA=0.0) -> float:
        part = self.ctx.chi2_image(image, dxy, self.obs, dRA, dDec, PA).item()
        return exchange(part, self.group)

    def chi2_profile(self, intensity, Rmin, dR, nxy, dxy, inc=0.0, dRA=0.0, dDec=0.0,
                     PA=0.0) -> float:
        part = self.ctx.chi2_profile(intensity, Rmin, dR, nxy, dxy, self.obs, inc, dRA, dDec,
                                     PA).item()
        return exchange(part, self.group)
