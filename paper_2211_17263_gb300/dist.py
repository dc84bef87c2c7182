"""Multi-process pieces of the library (one process per GPU).

* Ranks from the launcher's environment (RANK, WORLD_SIZE, LOCAL_RANK), and the two
  collectives a replica run needs: a barrier and the maximum of a value over ranks (the
  bench times every rank and reports the slowest).
* A sharded estimate of ONE job's gradient: Eq. 10's antithetic pairs are independent,
  so rank s computes a contiguous block of pairs [b_s, b_s + P_s) -- with their global
  draw indices and path-stream fields (prdpt_grad_opts.pair_begin), hence exactly the
  renders a single process would compute -- and the only exchange is an all-reduce of
  the D-vector sum_s (P_s / P) g_s, plus an all-gather of the per-render losses.

The collectives run on whatever process group is initialised (NCCL between GPUs, gloo on
CPU); nothing here touches the device except through the tensors it is given.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env_rank() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    def get(name, default):
        try:
            return int(os.environ.get(name, default))
        except ValueError:
            return default
    return get("RANK", 0), get("WORLD_SIZE", 1), get("LOCAL_RANK", 0)


def barrier(world: int) -> None:
    if world > 1:
        dist.barrier()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The maximum of a per-rank value (e.g. a step time) over all ranks."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(pairs: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block of pairs of `rank`: (first pair, number of pairs); blocks follow
    rank order, cover [0, pairs) exactly and differ in size by at most one."""
    base, extra = divmod(pairs, world)
    count = base + (1 if rank < extra else 0)
    begin = rank * base + min(rank, extra)
    return begin, count


def sharded_estimate(local_fn, pairs: int, D: int, group=None, device=None):
    """Eq. 10 over `pairs` antithetic pairs split across the ranks of `group`.

    local_fn(pair_begin, count) -> (grad [D], losses [2 count]) computes this rank's block
    (the mean over its pairs). Returns (grad [D] float64, losses [2 pairs] float64) on
    every rank: g = sum_s (P_s / P) g_s by one all-reduce, losses gathered in pair order.
    """
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    begin, count = shard(pairs, world, rank)
    g = torch.zeros(D, dtype=torch.float64, device=device)
    losses = torch.zeros(2 * count, dtype=torch.float64, device=device)
    if count > 0:
        gl, ll = local_fn(begin, count)
        g = torch.as_tensor(gl, dtype=torch.float64, device=device) * (count / pairs)
        losses = torch.as_tensor(ll, dtype=torch.float64, device=device).reshape(-1)
    if world == 1:
        return g, losses
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    # losses: every rank's block, padded to the largest, gathered in rank (= pair) order
    cmax = shard(pairs, world, 0)[1]
    padded = torch.zeros(2 * cmax, dtype=torch.float64, device=device)
    padded[: losses.numel()] = losses
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    out = torch.cat([parts[s][: 2 * shard(pairs, world, s)[1]] for s in range(world)])
    return g, out


def sharded_smoothed_grad(scene, wl, theta, sigma, target, step: int = 0, group=None, **opts):
    """One job's plateau-reduced gradient with its pairs sharded over the ranks of `group`
    (each rank on its own GPU): returns (grad, losses) as float64 tensors on theta's device."""
    def local(begin, count):
        o = scene.grad_opts(wl, step=step, pairs=count, pair_begin=begin, **opts)
        return scene.smoothed_grad(theta, sigma, target, o)
    return sharded_estimate(local, wl.pairs, scene.D, group=group, device=theta.device)
