"""Multi-process paths on CPU (gloo, world size 2): the replica bench's max-over-ranks
timing, and the sharded estimate of one job's gradient -- each rank computes a block of
antithetic pairs with their global draw indices (the oracle stands in for each rank's
GPU), one all-reduce combines them -- against the single-process estimate."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads
from paper_2211_17263_gb300 import dist as pdist


def test_shard_blocks_cover_the_pairs_in_order():
    for pairs in (1, 2, 7, 8, 33, 256):
        for world in (1, 2, 3, 8):
            blocks = [pdist.shard(pairs, world, r) for r in range(world)]
            assert blocks[0][0] == 0
            for (b0, c0), (b1, _) in zip(blocks, blocks[1:]):
                assert b1 == b0 + c0
            assert sum(c for _, c in blocks) == pairs
            assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tiny(crn):
    wl = workloads.scaled(workloads.config_occlusion(seed=3), width=12, height=10, spp=2, pairs=5)
    wl.crn = crn
    return wl


def _worker(rank, world, port, crn, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _tiny(crn)
        target = oracle.render_target(wl, nthreads=1)

        def local(begin, count):
            r = oracle.smoothed_grad(wl, target=target, step=4, pairs=count, pair_begin=begin, nthreads=1)
            return r["grad"], r["losses"]

        g, losses = pdist.sharded_estimate(local, wl.pairs, wl.D)
        t = pdist.max_over_ranks(float(rank + 1) * 0.5, world)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([g.numpy(), losses.numpy(), [t]]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("crn", [1, 0])
def test_sharded_estimate_equals_single_process(tmp_path, crn):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), crn, str(tmp_path)), nprocs=world, join=True)
    wl = _tiny(crn)
    ref = oracle.smoothed_grad(wl, target=oracle.render_target(wl), step=4)
    for rank in range(world):
        v = np.load(tmp_path / f"r{rank}.npy")
        g, losses, t = v[: wl.D], v[wl.D: wl.D + wl.renders], v[-1]
        assert np.array_equal(losses, ref["losses"])         # the same renders, bit for bit
        np.testing.assert_allclose(g, ref["grad"], rtol=1e-12)  # one all-reduce of (P_s/P) g_s
        assert t == 1.0                                        # the max over ranks
