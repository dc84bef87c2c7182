"""GPU: an estimate computed in blocks of antithetic pairs (prdpt_grad_opts.pair_begin,
the per-rank work of a sharded job) composes to the single-call estimate: the same
renders bit for bit, and g = sum_s (P_s / P) g_s -- for Eq. 10 with path sharing, with
independent path streams, for Eq. 9, and for a texture's D-dimensional draws."""
import numpy as np
import pytest

import oracle
import workloads
from paper_2211_17263_gb300 import dist as pdist

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    from paper_2211_17263_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _cases():
    occ = workloads.scaled(workloads.config_occlusion(), width=48, height=40, spp=4, pairs=5)
    occ_indep = workloads.scaled(workloads.config_occlusion(), width=40, height=32, spp=2, pairs=4)
    occ_indep.crn = 0
    kdp = workloads.scaled(workloads.config_small_albedo(), width=32, height=24, spp=2, pairs=3)
    tex = workloads.config_texture(res=8, px_per_texel=2)
    tex.pairs = 5
    return {"eq10-shared": occ, "eq10-independent-streams": occ_indep, "eq9": kdp, "texture": tex}


@pytest.mark.parametrize("case", list(_cases()))
def test_pair_blocks_compose_to_the_full_estimate(ctx, case):
    wl = _cases()[case]
    target = _t(oracle.render_target(wl))
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    theta, sigma = _t(wl.theta0), _t(wl.sigma)
    g, L = scene.smoothed_grad(theta, sigma, target, scene.grad_opts(wl, step=3))
    blocks = [pdist.shard(wl.pairs, 2, s) for s in range(2)]
    parts = [scene.smoothed_grad(theta, sigma, target, scene.grad_opts(wl, step=3, pairs=c, pair_begin=b))
             for b, c in blocks]
    torch.cuda.synchronize()
    L_blocks = np.concatenate([p[1].cpu().numpy() for p in parts])
    assert np.array_equal(L_blocks, L.cpu().numpy())
    g_comb = sum((c / wl.pairs) * p[0].cpu().numpy().astype(np.float64) for (b, c), p in zip(blocks, parts))
    g_full = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g_comb - g_full) <= 1e-6 * np.linalg.norm(g_full)
    # the single-process path of the sharding helper is the plain call
    g1, L1 = pdist.sharded_smoothed_grad(scene, wl, theta, sigma, target, step=3)
    assert np.array_equal(L1.cpu().numpy(), L.cpu().numpy().astype(np.float64))
