"""Autotuner for the render kernel's launch shape.

Candidates are (pixels per warp work item, resident CTAs per SM, render groups, path
sharing): the block of pixels a warp traces as one work item, how many 256-thread CTAs the
persistent grid keeps per SM (the number of live warps), whether renders are traced side
by side in one warp (render_groups = 0: automatic group size; -1: one render per work
item), and whether paths are shared across renders where the job allows it
(no_path_sharing = 0: paths no perturbation can reach traced once for geometry-only
perturbations; each path traced once with each render's own next-event estimates when only
emitters move) or every render traces its own. Each
candidate is timed with CUDA events on the render launches of a throwaway resident job of
the same shape; the fastest is cached in a JSON file keyed by the shape, so later jobs of
that shape start from the tuned launch (api.Job looks it up when given no shape). The CTA
count, the render grouping and path sharing never change results; the block shape
regroups the FP64 sums of per-block partials (results agree to rounding).
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "prdpt_gb300", "autotune.json")


def default_cache() -> str:
    """The cache file: $PRDPT_AUTOTUNE_CACHE if set, else DEFAULT_CACHE."""
    return os.environ.get("PRDPT_AUTOTUNE_CACHE") or DEFAULT_CACHE
# (block pixels, CTAs per SM, render groups, no path sharing); with sharing allowed, render
# groups apply only to jobs that cannot share paths (for the others the two sharing
# candidates of a block shape run the same launch)
CANDIDATES = [(px, cps, rg, nps) for px in (32, 16, 8) for cps in (3, 2) for rg, nps in ((0, 0), (-1, 0), (0, 1))]
_lock = threading.Lock()


def shape_key(wl) -> str:
    sc = wl.scene
    counts = [int((sc.prim_type == t).sum()) for t in range(3)]
    mats = sorted(set(int(m) for m in sc.mat_type))
    return (f"W{wl.width}xH{wl.height}_spp{wl.spp}_d{wl.depth}_rr{wl.rr_start}_R{wl.renders}_D{wl.D}"
            f"_prims{counts[0]}-{counts[1]}-{counts[2]}_mats{'-'.join(map(str, mats))}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, table):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cached_shape(wl, cache_path: str | None = ""):
    """The cached best launch shape for this workload's shape, or None (never tunes).
    cache_path "" means default_cache(); None disables the lookup."""
    if cache_path == "":
        cache_path = default_cache()
    if not cache_path:
        return None
    with _lock:
        hit = _load(cache_path).get(shape_key(wl))
    return hit


def time_candidate(scene: api.Scene, wl, target_host: np.ndarray, block_pixels: int, ctas_per_sm: int,
                   steps: int = 3, render_groups: int = 0, no_path_sharing: int = 0) -> float:
    """Mean render-kernel time (ms) of `steps` resident steps with this launch shape."""
    ctx = scene.ctx
    job = api.Job(scene, wl, target_host, block_pixels=block_pixels, ctas_per_sm=ctas_per_sm,
                  render_groups=render_groups, no_path_sharing=no_path_sharing, use_tuned=False)
    try:
        job.step()  # warm-up
        ctx.sync()
        ctx.kernel_timing(True)
        for _ in range(steps):
            job.step()
        ms, n = ctx.kernel_timing_read()
        ctx.kernel_timing(False)
        return ms / max(n, 1)
    finally:
        job.release()


def autotune(scene: api.Scene, wl, target_host: np.ndarray, cache_path: str | None = "",
             candidates=None, steps: int = 3, force: bool = False) -> dict:
    """Best (block_pixels, ctas_per_sm) for this workload shape; cached by shape_key
    (cache_path "" means default_cache(); None: no cache)."""
    if cache_path == "":
        cache_path = default_cache()
    key = shape_key(wl)
    if cache_path and not force:
        with _lock:
            hit = _load(cache_path).get(key)
        if hit:
            return dict(hit, cached=True)
    results = []
    for px, cps, rg, nps in (candidates or CANDIDATES):
        ms = time_candidate(scene, wl, target_host, px, cps, steps, rg, nps)
        results.append({"block_pixels": px, "ctas_per_sm": cps, "render_groups": rg, "no_path_sharing": nps,
                        "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    entry = {"block_pixels": best["block_pixels"], "ctas_per_sm": best["ctas_per_sm"],
             "render_groups": best["render_groups"], "no_path_sharing": best["no_path_sharing"], "ms": best["ms"],
             "tried": results}
    if cache_path:
        with _lock:
            table = _load(cache_path)
            table[key] = entry
            _store(cache_path, table)
    return dict(entry, cached=False)
