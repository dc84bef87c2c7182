"""Torch-facing convenience layer over the C ABI (marshalling only).

PyTorch supplies device memory and streams; every computation runs in
libprdpt.so. Tensors passed in must be contiguous CUDA float32 tensors on the
context's device; outputs are allocated here with torch and filled by the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import capi


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_ptr(t: torch.Tensor):
    if not t.is_cuda or t.dtype not in (torch.float32, torch.int32, torch.uint32) or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32/int32 tensor")
    return C.c_void_p(t.data_ptr())


def _host_ptr(a):
    """Address of a contiguous float32 host buffer (numpy array or CPU torch tensor)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("host buffers must be contiguous float32 CPU tensors")
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host buffers must be contiguous float32 arrays")
    return C.c_void_p(a.ctypes.data)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Context:
    """A library context on one CUDA device (owns scenes and resident jobs)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        capi.load()
        self.device = device
        self.handle = capi.prdpt_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle is not None:
            capi.prdpt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- scenes ---------------------------------------------------------------------------
    def upload_scene(self, scene, bindings) -> "Scene":
        return Scene(self, scene, bindings)

    # -- counters ---------------------------------------------------------------------------
    def counters_enable(self, on: bool = True):
        capi.prdpt_counters_enable(self.handle, 1 if on else 0)

    def counters_read(self):
        return capi.prdpt_counters_read(self.handle)

    def kernel_timing(self, on: bool = True):
        capi.prdpt_kernel_timing_enable(self.handle, 1 if on else 0)

    def kernel_timing_read(self):
        return capi.prdpt_kernel_timing_read(self.handle)

    def memory_used(self) -> int:
        return capi.prdpt_memory_used(self.handle)

    def fp32_peak_probe(self, iters: int = 1 << 19) -> tuple[float, float]:
        """Achieved FP32 FMA TFLOP/s of a full-occupancy FMA-chain launch, and its ms."""
        return capi.prdpt_fp32_peak_probe(self.handle, iters)

    def sync(self, stream=None):
        capi.prdpt_sync(self.handle, _stream_ptr(stream))

    def philox_words(self, seed, c0_base, c1, c2, c3, n, stream=None) -> torch.Tensor:
        out = torch.empty((n, 4), dtype=torch.int32, device=f"cuda:{self.device}")
        capi.prdpt_philox_words(self.handle, seed, c0_base, c1, c2, c3, n, _dev_ptr(out), _stream_ptr(stream))
        return out

    def sample_perturbations(self, sigma: torch.Tensor, pairs, sampler=0, antithetic=1, seed=0, step=0,
                             stream=None):
        D = sigma.numel()
        R = 2 * pairs
        tau = torch.empty((R, D), dtype=torch.float32, device=sigma.device)
        w = torch.empty((R, D), dtype=torch.float32, device=sigma.device)
        o = capi.prdpt_grad_opts(pairs=pairs, width=1, height=1, spp=1, depth=1, rr_start=-1, sampler=sampler,
                                 antithetic=antithetic, crn=1, seed=seed, step=step, block_pixels=0)
        capi.prdpt_sample_perturbations(self.handle, D, _dev_ptr(sigma), o, _dev_ptr(tau), _dev_ptr(w),
                                        _stream_ptr(stream))
        return tau, w

    def adam_step(self, theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        capi.prdpt_adam_step(self.handle, theta.numel(), _dev_ptr(theta), _dev_ptr(m), _dev_ptr(v), _dev_ptr(grad),
                             t, lr, beta1, beta2, eps, _stream_ptr(stream))


class Scene:
    """An uploaded scene plus its parameter bindings (theta -> scene fields)."""

    def __init__(self, ctx: Context, scene, bindings):
        self.ctx = ctx
        arrays = [np.ascontiguousarray(scene.prim_type, np.int32), np.ascontiguousarray(scene.prim_mat, np.int32),
                  np.ascontiguousarray(scene.prim_geom, np.float32), np.ascontiguousarray(scene.mat_type, np.int32),
                  np.ascontiguousarray(scene.mat_param, np.float32), np.ascontiguousarray(scene.camera, np.float32),
                  np.ascontiguousarray(scene.background, np.float32)]
        desc = capi.prdpt_scene_desc(int(arrays[0].shape[0]), int(arrays[3].shape[0]), *[_np_ptr(a) for a in arrays])
        b = np.ascontiguousarray(bindings, np.int32).reshape(-1, 3)
        # a texture binding (4, material, T) is one row standing for 3 T^2 parameters
        self.D = 3 * int(b[0, 2]) ** 2 if b.shape[0] == 1 and int(b[0, 0]) == 4 else int(b.shape[0])
        binds = (capi.prdpt_param_binding * b.shape[0])(*[capi.prdpt_param_binding(*map(int, row)) for row in b])
        self.id = capi.prdpt_scene_upload(ctx.handle, desc, binds, self.D)

    def render_batch(self, thetas: torch.Tensor, width, height, spp, depth, rr_start=-1, seed=0, step=0, tag=2,
                     crn=1, block_pixels=0, ctas_per_sm=0, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        thetas = thetas.reshape(-1, self.D)
        n = thetas.shape[0]
        if out is None:
            out = torch.empty((n, height, width, 4), dtype=torch.float32, device=thetas.device)
        o = capi.prdpt_render_opts(width=width, height=height, spp=spp, depth=depth, rr_start=rr_start, seed=seed,
                                   step=step, tag=tag, crn=crn, block_pixels=block_pixels, ctas_per_sm=ctas_per_sm)
        capi.prdpt_render_batch(self.ctx.handle, self.id, _dev_ptr(thetas), n, o, _dev_ptr(out), _stream_ptr(stream))
        return out

    def grad_opts(self, wl, step=0, pairs=None, sampler=None, antithetic=None, crn=None, block_pixels=0,
                  ctas_per_sm=0, no_path_sharing=0, estimator=None, pair_begin=0, render_groups=0):
        return capi.prdpt_grad_opts(
            pairs=wl.pairs if pairs is None else pairs, width=wl.width, height=wl.height, spp=wl.spp,
            depth=wl.depth, rr_start=wl.rr_start, sampler=wl.sampler if sampler is None else sampler,
            antithetic=wl.antithetic if antithetic is None else antithetic, crn=wl.crn if crn is None else crn,
            seed=wl.seed, step=step, block_pixels=block_pixels, ctas_per_sm=ctas_per_sm,
            no_path_sharing=no_path_sharing,
            estimator=getattr(wl, "estimator", 0) if estimator is None else estimator, pair_begin=pair_begin,
            render_groups=render_groups)

    def smoothed_grad_host(self, theta, sigma, target, opts, grad=None, losses=None, stream=None):
        """The gradient with host buffers (prdpt_smoothed_grad_host): theta, sigma [D] and target
        [H, W, 4] float32 in host memory (numpy or CPU tensors; page-locked ones copy fastest);
        returns (grad [D], losses [2P]) in host memory when the call returns."""
        if grad is None:
            grad = np.empty(self.D, np.float32)
        if losses is None:
            losses = np.empty(2 * opts.pairs, np.float32)
        capi.prdpt_smoothed_grad_host(self.ctx.handle, self.id, _host_ptr(theta), _host_ptr(sigma), opts,
                                      _host_ptr(target), _host_ptr(grad), _host_ptr(losses), _stream_ptr(stream))
        return grad, losses

    def step_host(self, theta, m, v, t, lr, sigma, target, opts, grad=None, losses=None, beta1=0.9, beta2=0.999,
                  eps=1e-8, stream=None):
        """One optimisation step with host buffers (prdpt_step_host): the gradient at theta,
        then Adam step t (1-based) updating theta, m, v [D] (float32 host arrays) in place.
        grad [D] and losses [2P], if given, receive the step's gradient and losses."""
        capi.prdpt_step_host(self.ctx.handle, self.id, _host_ptr(theta), _host_ptr(m), _host_ptr(v), int(t), lr,
                             beta1, beta2, eps, _host_ptr(sigma), opts, _host_ptr(target),
                             None if grad is None else _host_ptr(grad), None if losses is None else _host_ptr(losses),
                             _stream_ptr(stream))

    def smoothed_grad(self, theta: torch.Tensor, sigma: torch.Tensor, target: torch.Tensor, opts,
                      grad: torch.Tensor | None = None, losses: torch.Tensor | None = None, stream=None):
        if grad is None:
            grad = torch.empty(self.D, dtype=torch.float32, device=theta.device)
        if losses is None:
            losses = torch.empty(2 * opts.pairs, dtype=torch.float32, device=theta.device)
        capi.prdpt_smoothed_grad(self.ctx.handle, self.id, _dev_ptr(theta), _dev_ptr(sigma), opts, _dev_ptr(target),
                                 _dev_ptr(grad), _dev_ptr(losses), _stream_ptr(stream))
        return grad, losses


class Job:
    """A resident optimisation job: parameters, Adam state and target live on the device.

    target_host: the [H, W, 4] target image, or None to render it on the device later
    (render_target). With block_pixels = ctas_per_sm = 0 the launch shape is the one the
    autotuner cached for this workload's shape, if any (see autotune.py), else the
    library's default."""

    def __init__(self, scene: Scene, wl, target_host: np.ndarray | None, step0=0, block_pixels=0, ctas_per_sm=0,
                 anneal=None, lr=None, sampler=None, no_path_sharing=0, use_tuned=True, render_groups=0):
        self.scene = scene
        self.D = scene.D
        self.R = 2 * wl.pairs
        self._theta0 = np.ascontiguousarray(wl.theta0, np.float32)
        self._sigma0 = np.ascontiguousarray(wl.sigma, np.float32)
        self._target = None
        if target_host is not None:
            self._target = np.ascontiguousarray(target_host, np.float32)
            if self._target.shape != (wl.height, wl.width, 4):
                raise ValueError("target must be [H, W, 4] float32")
        self.launch_shape = {"block_pixels": block_pixels, "ctas_per_sm": ctas_per_sm,
                             "render_groups": render_groups, "no_path_sharing": no_path_sharing, "source": "given"}
        if use_tuned and block_pixels == 0 and ctas_per_sm == 0 and render_groups == 0 and no_path_sharing == 0:
            from . import autotune
            hit = autotune.cached_shape(wl)
            if hit is not None:
                block_pixels, ctas_per_sm = hit["block_pixels"], hit["ctas_per_sm"]
                render_groups = hit.get("render_groups", 0)
                no_path_sharing = hit.get("no_path_sharing", 0)
                self.launch_shape = {"block_pixels": block_pixels, "ctas_per_sm": ctas_per_sm,
                                     "render_groups": render_groups, "no_path_sharing": no_path_sharing,
                                     "source": "autotuner cache"}
            else:
                self.launch_shape["source"] = "library default"
        desc = capi.prdpt_job_desc(
            grad=scene.grad_opts(wl, step=step0, sampler=sampler, block_pixels=block_pixels,
                                 ctas_per_sm=ctas_per_sm, no_path_sharing=no_path_sharing,
                                 render_groups=render_groups),
            theta0_host=_np_ptr(self._theta0), sigma0_host=_np_ptr(self._sigma0),
            target_host=None if self._target is None else _np_ptr(self._target),
            lr=wl.lr if lr is None else lr, beta1=0.9, beta2=0.999, eps=1e-8, sigma_min=wl.sigma_min,
            anneal=wl.anneal if anneal is None else anneal, total_steps=wl.steps)
        self.id = capi.prdpt_job_create(scene.ctx.handle, scene.id, desc)

    def render_target(self, theta_ref: torch.Tensor, stream=None):
        """Render the job's target at theta_ref [D] (device tensor) into its device buffer
        (prdpt_job_render_target), enqueued on `stream`; no host round trip."""
        capi.prdpt_job_render_target(self.scene.ctx.handle, self.id, _dev_ptr(theta_ref.reshape(-1)),
                                     _stream_ptr(stream))

    def step(self, stream=None):
        capi.prdpt_step(self.scene.ctx.handle, self.id, _stream_ptr(stream))

    def read(self):
        theta = np.zeros(self.D, np.float32)
        grad = np.zeros(self.D, np.float32)
        losses = np.zeros(self.R, np.float32)
        steps = capi.prdpt_job_read(self.scene.ctx.handle, self.id, _np_ptr(theta), _np_ptr(grad), _np_ptr(losses))
        return {"theta": theta, "grad": grad, "losses": losses, "steps": steps}

    def release(self):
        if self.id is not None:
            capi.prdpt_job_release(self.scene.ctx.handle, self.id)
            self.id = None


def step_batch(ctx: Context, jobs, stream=None):
    capi.prdpt_step_batch(ctx.handle, [j.id for j in jobs], _stream_ptr(stream))
