"""ctypes binding of the C ABI in include/prdpt.h (argument marshalling only).

Every function below has the name and argument order of its C counterpart and
does nothing but convert Python values into C values; all computation happens in
libprdpt.so. `load()` builds the library when needed and raises if it cannot be
loaded -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

PRDPT_OK = 0
PRDPT_E_INVALID_ARG = 1
PRDPT_E_OUT_OF_BUDGET = 2
PRDPT_E_CUDA = 3
PRDPT_E_TIMEOUT = 4
PRDPT_E_NOT_READY = 5
PRDPT_E_NOT_FOUND = 6
PRDPT_E_DEVICE = 7

PRDPT_MAX_PRIMS = 32
PRDPT_MAX_MATS = 32
PRDPT_MAX_LIGHTS = 8
PRDPT_MAX_D = 64
PRDPT_MAX_PAIRS = 256

EXPORTS = [
    "prdpt_create", "prdpt_destroy", "prdpt_last_error", "prdpt_scene_upload", "prdpt_scene_release",
    "prdpt_render_batch", "prdpt_sample_perturbations", "prdpt_smoothed_grad", "prdpt_adam_step",
    "prdpt_job_create", "prdpt_step", "prdpt_step_batch", "prdpt_job_read", "prdpt_job_release",
    "prdpt_philox_words", "prdpt_counters_enable", "prdpt_counters_read", "prdpt_kernel_timing_enable",
    "prdpt_kernel_timing_read", "prdpt_sync", "prdpt_smoothed_grad_static", "prdpt_memory_used",
    "prdpt_fp32_peak_probe", "prdpt_smoothed_grad_host", "prdpt_step_host", "prdpt_job_render_target",
]


class prdpt_scene_desc(C.Structure):
    _fields_ = [
        ("n_prims", C.c_int32), ("n_mats", C.c_int32),
        ("prim_type", C.c_void_p), ("prim_mat", C.c_void_p), ("prim_geom", C.c_void_p),
        ("mat_type", C.c_void_p), ("mat_param", C.c_void_p), ("camera", C.c_void_p), ("background", C.c_void_p),
    ]


class prdpt_param_binding(C.Structure):
    _fields_ = [("kind", C.c_int32), ("index", C.c_int32), ("component", C.c_int32)]


class prdpt_render_opts(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32), ("depth", C.c_int32),
        ("rr_start", C.c_int32), ("seed", C.c_uint64), ("step", C.c_uint32), ("tag", C.c_uint32),
        ("crn", C.c_int32), ("block_pixels", C.c_int32), ("ctas_per_sm", C.c_int32),
    ]


class prdpt_grad_opts(C.Structure):
    _fields_ = [
        ("pairs", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
        ("depth", C.c_int32), ("rr_start", C.c_int32), ("sampler", C.c_int32), ("antithetic", C.c_int32),
        ("crn", C.c_int32), ("seed", C.c_uint64), ("step", C.c_uint32), ("block_pixels", C.c_int32),
        ("ctas_per_sm", C.c_int32), ("no_path_sharing", C.c_int32), ("estimator", C.c_int32),
        ("pair_begin", C.c_int32), ("render_groups", C.c_int32),
    ]


class prdpt_job_desc(C.Structure):
    _fields_ = [
        ("grad", prdpt_grad_opts), ("theta0_host", C.c_void_p), ("sigma0_host", C.c_void_p),
        ("target_host", C.c_void_p), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
        ("eps", C.c_float), ("sigma_min", C.c_float), ("anneal", C.c_int32), ("total_steps", C.c_int32),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libprdpt.so (building it first when stale). Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libprdpt.so not found at {path}; run paper_2211_17263_gb300/build.py")
    L = C.CDLL(path)
    vp, i32, u32, u64, f32 = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_float
    P = C.POINTER
    proto = {
        "prdpt_create": ([P(vp), i32, u64], i32),
        "prdpt_destroy": ([vp], i32),
        "prdpt_last_error": ([vp], C.c_char_p),
        "prdpt_scene_upload": ([vp, P(prdpt_scene_desc), P(prdpt_param_binding), i32, P(i32)], i32),
        "prdpt_scene_release": ([vp, i32], i32),
        "prdpt_render_batch": ([vp, i32, vp, i32, P(prdpt_render_opts), vp, vp], i32),
        "prdpt_sample_perturbations": ([vp, i32, vp, P(prdpt_grad_opts), vp, vp, vp], i32),
        "prdpt_smoothed_grad": ([vp, i32, vp, vp, P(prdpt_grad_opts), vp, vp, vp, vp], i32),
        "prdpt_smoothed_grad_host": ([vp, i32, vp, vp, P(prdpt_grad_opts), vp, vp, vp, vp], i32),
        "prdpt_step_host": ([vp, i32, vp, vp, vp, i32, f32, f32, f32, f32, vp, P(prdpt_grad_opts), vp, vp, vp, vp],
                            i32),
        "prdpt_adam_step": ([vp, i32, vp, vp, vp, vp, i32, f32, f32, f32, f32, vp], i32),
        "prdpt_job_create": ([vp, i32, P(prdpt_job_desc), P(i32)], i32),
        "prdpt_step": ([vp, i32, vp], i32),
        "prdpt_step_batch": ([vp, P(i32), i32, vp], i32),
        "prdpt_job_read": ([vp, i32, vp, vp, vp, P(i32)], i32),
        "prdpt_job_release": ([vp, i32], i32),
        "prdpt_job_render_target": ([vp, i32, vp, vp], i32),
        "prdpt_philox_words": ([vp, u64, u32, u32, u32, u32, i32, vp, vp], i32),
        "prdpt_counters_enable": ([vp, i32], i32),
        "prdpt_counters_read": ([vp, P(u64)], i32),
        "prdpt_kernel_timing_enable": ([vp, i32], i32),
        "prdpt_kernel_timing_read": ([vp, P(C.c_double), P(C.c_int64)], i32),
        "prdpt_sync": ([vp, vp], i32),
        "prdpt_memory_used": ([vp, P(u64)], i32),
        "prdpt_fp32_peak_probe": ([vp, i32, P(C.c_double), P(C.c_double)], i32),
        "prdpt_smoothed_grad_static": ([P(prdpt_scene_desc), P(prdpt_param_binding), i32, vp, vp,
                                        P(prdpt_grad_opts), vp, vp, vp, vp, C.c_char_p, C.c_size_t], i32),
    }
    for name, (args, res) in proto.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


class PrdptError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def check(code: int, where: str, ctx=None):
    if code != PRDPT_OK:
        msg = load().prdpt_last_error(ctx).decode(errors="replace")
        raise PrdptError(code, where, msg)
    return code


# -- same-name wrappers (marshalling only) ------------------------------------------------
def prdpt_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = C.c_void_p()
    check(load().prdpt_create(C.byref(h), device, hbm_budget_bytes), "prdpt_create")
    return h


def prdpt_destroy(ctx):
    return check(load().prdpt_destroy(ctx), "prdpt_destroy", ctx)


def prdpt_last_error(ctx) -> str:
    return load().prdpt_last_error(ctx).decode(errors="replace")


def prdpt_scene_upload(ctx, desc: prdpt_scene_desc, binds, D: int) -> int:
    sid = C.c_int32()
    check(load().prdpt_scene_upload(ctx, C.byref(desc), binds, D, C.byref(sid)), "prdpt_scene_upload", ctx)
    return sid.value


def prdpt_scene_release(ctx, scene_id: int):
    return check(load().prdpt_scene_release(ctx, scene_id), "prdpt_scene_release", ctx)


def prdpt_render_batch(ctx, scene_id, thetas_dev, n, opts, images_dev, stream):
    return check(load().prdpt_render_batch(ctx, scene_id, thetas_dev, n, C.byref(opts), images_dev, stream),
                 "prdpt_render_batch", ctx)


def prdpt_sample_perturbations(ctx, D, sigma_dev, opts, tau_dev, w_dev, stream):
    return check(load().prdpt_sample_perturbations(ctx, D, sigma_dev, C.byref(opts), tau_dev, w_dev, stream),
                 "prdpt_sample_perturbations", ctx)


def prdpt_smoothed_grad(ctx, scene_id, theta_dev, sigma_dev, opts, target_dev, grad_dev, losses_dev, stream):
    return check(load().prdpt_smoothed_grad(ctx, scene_id, theta_dev, sigma_dev, C.byref(opts), target_dev, grad_dev,
                                            losses_dev, stream), "prdpt_smoothed_grad", ctx)


def prdpt_smoothed_grad_host(ctx, scene_id, theta_host, sigma_host, opts, target_host, grad_host, losses_host,
                             stream):
    return check(load().prdpt_smoothed_grad_host(ctx, scene_id, theta_host, sigma_host, C.byref(opts), target_host,
                                                 grad_host, losses_host, stream), "prdpt_smoothed_grad_host", ctx)


def prdpt_step_host(ctx, scene_id, theta_host, m_host, v_host, t, lr, beta1, beta2, eps, sigma_host, opts,
                    target_host, grad_host, losses_host, stream):
    return check(load().prdpt_step_host(ctx, scene_id, theta_host, m_host, v_host, t, lr, beta1, beta2, eps,
                                        sigma_host, C.byref(opts), target_host, grad_host, losses_host, stream),
                 "prdpt_step_host", ctx)


def prdpt_adam_step(ctx, D, theta_dev, m_dev, v_dev, grad_dev, t, lr, beta1, beta2, eps, stream):
    return check(load().prdpt_adam_step(ctx, D, theta_dev, m_dev, v_dev, grad_dev, t, lr, beta1, beta2, eps, stream),
                 "prdpt_adam_step", ctx)


def prdpt_job_create(ctx, scene_id, desc: prdpt_job_desc) -> int:
    jid = C.c_int32()
    check(load().prdpt_job_create(ctx, scene_id, C.byref(desc), C.byref(jid)), "prdpt_job_create", ctx)
    return jid.value


def prdpt_step(ctx, job_id, stream):
    return check(load().prdpt_step(ctx, job_id, stream), "prdpt_step", ctx)


def prdpt_step_batch(ctx, job_ids, stream):
    arr = (C.c_int32 * len(job_ids))(*job_ids)
    return check(load().prdpt_step_batch(ctx, arr, len(job_ids), stream), "prdpt_step_batch", ctx)


def prdpt_job_read(ctx, job_id, theta_host, grad_host, losses_host):
    steps = C.c_int32()
    check(load().prdpt_job_read(ctx, job_id, theta_host, grad_host, losses_host, C.byref(steps)), "prdpt_job_read",
          ctx)
    return steps.value


def prdpt_job_release(ctx, job_id):
    return check(load().prdpt_job_release(ctx, job_id), "prdpt_job_release", ctx)


def prdpt_job_render_target(ctx, job_id, theta_ref_dev, stream):
    return check(load().prdpt_job_render_target(ctx, job_id, theta_ref_dev, stream), "prdpt_job_render_target", ctx)


def prdpt_philox_words(ctx, seed, c0_base, c1, c2, c3, n, words_dev, stream):
    return check(load().prdpt_philox_words(ctx, seed, c0_base, c1, c2, c3, n, words_dev, stream),
                 "prdpt_philox_words", ctx)


def prdpt_counters_enable(ctx, enable: int):
    return check(load().prdpt_counters_enable(ctx, enable), "prdpt_counters_enable", ctx)


def prdpt_counters_read(ctx):
    buf = (C.c_uint64 * 8)()
    check(load().prdpt_counters_read(ctx, buf), "prdpt_counters_read", ctx)
    return [int(x) for x in buf]


def prdpt_kernel_timing_enable(ctx, enable: int):
    return check(load().prdpt_kernel_timing_enable(ctx, enable), "prdpt_kernel_timing_enable", ctx)


def prdpt_kernel_timing_read(ctx):
    ms = C.c_double()
    n = C.c_int64()
    check(load().prdpt_kernel_timing_read(ctx, C.byref(ms), C.byref(n)), "prdpt_kernel_timing_read", ctx)
    return ms.value, n.value


def prdpt_smoothed_grad_static(desc, binds, D, theta_dev, sigma_dev, opts, target_dev, grad_dev, losses_dev, stream):
    """Context-free, allocation-free gradient call; raises PrdptError with the call's message."""
    err = C.create_string_buffer(256)
    code = load().prdpt_smoothed_grad_static(C.byref(desc), binds, D, theta_dev, sigma_dev, C.byref(opts),
                                             target_dev, grad_dev, losses_dev, stream, err, C.sizeof(err))
    if code != PRDPT_OK:
        raise PrdptError(code, "prdpt_smoothed_grad_static", err.value.decode(errors="replace"))
    return code


def prdpt_fp32_peak_probe(ctx, iters: int = 1 << 19) -> tuple[float, float]:
    """(achieved FP32 TFLOP/s, launch ms) of the FMA-chain probe."""
    tf, ms = C.c_double(), C.c_double()
    check(load().prdpt_fp32_peak_probe(ctx, int(iters), C.byref(tf), C.byref(ms)), "prdpt_fp32_peak_probe", ctx)
    return tf.value, ms.value


def prdpt_memory_used(ctx) -> int:
    n = C.c_uint64()
    check(load().prdpt_memory_used(ctx, C.byref(n)), "prdpt_memory_used", ctx)
    return n.value


def prdpt_sync(ctx, stream):
    return check(load().prdpt_sync(ctx, stream), "prdpt_sync", ctx)
