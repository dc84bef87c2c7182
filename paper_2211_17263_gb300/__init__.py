"""GB300 (sm_103a) implementation of the plateau-reduced gradient estimator of
Fischer & Ritschel, "Plateau-reduced Differentiable Path Tracing".

The compute path is libprdpt.so (hand-written CUDA, C ABI in include/prdpt.h);
`capi` binds it with ctypes, `api` wraps it for torch tensors and streams,
`autograd` exposes the smoothed loss as a torch.autograd.Function.
"""
from . import capi  # noqa: F401
