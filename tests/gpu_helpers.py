"""Shared helpers of the GPU parity tests (tolerances stated once)."""
import numpy as np

# Image parity (per-pixel, per-channel): mean |I_gpu - I_oracle| <= 1e-4 and at
# most 0.1 % of pixels with any channel off by more than 1e-3 (paths whose FP32 and
# FP64 branch decisions differ at a silhouette, shadow edge or Russian-roulette
# threshold).
IMG_MAE = 1e-4
IMG_OUTLIER_ABS = 1e-3
IMG_OUTLIER_FRAC = 1e-3
# Gradient parity: |g_gpu - g_orc|_2 / max(|g_orc|_2, 1e-6 * c_w * mean_r L_r) <= 1e-3.
GRAD_REL = 1e-3


def image_parity(gpu: np.ndarray, ref: np.ndarray, scale: float = 1.0):
    """gpu, ref: [..., H, W, 3]. `scale` normalises scenes whose radiance is far above 1."""
    diff = np.abs(gpu.astype(np.float64) - ref) / scale
    mae = float(diff.mean())
    outliers = float((diff.max(axis=-1) > IMG_OUTLIER_ABS).mean())
    return mae, outliers


def assert_image_parity(gpu, ref, scale=1.0, what=""):
    mae, out = image_parity(gpu, ref, scale)
    assert mae <= IMG_MAE and out <= IMG_OUTLIER_FRAC, f"{what}: MAE {mae:.3e}, outlier fraction {out:.3e}"
    return mae, out


def grad_rel_error(g_gpu, g_orc, weights, losses):
    c_w = float(np.abs(weights).max())
    floor = 1e-6 * c_w * float(np.mean(losses))
    return float(np.linalg.norm(np.asarray(g_gpu, np.float64) - g_orc) / max(np.linalg.norm(g_orc), floor))
