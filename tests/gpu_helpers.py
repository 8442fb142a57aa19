"""Helpers for the GPU parity tests: move seeded inputs to the device, run the
CUDA path through the C ABI, and compare with the oracle."""
import numpy as np
import torch

import paper_2107_12672_b300 as dvr
from paper_2107_12672_b300 import synthetic as syn

# Tolerances of the FP32 CUDA path against the FP64 oracle, per element:
# |gpu - ref| <= rtol * (|ref| + max|ref|), i.e. relative to the element or,
# for elements far below the array's scale, to the scale.
IMAGE_RTOL = 1e-5
GRAD_RTOL = 1e-3


def rel_err(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    if scale == 0:
        return float(np.abs(gpu).max())
    return float((np.abs(gpu - ref) / (np.abs(ref) + scale)).max())


# The oracle bounds what binary32 rounding may change at kinks (TF control
# points, cell faces); the parity tests take twice its error model.

FP32_MARGIN = 2.0


def assert_close(gpu, ref, rtol, what="", slack=None):
    """|gpu - ref| <= rtol (|ref| + max|ref|) + slack, elementwise; `slack` is
    the oracle's bound on what the choice of one-sided derivatives at TF
    kinks may change."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    excess = np.abs(gpu - ref) - (slack if slack is not None else 0.0)
    err = np.maximum(excess, 0.0) / (np.abs(ref) + scale) if scale > 0 else np.maximum(excess, 0.0)
    e = float(err.max())
    if e > rtol:
        i = np.unravel_index(int(np.argmax(err)), err.shape)
        sl = 0.0 if slack is None else float(np.asarray(slack)[i])
        raise AssertionError(f"{what}: max relative error {e:.3e} > {rtol:.1e} at {i}: gpu {gpu[i]:.7g} "
                             f"ref {ref[i]:.7g} scale {scale:.4g} kink slack {sl:.3g}")
    return e


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def as_oracle_volume(t):
    """The exact values the device holds (after BF16/FP16 rounding), as
    float32 (exact for those types; the oracle reads them without widening)."""
    return t.detach().to(torch.float32).cpu().numpy()


def seeded_grad_image(pixels, channels, seed):
    """dL/d(image) seeds for the adjoint: seeded and shared by both sides."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(pixels, channels)).astype(np.float32)


def pixel_offsets(views):
    off, out = 0, []
    for w in views:
        out.append(off)
        off += w.width * w.height
    return out, off
