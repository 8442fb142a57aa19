"""Helpers for the GPU parity tests: move seeded inputs to the device, run the
CUDA path through the C ABI, and compare with the oracle."""
import os

import numpy as np
import torch

import paper_2107_12672_b300 as dvr
from paper_2107_12672_b300 import synthetic as syn

# Tolerances of the FP32 CUDA path against the FP64 oracle, per element
# (1e-5 relative for binary32 images, 1e-3 relative for gradients), with a
# floor for elements far below the array's scale, where only an absolute
# error means anything (sums whose terms cancel, atomics in any order):
#   |gpu - ref| <= rtol * max(|ref|, FLOOR * max|ref|) + slack
IMAGE_RTOL = 1e-5
GRAD_RTOL = 1e-3
FLOOR = 1e-3


def rel_err(gpu, ref):
    """Max-norm relative error, max |gpu - ref| / (|ref| + max|ref|) (a
    summary figure; the parity bar is assert_close's per-element rule)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    if scale == 0:
        return float(np.abs(gpu).max())
    return float((np.abs(gpu - ref) / (np.abs(ref) + scale)).max())


def elem_err(gpu, ref, slack=None):
    """Per-element relative error max_i (|gpu - ref| - slack)+ / max(|ref|,
    FLOOR max|ref|), and its index."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    excess = np.abs(gpu - ref)
    if slack is not None:
        excess = np.maximum(excess - slack, 0.0)
    if scale == 0:
        err = excess
    else:
        err = excess / np.maximum(np.abs(ref), FLOOR * scale)
    i = np.unravel_index(int(np.argmax(err)), err.shape) if err.size else ()
    return (float(err[i]) if err.size else 0.0), i


# The oracle bounds what binary32 rounding may change at kinks (TF control
# points, cell faces); the parity tests take twice its error model.

FP32_MARGIN = 2.0

# every comparison made by assert_close in this process: (what, per-element
# error with slack, per-element error without slack, max-norm error)
RECORD = []


def assert_close(gpu, ref, rtol, what="", slack=None):
    """Per element: |gpu - ref| <= rtol max(|ref|, FLOOR max|ref|) + slack,
    `slack` being the oracle's bound on what the choice of one-sided
    derivatives at kinks (TF control points, cell faces) may change.
    Returns the per-element error (slack subtracted)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    e, i = elem_err(gpu, ref, slack)
    raw, _ = elem_err(gpu, ref)
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    RECORD.append((f"{test}: {what}", e, raw, rel_err(gpu, ref)))
    if e > rtol:
        scale = np.abs(ref).max()
        sl = 0.0 if slack is None else float(np.asarray(slack)[i])
        raise AssertionError(f"{what}: per-element relative error {e:.3e} > {rtol:.1e} at {i}: gpu {gpu[i]:.7g} "
                             f"ref {ref[i]:.7g} scale {scale:.4g} kink slack {sl:.3g} "
                             f"(without slack {raw:.3e}; max-norm {rel_err(gpu, ref):.3e})")
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
