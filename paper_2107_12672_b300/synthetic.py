"""Seeded synthetic inputs for the differentiable volume renderer.

This module produces volumes, transfer functions and camera placements and
nothing else: it holds none of the rendering arithmetic (no ray setup, no
interpolation of the rendered field, no transfer-function lookup, no
compositing). The FP64 oracle and the CUDA path both consume its arrays, so it
is the one place the two sides share.

The paper's datasets (CT scans and simulation volumes of Sec. 5) are not
available; these generators stand in for them with the paper's shapes: 256^3
volumes, 512^2 images, 8 or 64 views on an enclosing sphere, step sizes of a
fraction of a voxel (Sec. 5.2, Sec. 5.3).

* Gaussian blobs: a sum of isotropic Gaussians, separable per axis.
* Value noise: random lattice values blended with the smoothstep fade
  s(t) = t^2 (3 - 2t) per axis (a different weight from the renderer's
  trilinear one), summed over octaves and normalised to [0, 1].
* Transfer functions: R rows of (r, g, b, tau), colours U[0,1], absorption
  U[0, tau_max] per world unit.
* Views: points of a Fibonacci sphere (golden-angle spiral) scaled to a
  camera distance, or seeded orbit angles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "gaussian_blobs",
    "value_noise",
    "random_tf",
    "color_volume",
    "fibonacci_sphere",
    "View",
    "Workload",
    "workload",
    "WORKLOADS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def gaussian_blobs(n: int, count: int, seed: int, sigma=(4.0, 10.0),
                   amplitude=(0.5, 2.0), centre=None, scale_to: int = 64,
                   dtype=np.float32, device=None):
    """Sum of `count` isotropic Gaussians on an n^3 grid, layout [z][y][x].

    Centres are drawn U[centre] in voxels (default [n/4, 3n/4]); sigma and
    centre ranges are given for a 64^3 grid and scaled by n/scale_to, so the
    same seed gives the same shapes at every resolution. With a torch
    `device` the sum is formed there in float32 (large volumes).
    """
    rng = _rng(seed)
    s = n / float(scale_to)
    lo, hi = centre if centre is not None else (0.25 * scale_to, 0.75 * scale_to)
    c = rng.uniform(lo, hi, size=(count, 3)) * s
    sg = rng.uniform(sigma[0], sigma[1], size=count) * s
    a = rng.uniform(amplitude[0], amplitude[1], size=count)
    idx = np.arange(n, dtype=np.float64)
    if device is not None:
        import torch
        out = torch.zeros((n, n, n), dtype=torch.float32, device=device)
        for k in range(count):
            g = [torch.from_numpy(np.exp(-((idx - c[k, d]) ** 2) / (2 * sg[k] ** 2))).to(device, torch.float32)
                 for d in range(3)]
            out += float(a[k]) * (g[2][:, None, None] * (g[1][None, :, None] * g[0][None, None, :]))
        return out
    out = np.zeros((n, n, n), dtype=np.float64)
    for k in range(count):
        gx = np.exp(-((idx - c[k, 0]) ** 2) / (2 * sg[k] ** 2))
        gy = np.exp(-((idx - c[k, 1]) ** 2) / (2 * sg[k] ** 2))
        gz = np.exp(-((idx - c[k, 2]) ** 2) / (2 * sg[k] ** 2))
        out += a[k] * (gz[:, None, None] * (gy[None, :, None] * gx[None, None, :]))
    return out.astype(dtype)


def _fade_matrix(n: int, cells: int) -> np.ndarray:
    """[n][cells+1] weights blending lattice values with the smoothstep fade."""
    w = np.zeros((n, cells + 1), dtype=np.float64)
    for i in range(n):
        p = i * cells / max(n - 1, 1)
        c = min(int(math.floor(p)), cells - 1)
        t = p - c
        sm = t * t * (3.0 - 2.0 * t)
        w[i, c] += 1.0 - sm
        w[i, c + 1] += sm
    return w


def value_noise(n: int, seed: int, cells=(4, 8, 16), amps=(1.0, 0.5, 0.25),
                dtype=np.float32, device=None):
    """Multi-octave value noise on an n^3 grid normalised to [0, 1].

    With `device=None` the result is a numpy array computed in float64; with
    a torch device (e.g. "cuda") the same lattice and weights are combined
    with torch on that device in float32 (for volumes too large for the host).
    """
    rng = _rng(seed)
    lattices = [rng.uniform(0.0, 1.0, size=(c + 1, c + 1, c + 1)) for c in cells]
    if device is None:
        out = np.zeros((n, n, n), dtype=np.float64)
        for lat, c, a in zip(lattices, cells, amps):
            w = _fade_matrix(n, c)
            t = np.tensordot(w, lat, axes=([1], [0]))          # z c c
            t = np.tensordot(t, w, axes=([2], [1]))            # z c x
            t = np.einsum("zcx,yc->zyx", t, w)
            out += a * t
        lo, hi = out.min(), out.max()
        out = (out - lo) / (hi - lo)
        return out.astype(dtype)
    import torch
    out = torch.zeros((n, n, n), dtype=torch.float32, device=device)
    for lat, c, a in zip(lattices, cells, amps):
        w = torch.from_numpy(_fade_matrix(n, c)).to(device=device, dtype=torch.float32)
        lt = torch.from_numpy(lat).to(device=device, dtype=torch.float32)
        t = torch.tensordot(w, lt, dims=([1], [0]))
        t = torch.tensordot(t, w, dims=([2], [1]))
        out += a * torch.einsum("zcx,yc->zyx", t, w)
        del t
    lo, hi = out.min(), out.max()
    out.sub_(lo).div_(hi - lo)
    return out


def color_volume(n: int, seed: int, tau_max: float = 20.0, dtype=np.float32) -> np.ndarray:
    """[n][n][n][4] pre-shaded colour volume: value noise per channel
    (seeds seed..seed+3), colours in [0, 1], absorption in [0, tau_max]."""
    chans = [value_noise(n, seed=seed + k, dtype=np.float64) for k in range(4)]
    chans[3] = chans[3] * tau_max
    return np.stack(chans, axis=-1).astype(dtype)


def random_tf(R: int, seed: int, tau_max: float = 50.0, dtype=np.float32) -> np.ndarray:
    """[R][4] rows (r, g, b, tau): colours U[0,1], absorption U[0, tau_max]."""
    rng = _rng(seed)
    tf = np.empty((R, 4), dtype=np.float64)
    tf[:, :3] = rng.uniform(0.0, 1.0, size=(R, 3))
    tf[:, 3] = rng.uniform(0.0, tau_max, size=R)
    return tf.astype(dtype)


def fibonacci_sphere(k: int) -> np.ndarray:
    """k unit vectors on a golden-angle spiral (y from +1 towards -1)."""
    j = np.arange(k, dtype=np.float64)
    y = 1.0 - 2.0 * (j + 0.5) / k
    r = np.sqrt(np.maximum(0.0, 1.0 - y * y))
    phi = j * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), y, r * np.sin(phi)], axis=1)


@dataclass
class View:
    """Static description of one rendered view (the differentiable camera
    position lives in a separate [n_views][3] array)."""
    width: int
    height: int
    ortho: bool = False
    tan_half_fov_y: float = math.tan(math.radians(45.0) / 2)
    ortho_height: float = 1.0
    volume_index: int = 0


@dataclass
class Workload:
    name: str
    model: str                      # "absorption", "emission_absorption" or "color"
    volumes: list                   # numpy arrays [nz][ny][nx] ([nz][ny][nx][4] for "color")
    tf: np.ndarray | None           # [R][4] or None (absorption)
    views: list                     # list[View]
    eye: np.ndarray                 # [n_views][3] float32 camera positions
    orbit: np.ndarray | None        # [n_views][3] (yaw, pitch, distance) or None
    step_voxels: float
    grads: tuple                    # subset of ("volume", "tf", "camera")
    target: dict = field(default_factory=dict)  # what the loss compares to
    note: str = ""
    loss: str = "l2"                # "l2" against the target, or "entropy" (opacity entropy, maximised)
    volume_dtype: str = "float32"   # storage of the volume on the device (torch dtype name)
    tf_dtype: str = "float32"       # storage of the TF on the device


def _orbit_params(rng, count, distance):
    yaw = rng.uniform(-math.pi, math.pi, size=count)
    pitch = rng.uniform(-0.6, 0.6, size=count)
    return np.stack([yaw, pitch, np.full(count, distance)], axis=1)


def workload(name: str, scale: float = 1.0) -> Workload:
    """Build one of the named workloads.

    `scale` < 1 shrinks volume and image sizes (for CPU-checkable parity
    cases); the structure (model, seeds, camera, step) stays the same.
    """
    def sz(v, lo=8):
        return max(lo, int(round(v * scale)))

    if name == "absorption_64":
        n = sz(64)
        vol = gaussian_blobs(n, 8, seed=1)
        tgt = gaussian_blobs(n, 8, seed=2)
        w = sz(64)
        views = [View(w, w, ortho=True, ortho_height=1.0)]
        eye = np.array([[0.0, 0.0, 2.0]], dtype=np.float32)
        return Workload(name, "absorption", [vol], None, views, eye, None, 0.5,
                        ("volume",), target={"volume": tgt},
                        note="64^3 FP32 Gaussian blobs, ortho +z, 64x64, step 0.5 voxel")
    if name == "ea_256":
        n = sz(256)
        vol = value_noise(n, seed=3)
        tf = random_tf(16, seed=3)
        tf_target = random_tf(16, seed=103)
        w = sz(512)
        rng = _rng(3)
        orbit = _orbit_params(rng, 1, 2.5)
        views = [View(w, w, ortho=False)]
        eye = (fibonacci_sphere(7)[2:3] * 2.5).astype(np.float32)
        return Workload(name, "emission_absorption", [vol], tf, views, eye, orbit, 0.5,
                        ("tf", "camera"), target={"tf": tf_target},
                        note="256^3 FP32 value noise, R=16 TF (tau in [0,50]), perspective "
                             "distance 2.5, FOV 45 deg, 512x512, step 0.5 voxel")
    if name == "tomo_256x64":
        n = sz(256)
        vol = gaussian_blobs(n, 32, seed=4)
        rng = _rng(4)
        sizes = rng.choice([128, 256, 512, 1024], size=64)
        views = [View(sz(int(s), 4), sz(int(s), 4)) for s in sizes]
        eye = (fibonacci_sphere(64) * 2.5).astype(np.float32)
        return Workload(name, "absorption", [vol], None, views, eye, None, 0.5,
                        ("volume",), target={"volume": gaussian_blobs(n, 32, seed=104)},
                        note="256^3 FP32 Gaussian blobs, absorption, 64 Fibonacci views of "
                             "sizes {128..1024}^2, step 0.5 voxel")
    if name == "ea_bf16_512":
        n = sz(512)
        vol = value_noise(n, seed=5)
        tf = random_tf(64, seed=5, tau_max=50.0)
        w = sz(1024)
        views = [View(w, w) for _ in range(16)]
        eye = (fibonacci_sphere(16) * 2.5).astype(np.float32)
        return Workload(name, "emission_absorption", [vol], tf, views, eye, None, 0.25,
                        ("volume", "tf", "camera"), target={"tf": random_tf(64, seed=105)},
                        note="512^3 BF16 value noise, 64-point FP16 TF, 16 views 1024^2, "
                             "step 0.25 voxel",
                        volume_dtype="bfloat16", tf_dtype="float16")
    if name == "ea_fp16_1024":
        # volumes are left to the caller (device generation, see large_volume)
        n = sz(1024)
        tf = random_tf(32, seed=6, tau_max=50.0)
        w = sz(2048)
        views = [View(w, w) for _ in range(32)]
        eye = (fibonacci_sphere(32) * 2.5).astype(np.float32)
        return Workload(name, "emission_absorption", [], tf, views, eye, None, 0.25,
                        ("volume", "tf", "camera"), target={"n": n},
                        note="1024^3 FP16 value noise plus 32 Gaussian blobs, 32-point TF, "
                             "32 views 2048^2, step 0.25 voxel (~4000 steps on axis-aligned rays), "
                             "opacity-entropy loss",
                        loss="entropy", volume_dtype="float16")
    if name == "color_256":
        n = sz(256)
        vol = color_volume(n, seed=7)
        w = sz(512)
        views = [View(w, w) for _ in range(8)]
        eye = (fibonacci_sphere(8) * 2.5).astype(np.float32)
        return Workload(name, "color", [vol], None, views, eye, None, 0.5,
                        ("volume", "camera"), target={"volume": color_volume(n, seed=107)},
                        note="256^3 FP32 pre-shaded colour volume (r, g, b, tau per vertex, value noise, "
                             "tau in [0, 20]), 8 Fibonacci views 512^2, step 0.5 voxel, L2 loss against "
                             "a second colour volume's images")
    raise KeyError(name)


def large_volume(n: int, seed: int = 6, device="cuda"):
    """n^3 value noise plus 32 Gaussian blobs (scaled to [0, 1]) formed on a
    torch device in float32 (the 1024^3 workload)."""
    v = value_noise(n, seed=seed, device=device)
    b = gaussian_blobs(n, 32, seed=seed + 100, device=device)
    b.mul_(1.0 / float(b.max()))
    v.mul_(0.5).add_(b, alpha=0.5)
    return v


WORKLOADS = ("absorption_64", "ea_256", "tomo_256x64", "ea_bf16_512", "ea_fp16_1024", "color_256")
