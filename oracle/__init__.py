"""FP64 CPU oracle for differentiable direct volume rendering.

TEST INFRASTRUCTURE ONLY: the test suite, the package's smoke check and the
benchmark's CPU-baseline leg load this; the CUDA library never does. It shares
no code with the CUDA path. The arithmetic lives in `dvr_oracle.c` (plain C,
binary64, OpenMP over rays); this module builds it with gcc on first use and
marshals numpy arrays.

Parity pins (what fixes the oracle independently of itself) are in
tests/test_oracle.py; each function below names the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ABSORPTION = 0
EMISSION_ABSORPTION = 1
COLOR_VOLUME = 2
MODELS = {"absorption": ABSORPTION, "emission_absorption": EMISSION_ABSORPTION, "color": COLOR_VOLUME}

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-std=c11"]


def build(force: bool = False) -> str:
    """Compile dvr_oracle.c into liboracle.so (binary64, no FP contraction)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        L = ctypes.c_int64
        D = ctypes.c_double
        lib.ora_render.argtypes = [P, I, I, I, I, P, I, I, I, I, I, D, P, D, I, P, L, P, P, P]
        lib.ora_rays.argtypes = [I, I, I, I, I, I, D, P, D, I, P, P, P]
        lib.ora_interpolate.argtypes = [P, I, I, I, P, L, P]
        lib.ora_backward.argtypes = [P, I, I, I, I, P, I, I, I, I, I, D, P, D, I, P, L, P, I, P, P, P, P, D, P, P]
        lib.ora_backward_sel.argtypes = lib.ora_backward.argtypes + [P, L]
        lib.ora_backward_sel.restype = L
        lib.ora_touched.argtypes = [I, I, I, I, I, I, D, P, D, I, P, L, P, L]
        lib.ora_touched.restype = L
        lib.ora_render_dual.argtypes = [P, I, I, I, I, P, I, I, I, I, I, D, P, D, I, P, L, P, P]
        lib.ora_orbit_eye.argtypes = [P, L, P]
        lib.ora_orbit_eye_backward.argtypes = [P, L, P, P]
        lib.ora_threads.restype = I
        _lib = lib
    return _lib


def threads() -> int:
    return _load().ora_threads()


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _f32val(x):
    """A binary32 value carried in a binary64 (inputs arrive as float32)."""
    return float(np.float32(x))


class _Common:
    def __init__(self, volume, tf, model, view, eye, step, fp32):
        vol = np.asarray(volume)
        # float32 volumes are read as they are (their values are exact in
        # binary64); anything else is widened to binary64
        if vol.dtype != np.float32 and vol.dtype != np.float64:
            vol = vol.astype(np.float64)
        self.vol = np.ascontiguousarray(vol)
        self.vf32 = int(self.vol.dtype == np.float32)
        self.model = MODELS[model] if isinstance(model, str) else int(model)
        # colour volumes are [nz][ny][nx][4] (r, g, b, tau per vertex)
        self.nz, self.ny, self.nx = self.vol.shape[:3]
        if self.model == EMISSION_ABSORPTION:
            self.tf = _f64(tf)
            self.R = self.tf.shape[0]
        else:
            self.tf = np.zeros((2, 4))
            self.R = 2
        self.W, self.H = int(view.width), int(view.height)
        self.ortho = int(bool(view.ortho))
        self.fp32 = int(bool(fp32))
        # camera and step are binary32 inputs of the kernel; the binary64
        # setup (finite differences, duals) takes them unrounded
        cv = _f32val if self.fp32 else float
        self.lens = cv(view.ortho_height if view.ortho else view.tan_half_fov_y)
        self.eye = np.array([cv(e) for e in np.asarray(eye).reshape(3)], dtype=np.float64)
        self.step = cv(step)
        self.nc = 1 if self.model == ABSORPTION else 4

    def head(self):
        return (_p(self.vol), self.vf32, self.nx, self.ny, self.nz, _p(self.tf), self.R, self.model,
                self.W, self.H, self.ortho, self.lens, _p(self.eye), self.step)


def _pix(pix):
    if pix is None:
        return None, 0
    p = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    return p, p.size


def render(volume, tf, model, view, eye, step, fp32=True, pix=None):
    """Alg. 1 for one view. Returns (image [npix][C], N [npix], S [npix]).

    image is RGBA (emission-absorption) or A (absorption); S is the optical
    depth sum(dt * tau). `pix` selects linear pixel indices (default all).
    """
    c = _Common(volume, tf, model, view, eye, step, fp32)
    p, n = _pix(pix)
    total = n if p is not None else c.W * c.H
    img = np.zeros((total, c.nc))
    N = np.zeros(total, dtype=np.int32)
    S = np.zeros(total)
    _load().ora_render(*c.head(), c.fp32, _p(p), n, _p(img), _p(N), _p(S))
    return img, N, S


def backward(volume, tf, model, view, eye, step, grad_image, fp32=True, pix=None,
             invert=False, want=("volume", "tf", "eye", "step"), margin=0.0, sel=None):
    """Alg. 2 for one view with the stored-state tape (invert=False) or the
    inversion of Eq. inv-blend-forward (invert=True). Returns a dict of
    binary64 gradients for the requested parameters.

    With margin > 0, ambiguity bounds for a binary32 evaluation of the
    same samples (the kernel's precision) are returned as
    out["volume_ambiguity"] (per voxel) and out["eye_ambiguity"] (3): how
    far a correct gradient may move when samples closer to a kink of the
    piecewise-linear TF, or to a cell face, than binary32 rounding (times
    `margin`) take the other one-sided derivative.

    With `sel` (ascending linear vertex indices, e.g. np.unique of
    touched()), the volume gradient and its bound are returned compactly,
    one entry (four for colour volumes) per selected vertex, for volumes
    whose dense binary64 gradient would not fit in host memory; every
    vertex the rays touch must be selected.
    """
    c = _Common(volume, tf, model, view, eye, step, fp32)
    p, n = _pix(pix)
    total = n if p is not None else c.W * c.H
    gi = _f64(grad_image).reshape(total, c.nc)
    out = {}
    if sel is not None:
        sel = np.ascontiguousarray(np.asarray(sel, dtype=np.int64))
        vshape = (sel.size,) + c.vol.shape[3:]
    else:
        vshape = c.vol.shape
    gv = np.zeros(vshape) if "volume" in want else None
    gt = np.zeros((c.R, 4)) if ("tf" in want and c.model == EMISSION_ABSORPTION) else None
    ge = np.zeros(3) if "eye" in want else None
    gs = np.zeros(1) if "step" in want else None
    amb = np.zeros(vshape[:1] if sel is not None else c.vol.shape) if (gv is not None and margin > 0) else None
    amb_e = np.zeros(3) if (ge is not None and margin > 0) else None
    args = (*c.head(), c.fp32, _p(p), n, _p(gi), int(bool(invert)),
            _p(gv), _p(gt), _p(ge), _p(gs), float(margin), _p(amb), _p(amb_e))
    if sel is not None:
        miss = _load().ora_backward_sel(*args, _p(sel), sel.size)
        if miss:
            raise ValueError(f"{miss} vertex contributions fell outside `sel`")
    else:
        _load().ora_backward(*args)
    if amb is not None:
        out["volume_ambiguity"] = amb
    if amb_e is not None:
        out["eye_ambiguity"] = amb_e
    if gv is not None:
        out["volume"] = gv
    if gt is not None:
        out["tf"] = gt
    if ge is not None:
        out["eye"] = ge
    if gs is not None:
        out["step"] = gs[0]
    return out


def touched(shape, view, eye, step, pix=None, fp32=True):
    """Ascending unique linear indices of the vertices whose values the
    listed rays read (the 8 corners of every sample, Alg. 1's
    f_interpolate), for backward(..., sel=...)."""
    nz, ny, nx = shape[:3]
    W, H = int(view.width), int(view.height)
    cv = _f32val if fp32 else float
    lens = cv(view.ortho_height if view.ortho else view.tan_half_fov_y)
    e = np.array([cv(v) for v in np.asarray(eye).reshape(3)], dtype=np.float64)
    p, n = _pix(pix)
    lib = _load()
    head = (nx, ny, nz, W, H, int(bool(view.ortho)), lens, _p(e), cv(step), int(bool(fp32)), _p(p), n)
    count = lib.ora_touched(*head, None, 0)
    out = np.empty(count, dtype=np.int64)
    lib.ora_touched(*head, _p(out), count)
    return np.unique(out)


def render_dual(volume, tf, model, view, eye, step, pix=None, n_fp32=False):
    """Forward-mode (Sec. 4.2) render seeded on the eye position; binary64
    ray setup (with n_fp32, the sample count N of each ray is the binary32
    decision the kernels take). Returns (image [npix][C], dimage [npix][C][3])."""
    c = _Common(volume, tf, model, view, eye, step, False)
    if n_fp32:
        c.eye = np.array([_f32val(e) for e in c.eye])
        c.step = _f32val(c.step)
        c.lens = _f32val(c.lens)
    p, n = _pix(pix)
    total = n if p is not None else c.W * c.H
    img = np.zeros((total, c.nc))
    dimg = np.zeros((total, c.nc, 3))
    _load().ora_render_dual(*c.head(), int(bool(n_fp32)), _p(p), n, _p(img), _p(dimg))
    return img, dimg


def rays(shape, view, eye, step, fp32=True):
    """Per-pixel ray description: N, q = L/dt and geo [W*H][8] =
    (tn, tfar, x_o[3], w[3])."""
    nz, ny, nx = shape
    W, H = int(view.width), int(view.height)
    cv = _f32val if fp32 else float
    lens = cv(view.ortho_height if view.ortho else view.tan_half_fov_y)
    e = np.array([cv(v) for v in np.asarray(eye).reshape(3)], dtype=np.float64)
    N = np.zeros(W * H, dtype=np.int32)
    q = np.zeros(W * H)
    geo = np.zeros((W * H, 8))
    _load().ora_rays(nx, ny, nz, W, H, int(bool(view.ortho)), lens, _p(e), cv(step),
                     int(bool(fp32)), _p(N), _p(q), _p(geo))
    return N, q, geo


def interpolate(volume, x):
    """Trilinear density (f_interpolate) at world points x [n][3]."""
    vol = _f64(volume)
    nz, ny, nx = vol.shape
    xx = _f64(x).reshape(-1, 3)
    d = np.zeros(xx.shape[0])
    _load().ora_interpolate(_p(vol), nx, ny, nz, _p(xx), xx.shape[0], _p(d))
    return d


def orbit_eye(params):
    """Eye positions from (yaw, pitch, distance) per view (Sec. 5.1)."""
    pr = _f64(params).reshape(-1, 3)
    e = np.zeros_like(pr)
    _load().ora_orbit_eye(_p(pr), pr.shape[0], _p(e))
    return e


def orbit_eye_backward(params, grad_eye):
    pr = _f64(params).reshape(-1, 3)
    ge = _f64(grad_eye).reshape(-1, 3)
    g = np.zeros_like(pr)
    _load().ora_orbit_eye_backward(_p(pr), pr.shape[0], _p(ge), _p(g))
    return g


# ---------------------------------------------------------------------------
# Multi-view helpers: one volume list, one view list, eye [n_views][3].
# ---------------------------------------------------------------------------
def render_views(volumes, tf, model, views, eye, step, fp32=True):
    out = []
    for v, view in enumerate(views):
        img, N, S = render(volumes[view.volume_index], tf, model, view, eye[v], step, fp32)
        out.append((img, N, S))
    return out


def backward_views(volumes, tf, model, views, eye, step, grad_images, fp32=True,
                   want=("volume", "tf", "eye")):
    gv = [np.zeros(np.asarray(v).shape) for v in volumes] if "volume" in want else None
    gt = None
    ge = np.zeros((len(views), 3))
    for v, view in enumerate(views):
        g = backward(volumes[view.volume_index], tf, model, view, eye[v], step, grad_images[v],
                     fp32=fp32, want=want)
        if gv is not None:
            gv[view.volume_index] += g["volume"]
        if "tf" in g:
            gt = g["tf"] if gt is None else gt + g["tf"]
        if "eye" in g:
            ge[v] = g["eye"]
    return {"volume": gv, "tf": gt, "eye": ge}


# ---------------------------------------------------------------------------
# Optimisation-side terms (Sec. 5.2, Sec. 5.3), by their definitions.
# ---------------------------------------------------------------------------
def volume_prior(volume):
    """sum over all pairs of neighbouring vertices (along x, y, z) of the
    squared difference, and its gradient (binary64)."""
    v = _f64(volume)
    loss = 0.0
    grad = np.zeros_like(v)
    for axis in range(3):
        d = np.diff(v, axis=axis)
        loss += float((d * d).sum())
        pad_lo = [(0, 0)] * 3
        pad_hi = [(0, 0)] * 3
        pad_lo[axis] = (1, 0)
        pad_hi[axis] = (0, 1)
        # d/dv_i of (v_{i+1} - v_i)^2 = -2 d_i ; of (v_i - v_{i-1})^2 = +2 d_{i-1}
        grad += 2.0 * np.pad(d, pad_lo) - 2.0 * np.pad(d, pad_hi)
    return loss, grad


def opacity_entropy(alpha, a_min=1e-12):
    """Opacity entropy of one view (Sec. 5.1, the viewpoint-selection
    objective) and its gradient, binary64. Over the view's N pixels,
    p_i = A_i / sum_j A_j and H = -(1 / log2 N) sum_i p_i log2 p_i with
    0 log 0 = 0 (the minus sign: the paper prints H without it but reports a
    best value of 1.72 > 0, and the normalised entropy lies in [0, 1]).
    Written out: H = -(sum_i p_i ln p_i) / ln N. Its derivative is the
    quotient rule applied to p_i: dH/dA_k = -(ln p_k - sum_i p_i ln p_i) /
    (S ln N) with S = sum_j A_j; at A_k = 0, where ln p_k is -inf, the
    logarithm is taken at a_min (pixels no ray lights). Returns (H, dH/dA)."""
    a = np.asarray(alpha, dtype=np.float64).reshape(-1)
    n = a.size
    S = a.sum()
    if n < 2 or S <= 0.0:
        return 0.0, np.zeros_like(a)
    p = a / S
    plogp = np.where(a > 0, p * np.log(np.where(a > 0, p, 1.0)), 0.0)
    E = plogp.sum()
    H = -E / np.log(n)
    lnp = np.log(np.maximum(a, a_min) / S)
    grad = -(lnp - E) / (S * np.log(n))
    return float(H), grad


def tf_prior(tf):
    """Eq. tf-loss prior without its normalisation: sum_c sum_r
    (T[r+1][c] - T[r][c])^2, and its gradient."""
    t = _f64(tf)
    d = np.diff(t, axis=0)
    grad = 2.0 * np.pad(d, [(1, 0), (0, 0)]) - 2.0 * np.pad(d, [(0, 1), (0, 0)])
    return float((d * d).sum()), grad


def resample(volume, shape):
    """Trilinear resampling to `shape` (nz, ny, nx) over the same box:
    f_interpolate of the source at the world positions of the new vertices."""
    v = _f64(volume)
    dz, dy, dx = shape
    dmax = max(shape)
    coords = []
    for n in (dx, dy, dz):
        ext = (n - 1) / (dmax - 1)
        coords.append(-0.5 * ext + np.arange(n) / (dmax - 1))
    Z, Y, X = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return interpolate(v, pts).reshape(shape)
