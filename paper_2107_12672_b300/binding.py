"""PyTorch-facing binding of the C ABI (marshalling only).

Every step of the rendering and of its adjoint runs in the CUDA kernels of
libdvr.so; this module only turns tensors into pointers, descriptors and
the current stream, and allocates outputs with PyTorch.

    image, aux = forward(volumes, tf, "emission_absorption", views, eye, 0.5)
    grads = backward(volumes, tf, "emission_absorption", views, eye, 0.5, aux, grad_image,
                     want=("tf", "eye"))
    image = render(volume, tf, eye, views, 0.5, "emission_absorption")   # autograd
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from .synthetic import View

__all__ = ["View", "Scene", "make_cells", "cell_workspace_bytes", "forward", "backward", "forward_tangent", "tangent_contract", "loss_l2",
           "loss_l1", "tf_prior", "volume_prior", "resample", "volume_smoothness", "orbit_eye", "orbit_eye_backward",
           "render", "orbit_camera", "split_views", "MODELS"]

MODELS = {"absorption": _abi.DVR_ABSORPTION, "emission_absorption": _abi.DVR_EMISSION_ABSORPTION,
          "color": _abi.DVR_COLOR_VOLUME}
_DTYPES = {torch.float32: _abi.DVR_F32, torch.float16: _abi.DVR_F16, torch.bfloat16: _abi.DVR_BF16}


def _model(m) -> int:
    return MODELS[m] if isinstance(m, str) else int(m)


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _require_cuda(t, name):
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclass
class Scene:
    """Descriptor arrays for one set of volumes, TF and views."""
    volumes: list
    tf: torch.Tensor | None
    model: int
    views: list
    vol_desc: ctypes.Array
    tf_desc: _abi.DvrTF | None
    view_desc: ctypes.Array
    pixels: int
    channels: int
    offsets: list

    @staticmethod
    def make(volumes, tf, model, views, cells=None, cells_brick=1) -> "Scene":
        """`cells`: None, or one cell layout per volume (make_cells, all in
        the record order `cells_brick`), which the march kernels then read
        instead of the volumes' arrays."""
        if isinstance(volumes, torch.Tensor):
            volumes = [volumes]
        model = _model(model)
        if cells is not None and len(cells) != len(volumes):
            raise ValueError("one cell layout per volume")
        vd = (_abi.DvrVolume * len(volumes))()
        for i, v in enumerate(volumes):
            _require_cuda(v, f"volume {i}")
            if model == _abi.DVR_COLOR_VOLUME:
                if v.dim() != 4 or v.shape[3] != 4:
                    raise ValueError("a colour volume is a [nz][ny][nx][4] tensor")
            elif v.dim() != 3:
                raise ValueError("a volume is a 3-D tensor [nz][ny][nx]")
            if v.dtype not in _DTYPES:
                raise ValueError(f"volume dtype {v.dtype} unsupported")
            nz, ny, nx = v.shape[:3]
            c = None
            if cells is not None:
                _require_cuda(cells[i], f"cells {i}")
                c = cells[i].data_ptr()
            vd[i] = _abi.DvrVolume(nx, ny, nz, _DTYPES[v.dtype], v.data_ptr(), c, int(cells_brick), 0)
        td = None
        if model == _abi.DVR_EMISSION_ABSORPTION:
            _require_cuda(tf, "tf")
            if tf.dim() != 2 or tf.shape[1] != 4:
                raise ValueError("the transfer function is a [R][4] tensor")
            if tf.dtype not in (torch.float32, torch.float16):
                raise ValueError("TF dtype must be float32 or float16")
            td = _abi.DvrTF(tf.shape[0], _DTYPES[tf.dtype], tf.data_ptr())
        wd = (_abi.DvrView * len(views))()
        off = 0
        offsets = []
        for i, w in enumerate(views):
            lens = w.ortho_height if w.ortho else w.tan_half_fov_y
            wd[i] = _abi.DvrView(int(w.width), int(w.height), int(bool(w.ortho)),
                                 int(getattr(w, "volume_index", 0)), float(lens), 0, off)
            offsets.append(off)
            off += int(w.width) * int(w.height)
        ch = 1 if model == _abi.DVR_ABSORPTION else 4
        sc = Scene(list(volumes), tf, model, list(views), vd, td, wd, off, ch, offsets)
        sc.cells = list(cells) if cells is not None else None      # kept alive with the descriptors
        sc.cells_brick = int(cells_brick)
        return sc

    def tf_ref(self):
        return ctypes.byref(self.tf_desc) if self.tf_desc is not None else None

    def tile_order(self, lib, adjoint: bool):
        """(device uint32 tensor, length) of the centre-out tile order for
        the tile width now in force for the pass (dvr_tile_order), made
        once per scene and width."""
        pass_ = _abi.DVR_PASS_ADJOINT if adjoint else _abi.DVR_PASS_FORWARD
        width = int(lib.dvr_get_pass_tile_width(pass_))
        cache = self.__dict__.setdefault("_orders", {})
        key = (pass_, width)
        if key not in cache:
            n = int(lib.dvr_tile_order(self.view_desc, len(self.views), pass_, None, 0))
            if n < 0:
                raise _abi.DVRError(f"dvr_tile_order: {lib.dvr_last_error().decode()}")
            host = np.empty(n, dtype=np.uint32)
            got = int(lib.dvr_tile_order(self.view_desc, len(self.views), pass_, host.ctypes.data, n))
            if got != n:
                raise _abi.DVRError(f"dvr_tile_order: {lib.dvr_last_error().decode()}")
            dev = torch.from_numpy(host.view(np.int32)).to(self.volumes[0].device)
            cache[key] = (dev, n)
        return cache[key]

    def workspace(self, lib, stream=None) -> torch.Tensor:
        """Fresh adjoint workspace (tile-queue counters) from the caching
        allocator, tied to the stream the call runs on."""
        n = int(lib.dvr_backward_workspace_bytes(len(self.views)))
        ws = torch.empty(n, dtype=torch.uint8, device=self.volumes[0].device)
        if stream is not None:
            ws.record_stream(stream)
        return ws


def cell_workspace_bytes(scene: Scene) -> int:
    """Workspace bytes of backward(..., cell_gradient=True) on this scene
    (dvr_backward_cell_workspace_bytes)."""
    return int(_abi.load().dvr_backward_cell_workspace_bytes(scene.vol_desc, len(scene.volumes),
                                                             len(scene.views)))


def make_cells(volume: torch.Tensor, out: torch.Tensor | None = None, stream=None, brick: int = 1) -> torch.Tensor:
    """The cell layout of `volume` (dvr_make_cells): per cell its 8 corner
    values, 8x the volume's bytes, as a flat tensor of the volume's dtype
    (written into `out` if given), records in row order (brick 1) or in
    bricks of 4^3 or 8^3 cells (brick 4 or 8). Remake it whenever the volume
    changes."""
    _require_cuda(volume, "volume")
    if volume.dim() != 3 or volume.dtype not in _DTYPES:
        raise ValueError("cell layout: a 3-D float32/float16/bfloat16 volume")
    lib = _abi.load()
    nz, ny, nx = volume.shape
    desc = _abi.DvrVolume(nx, ny, nz, _DTYPES[volume.dtype], volume.data_ptr(), None, int(brick), 0)
    nbytes = int(lib.dvr_cells_bytes(ctypes.byref(desc)))
    n = nbytes // volume.element_size()
    if out is None:
        out = torch.empty(n, dtype=volume.dtype, device=volume.device)
    elif out.numel() * out.element_size() < nbytes or out.dtype != volume.dtype or not out.is_contiguous():
        raise ValueError("out is too small, of another dtype or not contiguous")
    _abi.check(lib.dvr_make_cells(ctypes.byref(desc), out.data_ptr(), out.numel() * out.element_size(),
                                  _stream_ptr(stream)), "dvr_make_cells")
    return out


def checkpoint_slots(scene: "Scene", step_voxels, k: int) -> int:
    """Floats per pixel for the per-K-step opacity checkpoints of the
    alpha-form recovery (dvr_checkpoint_slots)."""
    n = int(_abi.load().dvr_checkpoint_slots(scene.vol_desc, len(scene.volumes), float(step_voxels), int(k)))
    if n < 0:
        raise _abi.DVRError(f"dvr_checkpoint_slots: {_abi.load().dvr_last_error().decode()}")
    return n


def forward(volumes, tf, model, views, eye, step_voxels, *, scene: Scene | None = None, image=None,
            aux=None, sample_count=None, stream=None, checkpoints=None, workspace=None):
    """Alg. 1 for all views in one persistent launch (its tile-queue
    workspace from `workspace`, a uint8 tensor of at least
    dvr_backward_workspace_bytes(n_views) bytes, or else from torch's
    caching allocator). Returns (image [P][C], aux [P][2]).
    `checkpoints` = (tensor [P][slots], K): also record the transmittance
    before every K-th sample (dvr_forward_checkpointed, one tile per warp)."""
    sc = scene or Scene.make(volumes, tf, model, views)
    dev = sc.volumes[0].device
    _require_cuda(eye, "eye")
    if eye.dtype != torch.float32 or eye.numel() != 3 * len(sc.views):
        raise ValueError("eye must be float32 [n_views][3]")
    if image is None:
        image = torch.empty((sc.pixels, sc.channels), device=dev, dtype=torch.float32)
    if aux is None:
        aux = torch.empty((sc.pixels, 2), device=dev, dtype=torch.float32)
    lib = _abi.load()
    if checkpoints is not None:
        ck, k = checkpoints
        rc = lib.dvr_forward_checkpointed(sc.vol_desc, len(sc.volumes), sc.tf_ref(), sc.model, sc.view_desc,
                                          len(sc.views), _ptr(eye), float(step_voxels), _ptr(image), _ptr(aux),
                                          _ptr(sample_count), int(k), _ptr(ck), int(ck.shape[1]),
                                          _stream_ptr(stream))
        _abi.check(rc, "dvr_forward_checkpointed")
        return image, aux
    # the forward keeps the fixed tile order: the centre-out order measured no
    # faster on one 512^2 view and 3% slower on 64 uneven views (B300)
    ws = workspace if workspace is not None else sc.workspace(lib, stream)
    rc = lib.dvr_forward(sc.vol_desc, len(sc.volumes), sc.tf_ref(), sc.model, sc.view_desc,
                         len(sc.views), _ptr(eye), float(step_voxels), _ptr(image), _ptr(aux),
                         _ptr(sample_count), None, 0, _ptr(ws), ws.numel(), _stream_ptr(stream))
    _abi.check(rc, "dvr_forward")
    return image, aux


def backward(volumes, tf, model, views, eye, step_voxels, aux, grad_image, *, want=("volume", "tf", "eye"),
             scene: Scene | None = None, grads: dict | None = None, tf_immediate=False, inversion="depth",
             stream=None, checkpoints=None, cell_gradient=False, workspace=None, persistent_scatter=False):
    """Alg. 2 for all views in one launch. Returns a dict with float32
    gradients for the requested parameters ("volume" -> list, "tf", "eye",
    "step"); buffers passed in `grads` are accumulated into. `inversion`
    selects how the opacity before each sample is recovered: "depth"
    (default), or the ablations "alpha32" / "alpha64" (the paper's form),
    which with `checkpoints` = (tensor, K) from a checkpointed forward
    restart from the forward's value every K samples. `cell_gradient`
    accumulates the volume gradient per cell first
    (DVR_FLAG_CELL_GRADIENT); its workspace, 32 bytes per cell, comes from
    `workspace` (a uint8 tensor of at least cell_workspace_bytes(scene)
    bytes, kept by the caller) or else from torch's caching allocator.
    `persistent_scatter` makes the volume-gradient adjoint of 16-bit
    volumes a persistent launch whose warps take tiles from a queue
    (DVR_FLAG_PERSISTENT_SCATTER; the adjoint without a volume gradient
    always is one; binary32 volumes keep one tile per warp)."""
    sc = scene or Scene.make(volumes, tf, model, views)
    dev = sc.volumes[0].device
    g = dict(grads or {})
    if "volume" in want and "volume" not in g:
        g["volume"] = [torch.zeros(v.shape, device=dev, dtype=torch.float32) for v in sc.volumes]
    if "tf" in want and sc.model == _abi.DVR_EMISSION_ABSORPTION and "tf" not in g:
        g["tf"] = torch.zeros((sc.tf.shape[0], 4), device=dev, dtype=torch.float32)
    if "eye" in want and "eye" not in g:
        g["eye"] = torch.zeros((len(sc.views), 3), device=dev, dtype=torch.float32)
    if "step" in want and "step" not in g:
        g["step"] = torch.zeros(1, device=dev, dtype=torch.float32)
    gv = None
    if "volume" in g:
        gv = (ctypes.c_void_p * len(sc.volumes))(*[_ptr(t) for t in g["volume"]])
    flags = _abi.DVR_FLAG_TF_IMMEDIATE if tf_immediate else 0
    flags |= {"depth": 0, "alpha32": _abi.DVR_FLAG_INVERT_ALPHA32, "alpha64": _abi.DVR_FLAG_INVERT_ALPHA64}[inversion]
    if persistent_scatter:
        flags |= _abi.DVR_FLAG_PERSISTENT_SCATTER
    lib = _abi.load()
    if cell_gradient and "volume" in g:
        flags |= _abi.DVR_FLAG_CELL_GRADIENT
        ws = workspace if workspace is not None else torch.empty(cell_workspace_bytes(sc), dtype=torch.uint8,
                                                                 device=dev)
        if stream is not None and workspace is None:
            ws.record_stream(stream)
    else:
        ws = workspace if workspace is not None else sc.workspace(lib, stream)
    if checkpoints is not None:
        ck, k = checkpoints
        rc = lib.dvr_backward_checkpointed(sc.vol_desc, len(sc.volumes), sc.tf_ref(), sc.model, sc.view_desc,
                                           len(sc.views), _ptr(eye), float(step_voxels), _ptr(aux),
                                           _ptr(grad_image), gv, _ptr(g.get("tf")), _ptr(g.get("eye")),
                                           _ptr(g.get("step")), flags, int(k), _ptr(ck), int(ck.shape[1]),
                                           _ptr(ws), ws.numel(), _stream_ptr(stream))
        _abi.check(rc, "dvr_backward_checkpointed")
        return g
    # centre-out tile order for the adjoints without a density gradient: 0.365
    # -> 0.351 ms on a 512^2 view of a 256^3 volume (B300). The scattering
    # adjoints keep the fixed order, in which the density gradients of
    # 512^3 and 1024^3 volumes (in HBM) accumulate 5-7% faster.
    order, n_order = (None, 0) if "volume" in g else sc.tile_order(lib, adjoint=True)
    rc = lib.dvr_backward(sc.vol_desc, len(sc.volumes), sc.tf_ref(), sc.model, sc.view_desc,
                          len(sc.views), _ptr(eye), float(step_voxels), _ptr(aux),
                          _ptr(grad_image), gv, _ptr(g.get("tf")), _ptr(g.get("eye")),
                          _ptr(g.get("step")), flags, _ptr(order), n_order, _ptr(ws), ws.numel(),
                          _stream_ptr(stream))
    _abi.check(rc, "dvr_backward")
    return g


def forward_tangent(volumes, tf, model, views, eye, step_voxels, *, scene: Scene | None = None, image=None,
                    tangent=None, stream=None):
    """Forward-mode pass (Sec. 4.2): image [P][C] and d(image)/d(eye)
    [P][C][3] in one launch."""
    sc = scene or Scene.make(volumes, tf, model, views)
    dev = sc.volumes[0].device
    if image is None:
        image = torch.empty((sc.pixels, sc.channels), device=dev, dtype=torch.float32)
    if tangent is None:
        tangent = torch.empty((sc.pixels, sc.channels, 3), device=dev, dtype=torch.float32)
    rc = _abi.load().dvr_forward_tangent(sc.vol_desc, len(sc.volumes), sc.tf_ref(), sc.model, sc.view_desc,
                                         len(sc.views), _ptr(eye), float(step_voxels), _ptr(image),
                                         _ptr(tangent), _stream_ptr(stream))
    _abi.check(rc, "dvr_forward_tangent")
    return image, tangent


def tangent_contract(scene: Scene, tangent, grad_image, *, grad_eye=None, stream=None):
    """Camera gradient from tangents: grad_eye[v] += sum G * d(image)/d(eye)."""
    if grad_eye is None:
        grad_eye = torch.zeros((len(scene.views), 3), device=tangent.device, dtype=torch.float32)
    rc = _abi.load().dvr_tangent_contract(scene.view_desc, len(scene.views), scene.model, _ptr(tangent),
                                          _ptr(grad_image), _ptr(grad_eye), _stream_ptr(stream))
    _abi.check(rc, "dvr_tangent_contract")
    return grad_eye


def loss_l2(image, target, scale=1.0, *, grad_image=None, loss=None, stream=None):
    """L2 loss seed of Alg. 2: loss += scale*sum((x-y)^2), grad = 2 scale (x-y)."""
    if grad_image is None:
        grad_image = torch.empty_like(image)
    rc = _abi.load().dvr_loss_l2(_ptr(image), _ptr(target), image.numel(), float(scale),
                                 _ptr(grad_image), _ptr(loss), _stream_ptr(stream))
    _abi.check(rc, "dvr_loss_l2")
    return grad_image


def loss_entropy(image, scene: "Scene", scale=1.0, *, grad_image=None, loss=None, stream=None):
    """Opacity-entropy loss of Sec. 5.1 (maximised): loss += scale * sum over
    the scene's views of -H, with H the normalised entropy of the view's
    opacities; returns grad_image (dL/d(image), zero in colour channels)."""
    if grad_image is None:
        grad_image = torch.empty_like(image)
    stats = torch.empty((len(scene.views), 2), dtype=torch.float64, device=image.device)
    rc = _abi.load().dvr_loss_entropy(_ptr(image), int(image.shape[1]), scene.view_desc, len(scene.views),
                                      float(scale), _ptr(grad_image), _ptr(loss), _ptr(stats),
                                      _stream_ptr(stream))
    _abi.check(rc, "dvr_loss_entropy")
    return grad_image


def loss_l1(image, target, scale=1.0, *, grad_image=None, loss=None, stream=None):
    """L1 loss of Eq. tf-loss: loss += scale*sum|x-y|, grad = scale*sign(x-y)."""
    if grad_image is None:
        grad_image = torch.empty_like(image)
    rc = _abi.load().dvr_loss_l1(_ptr(image), _ptr(target), image.numel(), float(scale), _ptr(grad_image),
                                 _ptr(loss), _stream_ptr(stream))
    _abi.check(rc, "dvr_loss_l1")
    return grad_image


def tf_prior(tf, weight, *, grad=None, loss=None, stream=None):
    """Smoothing prior of Eq. tf-loss with the paper's normalisation
    weight / (4 (R - 1)); returns (loss[1], grad) accumulated into the given
    buffers (fresh zeros otherwise)."""
    R = tf.shape[0]
    loss = torch.zeros(1, device=tf.device) if loss is None else loss
    grad = torch.zeros_like(tf) if grad is None else grad
    rc = _abi.load().dvr_tf_prior(_ptr(tf), R, float(weight) / (4 * (R - 1)), _ptr(grad), _ptr(loss),
                                  _stream_ptr(stream))
    _abi.check(rc, "dvr_tf_prior")
    return loss, grad


def volume_prior(volume, weight, *, grad=None, loss=None, stream=None):
    """3D smoothing prior (Sec. 5.3): weight times the mean over all pairs of
    neighbouring vertices of their squared difference."""
    nz, ny, nx = volume.shape
    pairs = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    loss = torch.zeros(1, device=volume.device) if loss is None else loss
    grad = torch.zeros_like(volume) if grad is None else grad
    rc = _abi.load().dvr_volume_prior(_ptr(volume), nx, ny, nz, float(weight) / pairs, _ptr(grad), _ptr(loss),
                                      _stream_ptr(stream))
    _abi.check(rc, "dvr_volume_prior")
    return loss, grad


def resample(volume, shape, *, out=None, stream=None):
    """Trilinear resampling of a float32 vertex grid to `shape` (nz, ny, nx)
    over the same box (multi-resolution schedule, Sec. 5.3)."""
    sz, sy, sx = volume.shape
    dz, dy, dx = shape
    out = torch.empty(shape, device=volume.device, dtype=torch.float32) if out is None else out
    rc = _abi.load().dvr_resample(_ptr(volume), sx, sy, sz, _ptr(out), dx, dy, dz, _stream_ptr(stream))
    _abi.check(rc, "dvr_resample")
    return out


class _VolumePriorFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, volume, weight):
        loss, grad = volume_prior(volume.detach().contiguous(), weight)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None


def volume_smoothness(volume, weight):
    """Differentiable 3D smoothing prior (autograd)."""
    return _VolumePriorFn.apply(volume, float(weight))


def orbit_eye(params, *, eye=None, stream=None):
    """Eye positions [n][3] from orbit parameters (yaw, pitch, distance) [n][3]."""
    _require_cuda(params, "params")
    if eye is None:
        eye = torch.empty_like(params)
    rc = _abi.load().dvr_orbit_eye(_ptr(params), params.shape[0], _ptr(eye), _stream_ptr(stream))
    _abi.check(rc, "dvr_orbit_eye")
    return eye


def orbit_eye_backward(params, grad_eye, *, grad_params=None, stream=None):
    if grad_params is None:
        grad_params = torch.zeros_like(params)
    rc = _abi.load().dvr_orbit_eye_backward(_ptr(params), _ptr(grad_eye), params.shape[0],
                                            _ptr(grad_params), _stream_ptr(stream))
    _abi.check(rc, "dvr_orbit_eye_backward")
    return grad_params


def split_views(image, scene_or_views):
    """Split a flat [P][C] image into per-view [H][W][C] tensors."""
    views = scene_or_views.views if isinstance(scene_or_views, Scene) else scene_or_views
    out, off = [], 0
    for w in views:
        n = w.width * w.height
        out.append(image[off:off + n].view(w.height, w.width, -1))
        off += n
    return out


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, spec, eye, tf, *volumes):
        model, views, step, tf_immediate, cells, cell_gradient, persistent_scatter = spec
        layouts = [make_cells(v, brick=cells) for v in volumes] if cells else None
        sc = Scene.make(list(volumes), tf, model, views, cells=layouts, cells_brick=cells or 1)
        image, aux = forward(None, None, None, None, eye, step, scene=sc)
        ctx.spec = spec
        ctx.layouts = layouts            # the cell layouts the adjoint gathers from too
        ctx.save_for_backward(eye, tf, aux, *volumes)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        model, views, step, tf_immediate, cells, cell_gradient, persistent_scatter = ctx.spec
        eye, tf, aux, *volumes = ctx.saved_tensors
        sc = Scene.make(volumes, tf, model, views, cells=ctx.layouts, cells_brick=cells or 1)
        want = []
        if ctx.needs_input_grad[1]:
            want.append("eye")
        if tf is not None and ctx.needs_input_grad[2]:
            want.append("tf")
        if any(ctx.needs_input_grad[3:]):
            want.append("volume")
        g = backward(None, None, None, None, eye, step, aux, grad_image.contiguous(), want=tuple(want),
                     scene=sc, tf_immediate=tf_immediate, cell_gradient=cell_gradient,
                     persistent_scatter=persistent_scatter)
        ctx.layouts = None
        gvol = g.get("volume") or [None] * len(volumes)
        gvol = [gv if need else None for gv, need in zip(gvol, ctx.needs_input_grad[3:])]
        return (None, g.get("eye"), g.get("tf"), *gvol)


def render(volumes, tf, eye, views, step_voxels, model="emission_absorption", tf_immediate=False, *, cells=0,
           cell_gradient=False, persistent_scatter=False):
    """Differentiable render of all views: image [P][C] (C = 4 or 1).
    Gradients flow to eye, tf and the volumes (Alg. 2). `cells` (1, 4 or
    8) makes both passes gather from the volumes' cell layout with records
    in row order or in bricks of that edge (made from the volumes on every
    call and kept until the backward: 8x their bytes; not for the colour
    model); `cell_gradient` and `persistent_scatter` choose how the volume
    gradient is accumulated and launched, as in backward(). The autotuner
    (autotune.autotune) times all three for a workload."""
    if isinstance(volumes, torch.Tensor):
        volumes = [volumes]
    m = _model(model)
    if cells and m == _abi.DVR_COLOR_VOLUME:
        raise ValueError("the cell layout is not made for colour volumes")
    spec = (m, list(views), float(step_voxels), bool(tf_immediate), int(cells), bool(cell_gradient),
            bool(persistent_scatter))
    return _RenderFn.apply(spec, eye, tf, *volumes)


class _OrbitFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params):
        ctx.save_for_backward(params)
        return orbit_eye(params.contiguous())

    @staticmethod
    def backward(ctx, grad_eye):
        (params,) = ctx.saved_tensors
        return orbit_eye_backward(params.contiguous(), grad_eye.contiguous())


def orbit_camera(params):
    """Differentiable eye positions from (yaw, pitch, distance) [n][3]."""
    return _OrbitFn.apply(params)
