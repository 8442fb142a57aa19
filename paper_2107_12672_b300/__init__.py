"""B300-native differentiable direct volume rendering (Weiss & Westermann,
"Differentiable Direct Volume Rendering").

The forward march (Alg. 1) and its constant-memory adjoint (Alg. 2 with the
inversion of Sec. 4.4) are hand-written CUDA kernels for sm_103a behind the
C ABI of include/dvr.h; `render` wraps them in a torch.autograd.Function.
The CUDA library is loaded on first use; nothing falls back to the CPU.
"""
from . import synthetic
from .synthetic import View

__all__ = ["synthetic", "View", "forward", "backward", "forward_tangent", "tangent_contract", "render", "loss_l2", "orbit_eye",
           "orbit_eye_backward", "orbit_camera", "Scene", "split_views", "checkpoint_slots",
           "loss_entropy", "make_cells", "cell_workspace_bytes", "lib"]


def __getattr__(name):
    # the torch binding (and with it the CUDA library) loads lazily, so that
    # the input generators can be imported without CUDA
    if name in ("forward", "backward", "forward_tangent", "tangent_contract", "render", "loss_l2", "loss_l1",
                "tf_prior", "volume_prior", "resample", "volume_smoothness", "orbit_eye",
                "orbit_eye_backward", "orbit_camera", "Scene", "split_views", "MODELS", "checkpoint_slots",
                "loss_entropy", "make_cells", "cell_workspace_bytes"):
        from . import binding as _r
        return getattr(_r, name)
    if name == "lib":
        from . import _abi
        return _abi.load()
    raise AttributeError(name)
