"""ctypes view of the C ABI in include/dvr.h (argument marshalling only).

The CUDA library `_lib/libdvr.so` is required: there is no CPU or
PyTorch fallback. If it is missing it is built in-tree with nvcc; if that is
impossible, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# DVR_LIBRARY may name another build of the same library (e.g. the
# bounds-checked build BOUNDS_LIB_PATH); by default the in-tree build is
# loaded.
BOUNDS_LIB_PATH = os.path.join(_HERE, "_lib", "libdvr_bounds.so")
LIB_PATH = os.environ.get("DVR_LIBRARY") or os.path.join(_HERE, "_lib", "libdvr.so")

ABI_VERSION = 13         # DVR_ABI_VERSION of the header these argtypes follow
DVR_OK = 0
DVR_F32, DVR_F16, DVR_BF16 = 0, 1, 2
DVR_ABSORPTION, DVR_EMISSION_ABSORPTION, DVR_COLOR_VOLUME = 0, 1, 2
DVR_PASS_FORWARD, DVR_PASS_ADJOINT = 0, 1
DVR_PROBE_L2_READ, DVR_PROBE_L1_READ, DVR_PROBE_L2_RED = 0, 1, 2
DVR_FLAG_TF_IMMEDIATE = 1
DVR_FLAG_INVERT_ALPHA32 = 2
DVR_FLAG_INVERT_ALPHA64 = 4
DVR_FLAG_CELL_GRADIENT = 8
DVR_FLAG_PERSISTENT_SCATTER = 16
DVR_ERR_BOUNDS = -5
DVR_SITE_VOLUME, DVR_SITE_CELLS, DVR_SITE_PIXEL, DVR_SITE_TF, DVR_SITE_CELL_GRADIENT = 1, 2, 3, 4, 5

# every symbol include/dvr.h declares
SYMBOLS = ("dvr_abi_version", "dvr_last_error", "dvr_set_tile_width", "dvr_get_tile_width",
           "dvr_set_pass_tile_width", "dvr_get_pass_tile_width", "dvr_forward", "dvr_backward",
           "dvr_backward_workspace_bytes", "dvr_forward_tangent",
           "dvr_tangent_contract", "dvr_loss_l2", "dvr_loss_l1", "dvr_tf_prior", "dvr_volume_prior",
           "dvr_resample", "dvr_orbit_eye", "dvr_orbit_eye_backward", "dvr_backward_noalloc", "dvr_probe",
           "dvr_tile_order", "dvr_checkpoint_slots", "dvr_forward_checkpointed", "dvr_backward_checkpointed",
           "dvr_loss_entropy", "dvr_cells_bytes", "dvr_make_cells", "dvr_backward_cell_workspace_bytes",
           "dvr_bounds_checked", "dvr_bounds_status", "dvr_bounds_cap")


class DvrVolume(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("data", ctypes.c_void_p), ("cells", ctypes.c_void_p),
                ("cells_brick", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class DvrTF(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("dtype", ctypes.c_int32), ("rgba", ctypes.c_void_p)]


class DvrView(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("ortho", ctypes.c_int32),
                ("volume", ctypes.c_int32), ("lens", ctypes.c_float), ("reserved", ctypes.c_int32),
                ("pixel_offset", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libdvr.so (building it first if it does not exist)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if os.environ.get("DVR_LIBRARY"):
                raise DVRError(f"DVR_LIBRARY={LIB_PATH} does not exist")
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        P, I32, I64, F, U32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                               ctypes.c_uint32)
        lib.dvr_abi_version.restype = ctypes.c_int
        if lib.dvr_abi_version() != ABI_VERSION:
            raise DVRError(f"{LIB_PATH} has ABI version {lib.dvr_abi_version()}, the binding expects "
                           f"{ABI_VERSION}: rebuild it")
        lib.dvr_set_tile_width.argtypes = [I32]
        lib.dvr_set_tile_width.restype = ctypes.c_int
        lib.dvr_get_tile_width.restype = ctypes.c_int
        lib.dvr_set_pass_tile_width.argtypes = [I32, I32]
        lib.dvr_set_pass_tile_width.restype = ctypes.c_int
        lib.dvr_get_pass_tile_width.argtypes = [I32]
        lib.dvr_get_pass_tile_width.restype = ctypes.c_int
        lib.dvr_last_error.restype = ctypes.c_char_p
        lib.dvr_forward.argtypes = [P, I32, P, I32, P, I32, P, F, P, P, P, P, I64, P, ctypes.c_size_t, P]
        lib.dvr_backward.argtypes = [P, I32, P, I32, P, I32, P, F, P, P, P, P, P, P, U32, P, I64, P,
                                     ctypes.c_size_t, P]
        lib.dvr_checkpoint_slots.argtypes = [P, I32, F, I32]
        lib.dvr_checkpoint_slots.restype = ctypes.c_int32
        lib.dvr_forward_checkpointed.argtypes = [P, I32, P, I32, P, I32, P, F, P, P, P, I32, P, I32, P]
        lib.dvr_forward_checkpointed.restype = ctypes.c_int
        lib.dvr_backward_checkpointed.argtypes = [P, I32, P, I32, P, I32, P, F, P, P, P, P, P, P, U32, I32, P, I32,
                                                  P, ctypes.c_size_t, P]
        lib.dvr_backward_checkpointed.restype = ctypes.c_int
        lib.dvr_loss_entropy.argtypes = [P, I32, P, I32, F, P, P, P, P]
        lib.dvr_loss_entropy.restype = ctypes.c_int
        lib.dvr_tile_order.argtypes = [P, I32, I32, P, I64]
        lib.dvr_tile_order.restype = ctypes.c_int64
        lib.dvr_backward_workspace_bytes.argtypes = [I32]
        lib.dvr_backward_workspace_bytes.restype = ctypes.c_size_t
        lib.dvr_backward_noalloc.argtypes = [P, I32, P, I32, P, I32, P, F, P, P, P, P, P, P, U32, P]
        lib.dvr_backward_noalloc.restype = ctypes.c_int
        lib.dvr_backward_cell_workspace_bytes.argtypes = [P, I32, I32]
        lib.dvr_backward_cell_workspace_bytes.restype = ctypes.c_size_t
        lib.dvr_cells_bytes.argtypes = [P]
        lib.dvr_cells_bytes.restype = ctypes.c_size_t
        lib.dvr_make_cells.argtypes = [P, P, ctypes.c_size_t, P]
        lib.dvr_make_cells.restype = ctypes.c_int
        lib.dvr_probe.argtypes = [I32, P, ctypes.c_size_t, I32, P, P]
        lib.dvr_probe.restype = ctypes.c_int
        lib.dvr_forward_tangent.argtypes = [P, I32, P, I32, P, I32, P, F, P, P, P]
        lib.dvr_tangent_contract.argtypes = [P, I32, I32, P, P, P, P]
        lib.dvr_loss_l2.argtypes = [P, P, I64, F, P, P, P]
        lib.dvr_loss_l1.argtypes = [P, P, I64, F, P, P, P]
        lib.dvr_tf_prior.argtypes = [P, I32, F, P, P, P]
        lib.dvr_volume_prior.argtypes = [P, I32, I32, I32, F, P, P, P]
        lib.dvr_resample.argtypes = [P, I32, I32, I32, P, I32, I32, I32, P]
        lib.dvr_orbit_eye.argtypes = [P, I32, P, P]
        lib.dvr_orbit_eye_backward.argtypes = [P, P, I32, P, P]
        lib.dvr_bounds_checked.restype = ctypes.c_int
        lib.dvr_bounds_status.argtypes = [P, I32]
        lib.dvr_bounds_status.restype = ctypes.c_int
        lib.dvr_bounds_cap.argtypes = [I32, I64]
        lib.dvr_bounds_cap.restype = ctypes.c_int
        for name in ("dvr_forward", "dvr_backward", "dvr_forward_tangent", "dvr_tangent_contract",
                     "dvr_loss_l2", "dvr_loss_l1", "dvr_tf_prior", "dvr_volume_prior", "dvr_resample",
                     "dvr_orbit_eye", "dvr_orbit_eye_backward"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


class DVRError(RuntimeError):
    pass


def check(rc: int, what: str):
    if rc != DVR_OK:
        msg = load().dvr_last_error().decode(errors="replace")
        raise DVRError(f"{what} failed with code {rc}: {msg}")
