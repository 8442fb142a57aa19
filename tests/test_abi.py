"""The C-ABI library: it loads, exports every symbol include/dvr.h declares,
its ctypes mirror matches the header's struct layout, and argument errors
are reported without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2107_12672_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dvr.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"DVR_API\s+[\w\s\*]+?\b(dvr_\w+)\s*\(", src)))


def test_header_declares_what_binding_lists():
    assert _declared() == sorted(_abi.SYMBOLS)


def test_flag_values_match_header():
    """Every DVR_FLAG_* of the header has the same value in the binding's
    mirror, and the flags are distinct bits."""
    header = open(os.path.join(ROOT, "include", "dvr.h")).read()
    flags = {k: int(v) for k, v in re.findall(r"#define (DVR_FLAG_\w+) (\d+)u", header)}
    assert "DVR_FLAG_PERSISTENT_SCATTER" in flags
    for k, v in flags.items():
        assert getattr(_abi, k) == v, k
        assert v & (v - 1) == 0, k
    assert len(set(flags.values())) == len(flags)


def test_library_loads_and_exports_every_symbol():
    lib = _abi.load()
    for name in _declared():
        assert hasattr(lib, name), name
    header = open(os.path.join(ROOT, "include", "dvr.h")).read()
    version = int(re.search(r"#define DVR_ABI_VERSION (\d+)", header).group(1))
    assert lib.dvr_abi_version() == version == _abi.ABI_VERSION
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dvr_\w+)", out))
    assert set(_declared()) <= exported
    # everything else stays hidden
    assert exported == set(_declared())


def test_bounds_checked_library_exports_the_same_abi():
    """libdvr_bounds.so (DVR_DEBUG_BOUNDS) exports exactly the symbols of
    the header and says it is the checked build; the release library says
    it is not and refuses the bounds calls without a GPU."""
    from paper_2107_12672_b300 import build
    path = build.build(bounds=True)
    lib = ctypes.CDLL(path)
    lib.dvr_last_error.restype = ctypes.c_char_p
    assert lib.dvr_abi_version() == _abi.ABI_VERSION
    assert lib.dvr_bounds_checked() == 1
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert set(re.findall(r"\bT (dvr_\w+)", out)) == set(_declared())
    # argument errors come before any CUDA call
    assert lib.dvr_bounds_cap(ctypes.c_int32(0), ctypes.c_int64(5)) == -1
    assert lib.dvr_bounds_cap(ctypes.c_int32(_abi.DVR_SITE_CELL_GRADIENT + 1), ctypes.c_int64(5)) == -1
    assert lib.dvr_bounds_cap(ctypes.c_int32(_abi.DVR_SITE_TF), ctypes.c_int64(-1)) == -1
    assert lib.dvr_bounds_status(None, 0) == -1
    rel = _abi.load()
    assert rel.dvr_bounds_checked() == 0
    out4 = (ctypes.c_int64 * 4)()
    assert rel.dvr_bounds_status(out4, 1) == -4
    assert b"DVR_DEBUG_BOUNDS" in rel.dvr_last_error()
    assert rel.dvr_bounds_cap(_abi.DVR_SITE_TF, 5) == -4


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "dvr.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu\\n", sizeof(dvr_volume), offsetof(dvr_volume, dtype), offsetof(dvr_volume, data),'
        " offsetof(dvr_volume, cells), offsetof(dvr_volume, cells_brick));\n"
        'printf("%zu %zu\\n", sizeof(dvr_tf), offsetof(dvr_tf, rgba));\n'
        'printf("%zu %zu %zu %zu\\n", sizeof(dvr_view), offsetof(dvr_view, volume), offsetof(dvr_view, lens),'
        " offsetof(dvr_view, pixel_offset));\n"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    lines = subprocess.check_output([str(exe)], text=True).split("\n")
    V, T, W = _abi.DvrVolume, _abi.DvrTF, _abi.DvrView
    assert lines[0].split() == [str(ctypes.sizeof(V)), str(V.dtype.offset), str(V.data.offset), str(V.cells.offset),
                                str(V.cells_brick.offset)]
    assert lines[1].split() == [str(ctypes.sizeof(T)), str(T.rgba.offset)]
    assert lines[2].split() == [str(ctypes.sizeof(W)), str(W.volume.offset), str(W.lens.offset),
                                str(W.pixel_offset.offset)]


def _call_forward(vols, nvol, tf, model, views, nviews, eye=1, step=0.5, image=16):
    lib = _abi.load()
    return lib.dvr_forward(vols, nvol, tf, model, views, nviews, eye, step, image, None, None, None, 0, None, 0,
                           None)


def _one_volume(nx=8, dtype=_abi.DVR_F32, data=4096):
    v = (_abi.DvrVolume * 1)()
    v[0] = _abi.DvrVolume(nx, nx, nx, dtype, data)
    return v


def _one_view(w=4, h=4, volume=0, lens=0.4, ortho=0):
    a = (_abi.DvrView * 1)()
    a[0] = _abi.DvrView(w, h, ortho, volume, lens, 0, 0)
    return a


@pytest.mark.parametrize("case,code", [
    ("null_volumes", _abi.DVR_OK - 1),
    ("bad_model", -1),
    ("small_volume", -1),
    ("bad_dtype", -2),
    ("bad_view_volume", -1),
    ("bad_lens", -1),
    ("tiny_step", -1),
    ("too_many_samples", -1),
    ("null_image", -1),
    ("ea_without_tf", -1),
    ("misaligned_image", -1),
    ("misaligned_cells", -1),
    ("cells_for_colour_volume", -1),
    ("cells_on_some_volumes", -1),
    ("bad_cells_brick", -1),
])
def test_argument_errors_need_no_gpu(case, code):
    """Invalid arguments are rejected on the host before any CUDA call."""
    vols, view = _one_volume(), _one_view()
    lib = _abi.load()
    if case == "null_volumes":
        rc = _call_forward(None, 1, None, 0, view, 1)
    elif case == "bad_model":
        rc = _call_forward(vols, 1, None, 7, view, 1)
    elif case == "small_volume":
        rc = _call_forward(_one_volume(nx=1), 1, None, 0, view, 1)
    elif case == "bad_dtype":
        rc = _call_forward(_one_volume(dtype=9), 1, None, 0, view, 1)
    elif case == "bad_view_volume":
        rc = _call_forward(vols, 1, None, 0, _one_view(volume=3), 1)
    elif case == "bad_lens":
        rc = _call_forward(vols, 1, None, 0, _one_view(lens=-1.0), 1)
    elif case == "tiny_step":
        rc = _call_forward(vols, 1, None, 0, view, 1, step=1e-6)
    elif case == "too_many_samples":
        # a 16385 x 2 x 2 box at the smallest step: its diagonal, 16384.0001
        # voxels, takes 2^24 + 2 samples, past the binary32 sample index
        long_box = (_abi.DvrVolume * 1)()
        long_box[0] = _abi.DvrVolume(16385, 2, 2, _abi.DVR_F32, 4096)
        rc = _call_forward(long_box, 1, None, 0, view, 1, step=2.0 ** -10)
        assert "2^24" in lib.dvr_last_error().decode()
    elif case == "null_image":
        rc = _call_forward(vols, 1, None, 0, view, 1, image=None)
    elif case == "ea_without_tf":
        rc = _call_forward(vols, 1, None, 1, view, 1)
    elif case == "misaligned_image":
        tf = _abi.DvrTF(4, 0, 4096)
        rc = _call_forward(vols, 1, ctypes.byref(tf), 1, view, 1, image=4100)
    elif case == "misaligned_cells":
        vols[0].cells = 8200
        rc = _call_forward(vols, 1, None, 0, view, 1)
    elif case == "cells_for_colour_volume":
        vols[0].cells = 8192
        rc = _call_forward(vols, 1, None, 2, view, 1)
    elif case == "cells_on_some_volumes":
        two = (_abi.DvrVolume * 2)()
        two[0] = _abi.DvrVolume(8, 8, 8, _abi.DVR_F32, 4096, 8192)
        two[1] = _abi.DvrVolume(8, 8, 8, _abi.DVR_F32, 4096, None)
        rc = _call_forward(two, 2, None, 0, view, 1)
    elif case == "bad_cells_brick":
        vols[0].cells = 8192
        vols[0].cells_brick = 2
        rc = _call_forward(vols, 1, None, 0, view, 1)
    assert rc == code
    assert lib.dvr_last_error().decode()


def _call_backward(workspace=4096, nbytes=256, flags=0):
    lib = _abi.load()
    return lib.dvr_backward(_one_volume(), 1, None, 0, _one_view(), 1, 16, 0.5, 64, 64, None, None,
                            128, None, flags, None, 0, workspace, nbytes, None)


def test_backward_rejects_unknown_flags():
    assert _call_backward(flags=0x80) == -1
    assert b"flag" in _abi.load().dvr_last_error()


def test_backward_workspace_size():
    lib = _abi.load()
    # one 128-byte tile-queue counter per launch of up to 512 views, rounded to 256 bytes
    assert [lib.dvr_backward_workspace_bytes(n) for n in (0, 1, 512, 513, 1024, 1025, 4096)] == \
        [0, 256, 256, 256, 256, 512, 1024]


@pytest.mark.parametrize("workspace,nbytes", [(None, 256), (4096, 255), (4104, 256)])
def test_backward_rejects_bad_workspace(workspace, nbytes):
    assert _call_backward(workspace, nbytes) == -1
    assert b"workspace" in _abi.load().dvr_last_error()


def test_no_oracle_in_the_product_path():
    """The library and its binding never import, load or include the oracle."""
    pkg = os.path.join(ROOT, "paper_2107_12672_b300")
    banned = re.compile(r"(import\s+oracle|from\s+oracle|liboracle|dvr_oracle|ora_\w+\()")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not banned.search(text), f


def test_pass_tile_widths_are_separate_and_checked():
    """The forward and adjoint tile widths are set apart; dvr_set_tile_width
    sets both; unknown passes or widths are refused and change nothing. No
    CUDA call is made."""
    lib = _abi.load()
    F, A = _abi.DVR_PASS_FORWARD, _abi.DVR_PASS_ADJOINT
    old = lib.dvr_get_pass_tile_width(F), lib.dvr_get_pass_tile_width(A)
    try:
        assert lib.dvr_set_pass_tile_width(F, 16) == 0 and lib.dvr_set_pass_tile_width(A, 4) == 0
        assert (lib.dvr_get_pass_tile_width(F), lib.dvr_get_pass_tile_width(A)) == (16, 4)
        assert lib.dvr_get_tile_width() == 16
        assert lib.dvr_set_pass_tile_width(2, 8) == -1 and b"pass" in lib.dvr_last_error()
        assert lib.dvr_set_pass_tile_width(A, 3) == -1 and b"width" in lib.dvr_last_error()
        assert lib.dvr_get_pass_tile_width(7) == -1
        assert (lib.dvr_get_pass_tile_width(F), lib.dvr_get_pass_tile_width(A)) == (16, 4)
        assert lib.dvr_set_tile_width(32) == 0
        assert (lib.dvr_get_pass_tile_width(F), lib.dvr_get_pass_tile_width(A)) == (32, 32)
    finally:
        lib.dvr_set_pass_tile_width(F, old[0])
        lib.dvr_set_pass_tile_width(A, old[1])


@pytest.mark.parametrize("R", [1, 1025])
def test_tf_row_count_limits(R):
    """2 <= R <= 1024 TF rows (the shared-memory staging limit); others are
    refused before any CUDA call."""
    lib = _abi.load()
    tf = _abi.DvrTF(R, 0, 4096)
    rc = _call_forward(_one_volume(), 1, ctypes.byref(tf), 1, _one_view(), 1)
    assert rc == -1 and b"TF has" in lib.dvr_last_error()


def test_tile_count_overflow_refused():
    """512 views of 65536^2 pixels in one launch would need more than 2^31 - 1
    warp tiles: refused on the host."""
    lib = _abi.load()
    n = 512
    views = (_abi.DvrView * n)(*[_abi.DvrView(65536, 65536, 0, 0, 0.4, 0, 65536 * 65536 * i) for i in range(n)])
    rc = _call_forward(_one_volume(), 1, None, 0, views, n)
    assert rc == -1 and b"tiles" in lib.dvr_last_error()


@pytest.mark.parametrize("kind,buf,nbytes,reps", [(3, 4096, 1 << 20, 1), (0, None, 1 << 20, 1), (0, 4104, 1 << 20, 1),
                                                  (1, 4096, 1024, 1), (2, 4096, 1 << 20, 0), (0, 4096, (1 << 20) + 4, 1)])
def test_probe_argument_errors(kind, buf, nbytes, reps):
    """dvr_probe refuses unknown kinds, NULL or misaligned buffers, sizes
    outside [32768, 2^33) or not multiples of 16, and reps < 1, before any
    CUDA call."""
    lib = _abi.load()
    assert lib.dvr_probe(kind, buf, nbytes, reps, 8192, None) == -1
    assert lib.dvr_last_error()


def test_tile_order_is_a_centre_out_permutation():
    """dvr_tile_order (host only): a permutation of each launch's tiles,
    view by view, by non-decreasing distance of the tile centre from the
    view centre; the size query writes nothing; bad arguments are refused."""
    import numpy as np
    lib = _abi.load()
    old = lib.dvr_get_pass_tile_width(_abi.DVR_PASS_FORWARD)
    try:
        lib.dvr_set_pass_tile_width(_abi.DVR_PASS_FORWARD, 8)          # tiles of 8 x 4 pixels
        views = (_abi.DvrView * 2)(_abi.DvrView(37, 21, 0, 0, 0.4, 0, 0), _abi.DvrView(16, 9, 0, 0, 0.4, 0, 777))
        n = lib.dvr_tile_order(views, 2, _abi.DVR_PASS_FORWARD, None, 0)
        t0, t1 = 5 * 6, 2 * 3                                           # ceil(37/8) x ceil(21/4), ceil(16/8) x ceil(9/4)
        assert n == t0 + t1
        out = np.zeros(n, dtype=np.uint32)
        assert lib.dvr_tile_order(views, 2, _abi.DVR_PASS_FORWARD, out.ctypes.data, n - 1) == n
        assert not out.any()
        assert lib.dvr_tile_order(views, 2, _abi.DVR_PASS_FORWARD, out.ctypes.data, n) == n
        assert sorted(out[:t0]) == list(range(t0)) and sorted(out[t0:]) == list(range(t0, n))

        def co(r, k):
            c = (k - 1) >> 1
            return c + ((r + 1) >> 1) if r & 1 else c - ((r + 1) >> 1)

        def dist(t, W, H, off):
            tx_n, ty_n = (W + 7) // 8, (H + 3) // 4
            l = t - off
            tx, ty = co(l % tx_n, tx_n), co(l // tx_n, ty_n)
            return (2 * tx * 8 + 8 - W) ** 2 + (2 * ty * 4 + 4 - H) ** 2

        d0 = [dist(int(t), 37, 21, 0) for t in out[:t0]]
        d1 = [dist(int(t), 16, 9, t0) for t in out[t0:]]
        assert d0 == sorted(d0) and d1 == sorted(d1)
        assert lib.dvr_tile_order(views, 2, 5, None, 0) == -1
        assert lib.dvr_tile_order(views, 0, _abi.DVR_PASS_FORWARD, None, 0) == -1
    finally:
        lib.dvr_set_pass_tile_width(_abi.DVR_PASS_FORWARD, old)


def test_forward_refuses_a_tile_order_of_the_wrong_length():
    lib = _abi.load()
    n = lib.dvr_tile_order(_one_view(), 1, _abi.DVR_PASS_FORWARD, None, 0)
    rc = lib.dvr_forward(_one_volume(), 1, None, 0, _one_view(), 1, 16, 0.5, 16, None, None, 4096, n + 1, None, 0,
                         None)
    assert rc == -1 and b"tile_order" in lib.dvr_last_error()


@pytest.mark.parametrize("workspace,nbytes", [(4096, 255), (4104, 256)])
def test_forward_refuses_a_bad_workspace(workspace, nbytes):
    """A persistent forward's workspace must hold the tile-queue counters
    and be 16-byte aligned; checked before any CUDA call."""
    lib = _abi.load()
    assert lib.dvr_backward_workspace_bytes(1) == 256
    rc = lib.dvr_forward(_one_volume(), 1, None, 0, _one_view(), 1, 16, 0.5, 16, None, None, None, 0, workspace,
                         nbytes, None)
    assert rc == -1 and b"workspace" in lib.dvr_last_error()


def test_checkpoint_slots_and_argument_errors():
    """dvr_checkpoint_slots: ceil((ceil(box diagonal / step) + 2) / K) per
    pixel; the checkpointed entry points refuse other models, K < 1, too few
    slots and the default recovery, before any CUDA call."""
    lib = _abi.load()
    vols = _one_volume(nx=64)
    # 64^3: diagonal sqrt(3) * 63 = 109.12 voxels; / 0.5 -> 219 steps + 2 = 221; / 16 -> 14
    assert lib.dvr_checkpoint_slots(vols, 1, 0.5, 16) == 14
    assert lib.dvr_checkpoint_slots(vols, 1, 0.5, 0) == -1
    assert lib.dvr_checkpoint_slots(None, 1, 0.5, 16) == -1
    view = _one_view()
    tf = _abi.DvrTF(4, 0, 4096)
    fwd = lambda model, k, slots: lib.dvr_forward_checkpointed(vols, 1, ctypes.byref(tf), model, view, 1, 16, 0.5, 16,
                                                               None, None, k, 8192, slots, None)
    assert fwd(_abi.DVR_ABSORPTION, 16, 14) == -4
    assert fwd(_abi.DVR_EMISSION_ABSORPTION, 0, 14) == -1
    assert fwd(_abi.DVR_EMISSION_ABSORPTION, 16, 13) == -1 and b"slots" in lib.dvr_last_error()
    bwd = lambda flags: lib.dvr_backward_checkpointed(vols, 1, ctypes.byref(tf), _abi.DVR_EMISSION_ABSORPTION, view, 1,
                                                      16, 0.5, 64, 64, None, 128, None, None, flags, 16, 8192, 14,
                                                      4096, 256, None)
    assert bwd(0) == -1 and b"alpha" in lib.dvr_last_error()


@pytest.mark.parametrize("channels,stats,grad", [(3, 8192, 4096), (4, None, 4096), (1, 8196, 4096),
                                                 (4, 8192, 4100)])
def test_loss_entropy_argument_errors(channels, stats, grad):
    """dvr_loss_entropy refuses channel counts other than 1 and 4, a missing
    or misaligned stats array and an RGBA gradient that is not 16-byte
    aligned, before any CUDA call."""
    lib = _abi.load()
    rc = lib.dvr_loss_entropy(4096, channels, _one_view(), 1, 1.0, grad, None, stats, None)
    assert rc == -1 and lib.dvr_last_error()


def test_cell_layout_size_and_argument_errors():
    """dvr_cells_bytes is 8 elements per cell; dvr_make_cells refuses a
    buffer that is too small or misaligned, before any CUDA call."""
    lib = _abi.load()
    v = _abi.DvrVolume(5, 6, 7, _abi.DVR_BF16, 4096, None)
    assert lib.dvr_cells_bytes(ctypes.byref(v)) == 4 * 5 * 6 * 8 * 2
    v32 = _abi.DvrVolume(5, 6, 7, _abi.DVR_F32, 4096, None)
    assert lib.dvr_cells_bytes(ctypes.byref(v32)) == 4 * 5 * 6 * 8 * 4
    assert lib.dvr_cells_bytes(ctypes.byref(_abi.DvrVolume(1, 6, 7, _abi.DVR_F32, 4096, None))) == 0
    # bricks of 4^3 cells: whole bricks (4 x 5 x 6 cells -> 1 x 2 x 2 bricks)
    v4 = _abi.DvrVolume(5, 6, 7, _abi.DVR_BF16, 4096, None, 4, 0)
    assert lib.dvr_cells_bytes(ctypes.byref(v4)) == 1 * 2 * 2 * 64 * 8 * 2
    # bricks of 8^3 cells: 4 x 5 x 6 cells -> one brick of 512; 9 x 5 x 17 -> 2 x 1 x 3
    v8 = _abi.DvrVolume(5, 6, 7, _abi.DVR_F32, 4096, None, 8, 0)
    assert lib.dvr_cells_bytes(ctypes.byref(v8)) == 512 * 8 * 4
    v8b = _abi.DvrVolume(10, 6, 18, _abi.DVR_F16, 4096, None, 8, 0)
    assert lib.dvr_cells_bytes(ctypes.byref(v8b)) == 2 * 1 * 3 * 512 * 8 * 2
    assert lib.dvr_cells_bytes(ctypes.byref(_abi.DvrVolume(5, 6, 7, _abi.DVR_BF16, 4096, None, 2, 0))) == 0
    assert lib.dvr_make_cells(ctypes.byref(v), 8192, 100, None) == _abi.DVR_OK - 1
    assert lib.dvr_make_cells(ctypes.byref(v), 8200, 1 << 20, None) == _abi.DVR_OK - 1
    assert lib.dvr_make_cells(ctypes.byref(_abi.DvrVolume(5, 6, 7, 9, 4096, None)), 8192, 1 << 20, None) == -2
    assert lib.dvr_last_error().decode()


def test_render_refuses_a_cell_layout_for_colour_volumes():
    """render() checks its options on the host before any CUDA call: the
    colour model has no cell layout."""
    import torch

    import paper_2107_12672_b300 as dvr
    from paper_2107_12672_b300 import synthetic as syn
    with pytest.raises(ValueError, match="colour"):
        dvr.render(torch.zeros((3, 3, 3, 4)), None, torch.zeros((1, 3)), [syn.View(2, 2)], 0.5, model="color",
                   cells=4)
