"""Cases for the bounds-checked library (DVR_DEBUG_BOUNDS), run in a process
of their own because a process loads one build of the library.

    DVR_LIBRARY=<libdvr_bounds.so> python -m tests.bounds_cases OUT.npz

runs `cases()` (forward, adjoint, forward-mode and cell-layout calls on small
scenes), then `caps()` (each check site's extent lowered below the true one,
so that in-bounds indices fail their check: the calls must report
DVR_ERR_BOUNDS naming the site, with no bad access), and writes every output,
the bounds records and the return codes to OUT.npz. The test calls `cases()`
with the release library in its own process and compares.
"""
from __future__ import annotations

import ctypes
import json
import sys

import numpy as np
import torch

import paper_2107_12672_b300 as dvr
from paper_2107_12672_b300 import _abi
from paper_2107_12672_b300 import synthetic as syn


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a)).to("cuda", dtype).contiguous()


def _grad_image(pixels, channels, seed):
    return _dev(np.random.default_rng(seed).normal(size=(pixels, channels)).astype(np.float32))


def scenes():
    """(name, scene, eye, step, want, cell_gradient) of the cases."""
    out = []
    views = [syn.View(37, 29), syn.View(20, 21, volume_index=1), syn.View(16, 11, ortho=True, ortho_height=1.2)]
    eye = _dev((syn.fibonacci_sphere(3) * 2.2).astype(np.float32))
    tf = _dev(syn.random_tf(16, seed=4))
    v32 = [_dev(syn.value_noise(n, seed=s)[:, :n - 3, :]) for n, s in ((33, 2), (24, 3))]
    out.append(("ea_f32", dvr.Scene.make(v32, tf, "emission_absorption", views), eye, 0.4,
                ("volume", "tf", "eye"), False))
    v16 = [v.to(torch.float16) for v in v32]
    c4 = [dvr.make_cells(v, brick=4) for v in v16]
    out.append(("ea_f16_bricks_cellgrad", dvr.Scene.make(v16, tf, "emission_absorption", views, cells=c4,
                                                         cells_brick=4), eye, 0.4, ("volume", "tf", "eye"), True))
    vb = [v.to(torch.bfloat16) for v in v32]
    c1 = [dvr.make_cells(v, brick=1) for v in vb]
    out.append(("abs_bf16_rows", dvr.Scene.make(vb, None, "absorption", views, cells=c1, cells_brick=1), eye, 0.4,
                ("volume", "eye"), False))
    cv = _dev(syn.color_volume(24, seed=31))
    out.append(("color", dvr.Scene.make([cv], None, "color", [syn.View(23, 19)]), eye[:1].contiguous(), 0.5,
                ("volume", "eye"), False))
    return out


def cases() -> dict:
    """Outputs of every case with the library this process loaded."""
    res = {}
    for name, sc, eye, step, want, cg in scenes():
        img, aux = dvr.forward(None, None, None, None, eye, step, scene=sc)
        G = _grad_image(sc.pixels, sc.channels, 9)
        g = dvr.backward(None, None, None, None, eye, step, aux, G, scene=sc, want=want, cell_gradient=cg)
        torch.cuda.synchronize()
        res[f"{name}/image"] = img.cpu().numpy()
        res[f"{name}/aux"] = aux.cpu().numpy()
        for i, t in enumerate(g.get("volume", [])):
            res[f"{name}/grad_volume{i}"] = t.cpu().numpy()
        for k in ("tf", "eye"):
            if k in g:
                res[f"{name}/grad_{k}"] = g[k].cpu().numpy()
        if sc.model != _abi.DVR_COLOR_VOLUME:
            ti, tg = dvr.forward_tangent(None, None, None, None, eye, step, scene=sc)
            torch.cuda.synchronize()
            res[f"{name}/tangent_image"] = ti.cpu().numpy()
            res[f"{name}/tangent"] = tg.cpu().numpy()
        for b in (1, 4) if sc.model != _abi.DVR_COLOR_VOLUME else ():
            c = dvr.make_cells(sc.volumes[0], brick=b)
            torch.cuda.synchronize()
            res[f"{name}/cells{b}"] = c.view(torch.int16 if c.element_size() == 2 else torch.int32).cpu().numpy()
    return res


def status(reset=False):
    out = (ctypes.c_int64 * 4)()
    rc = _abi.load().dvr_bounds_status(out, 1 if reset else 0)
    return [rc] + list(out)


def _code(fn):
    """(return code, message) of a binding call: 0 or the DVRError's."""
    try:
        fn()
        torch.cuda.synchronize()
        return 0, ""
    except _abi.DVRError as e:
        msg = str(e)
        return int(msg.split("failed with code ")[1].split(":")[0]), msg


def caps() -> dict:
    """Per site: lower its extent, make the call that indexes it, record the
    call's code and message and the records afterwards; restore the extent
    and check that the same call passes again."""
    lib = _abi.load()
    sc_list = {s[0]: s for s in scenes()}
    name, sc, eye, step, want, _ = sc_list["ea_f32"]
    _, sb, eyeb, stepb, wantb, _ = sc_list["ea_f16_bricks_cellgrad"]
    img, aux = dvr.forward(None, None, None, None, eye, step, scene=sc)
    imgb, auxb = dvr.forward(None, None, None, None, eyeb, stepb, scene=sb)
    Gb = _grad_image(sb.pixels, sb.channels, 9)
    nvox = int(sc.volumes[0].numel())
    plan = [
        (_abi.DVR_SITE_VOLUME, nvox // 2, lambda: dvr.forward(None, None, None, None, eye, step, scene=sc)),
        (_abi.DVR_SITE_CELLS, 64, lambda: dvr.forward(None, None, None, None, eyeb, stepb, scene=sb)),
        (_abi.DVR_SITE_PIXEL, 100, lambda: dvr.forward(None, None, None, None, eye, step, scene=sc)),
        (_abi.DVR_SITE_TF, 1, lambda: dvr.forward(None, None, None, None, eye, step, scene=sc)),
        (_abi.DVR_SITE_CELL_GRADIENT, 64,
         lambda: dvr.backward(None, None, None, None, eyeb, stepb, auxb, Gb, scene=sb, want=wantb,
                              cell_gradient=True)),
    ]
    out = {}
    for site, cap, call in plan:
        _abi.check(lib.dvr_bounds_cap(site, cap), "dvr_bounds_cap")
        code, msg = _code(call)
        after = status()
        _abi.check(lib.dvr_bounds_cap(site, 0), "dvr_bounds_cap")
        again, _ = _code(call)
        out[str(site)] = {"code": code, "message": msg, "status_after": after, "again": again,
                          "status_end": status()}
    # a graph capture: the entry points skip their check, dvr_bounds_status
    # reads the records after the replay
    im2 = torch.empty_like(img)
    ax2 = torch.empty_like(aux)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            dvr.forward(None, None, None, None, eye, step, scene=sc, image=im2, aux=ax2, stream=s)
    g.replay()
    torch.cuda.synchronize()
    out["graph"] = {"equal": bool(torch.equal(im2, img) and torch.equal(ax2, aux)), "status": status()}
    _abi.check(lib.dvr_bounds_cap(_abi.DVR_SITE_PIXEL, 100), "dvr_bounds_cap")
    g.replay()
    out["graph_capped"] = {"status": status(reset=True), "status_reset": status()}
    _abi.check(lib.dvr_bounds_cap(_abi.DVR_SITE_PIXEL, 0), "dvr_bounds_cap")
    return out


def main(path):
    lib = _abi.load()
    assert lib.dvr_bounds_checked() == 1, f"{_abi.LIB_PATH} is not the bounds-checked build"
    res = cases()
    res["status_after_cases"] = np.array(status(), dtype=np.int64)
    res["caps"] = np.array(json.dumps(caps()))
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
