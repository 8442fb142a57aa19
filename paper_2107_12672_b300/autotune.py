"""Autotuner for the march kernels: ray tiling, gather layout and scatter.

A warp marches a tile of `width x (32 / width)` pixels; which shape touches
the fewest cache sectors per gather depends on the view direction, the
volume layout and the pass, so the tuner times the forward and the adjoint
passes of the caller's own workload for each candidate width and keeps the
fastest width for each pass. It also decides where the gathers read from
(the volume's array, or its cell layout: 8 corners per cell, 8x the bytes,
one or two 16-byte loads per cell, records in row order or in bricks of
4^3 cells; the layout is remade before each timed forward, as a step that
changes the volume must) and, when a volume
gradient is asked for, how it is accumulated (into the vertex array, or
per cell first: DVR_FLAG_CELL_GRADIENT) and whether that adjoint runs as a
persistent launch taking tiles from a queue (DVR_FLAG_PERSISTENT_SCATTER,
timed at the chosen layout and widths). None of the choices changes
results beyond the order of the gradient's additions. Choices are cached per
device and workload signature for the life of the process, and optionally
in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from . import _abi
from .binding import Scene, backward, cell_workspace_bytes, forward, make_cells

CANDIDATES = (4, 8, 16, 32)
_cache: dict = {}


def signature(scene: Scene, want) -> str:
    vols = ";".join(f"{tuple(v.shape)}:{v.dtype}" for v in scene.volumes)
    views = ";".join(f"{w.width}x{w.height}:{int(bool(w.ortho))}" for w in scene.views)
    tf = "" if scene.tf is None else f"{tuple(scene.tf.shape)}:{scene.tf.dtype}"
    dev = torch.cuda.get_device_name(scene.volumes[0].device)
    return f"{dev}|m{scene.model}|{vols}|{tf}|{views}|{','.join(sorted(want))}"


def set_tile_width(width: int, adjoint: int | None = None) -> None:
    """Set the forward tile width, and the adjoint's (the same if None)."""
    lib = _abi.load()
    _abi.check(lib.dvr_set_pass_tile_width(_abi.DVR_PASS_FORWARD, int(width)), "dvr_set_pass_tile_width")
    _abi.check(lib.dvr_set_pass_tile_width(_abi.DVR_PASS_ADJOINT, int(width if adjoint is None else adjoint)),
               "dvr_set_pass_tile_width")


def get_tile_width(adjoint: bool = False) -> int:
    return int(_abi.load().dvr_get_pass_tile_width(_abi.DVR_PASS_ADJOINT if adjoint else _abi.DVR_PASS_FORWARD))


def autotune(scene: Scene, eye, step_voxels, *, want=("tf", "eye"), reps: int = 5,
             candidates=CANDIDATES, cache_file: str | None = None, l2_flush: torch.Tensor | None = None,
             layouts=(0,), cell_gradients=(False,), persistent=(False,)) -> dict:
    """Time the forward and the adjoint pass for each tile width (two
    interleaved rounds, the faster of the two kept) and each gather layout
    in `layouts` (0: the volume's array; 1 / 4 / 8: its cell layout with
    records in row order / in bricks of 4^3 / 8^3 cells, so the brick edge,
    built before each forward and timed with it) and, for the adjoint of a
    volume gradient, each scatter in `cell_gradients` and then, at the
    chosen layout, scatter and width, each launch form in `persistent`
    (False: one tile per warp; True: DVR_FLAG_PERSISTENT_SCATTER, kept
    unless the other is more than 1% faster; 16-bit volumes only). Sets the
    fastest width of each pass and returns {"width", "adjoint_width",
    "cells", "cell_gradient", "persistent_scatter", "ms": {...}}. The layout
    is chosen by forward + adjoint time at each side's best width. Cached
    per signature. With `l2_flush` (a device buffer larger than L2), the
    buffer is overwritten before each timed pass, so that the passes start
    with the volume out of L2 as in a loop that touches other data between
    steps."""
    gvol = "volume" in want
    cell_gradients = cell_gradients if gvol else (False,)
    # the launch form exists for the volume-gradient adjoint of 16-bit volumes
    sixteen = all(v.dtype in (torch.float16, torch.bfloat16) for v in scene.volumes)
    persistent = persistent if gvol and sixteen else (False,)
    key = signature(scene, want) + f"|cells{tuple(layouts)}|cg{tuple(cell_gradients)}|ps{tuple(persistent)}"
    if key not in _cache and cache_file and os.path.exists(cache_file):
        try:
            _cache.update(json.load(open(cache_file)))
        except (OSError, ValueError):
            pass
    if key in _cache:
        set_tile_width(_cache[key]["width"], _cache[key]["adjoint_width"])
        return _cache[key]
    dev = scene.volumes[0].device
    image = torch.empty((scene.pixels, scene.channels), device=dev)
    aux = torch.empty((scene.pixels, 2), device=dev)
    seed = torch.full_like(image, 1e-3)
    grads = {}
    if gvol:
        grads["volume"] = [torch.zeros(v.shape, device=dev) for v in scene.volumes]
    if "tf" in want and scene.tf is not None:
        grads["tf"] = torch.zeros((scene.tf.shape[0], 4), device=dev)
    if "eye" in want:
        grads["eye"] = torch.zeros((len(scene.views), 3), device=dev)
    w_want = tuple(grads.keys())

    def timed(fn):
        if l2_flush is None:
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            start.record()
            for _ in range(reps):
                fn()
            end.record()
            torch.cuda.synchronize()
            return start.elapsed_time(end) / reps
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            l2_flush.zero_()
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / reps

    times = {}
    for use_cells in layouts:
        cells = [make_cells(v, brick=use_cells) for v in scene.volumes] if use_cells else None
        sc = Scene.make(scene.volumes, scene.tf, scene.model, scene.views, cells=cells, cells_brick=use_cells or 1)
        # the cell-major gradients' size depends on the record order (bricks pad)
        cg_ws = torch.empty(cell_workspace_bytes(sc), dtype=torch.uint8, device=dev) if True in cell_gradients else None

        def fwd():
            if cells is not None:
                for v, c in zip(sc.volumes, cells):
                    make_cells(v, out=c, brick=use_cells)
            forward(None, None, None, None, eye, step_voxels, scene=sc, image=image, aux=aux)

        for cg in cell_gradients:
            def bwd():
                backward(None, None, None, None, eye, step_voxels, aux, seed, scene=sc, grads=grads, want=w_want,
                         cell_gradient=cg, workspace=cg_ws if cg else None)

            fk, bk = f"forward|cells={int(use_cells)}", f"adjoint|cells={int(use_cells)}|cell_gradient={int(cg)}"
            times.setdefault(fk, {})
            times.setdefault(bk, {})
            for _ in range(2):
                for width in candidates:
                    set_tile_width(width)
                    fwd()
                    bwd()
                    torch.cuda.synchronize()
                    for name, fn in ((fk, fwd), (bk, bwd)):
                        if name == fk and cg != cell_gradients[0]:
                            continue            # the forward does not depend on the scatter
                        t = timed(fn)
                        times[name][width] = min(t, times[name].get(width, t))
        del cells, sc, cg_ws
    best = None
    for use_cells in layouts:
        f = times[f"forward|cells={int(use_cells)}"]
        bf = min(f, key=f.get)
        for cg in cell_gradients:
            b = times[f"adjoint|cells={int(use_cells)}|cell_gradient={int(cg)}"]
            bb = min(b, key=b.get)
            total = f[bf] + b[bb]
            if best is None or total < best[0]:
                best = (total, bf, bb, use_cells, cg)
    _, best_f, best_b, use_cells, cg = best
    set_tile_width(best_f, best_b)
    ps = persistent[0]
    if len(persistent) > 1:
        # the launch form of the volume-gradient adjoint, at the chosen layout,
        # scatter and width (two interleaved rounds, the faster kept)
        cells = [make_cells(v, brick=use_cells) for v in scene.volumes] if use_cells else None
        sc = Scene.make(scene.volumes, scene.tf, scene.model, scene.views, cells=cells, cells_brick=use_cells or 1)
        cg_ws = torch.empty(cell_workspace_bytes(sc), dtype=torch.uint8, device=dev) if cg else None
        forward(None, None, None, None, eye, step_voxels, scene=sc, image=image, aux=aux)
        pk = f"adjoint|cells={int(use_cells)}|cell_gradient={int(cg)}|width={best_b}|persistent"
        times[pk] = {}
        for _ in range(2):
            for p in persistent:
                def bwd():
                    backward(None, None, None, None, eye, step_voxels, aux, seed, scene=sc, grads=grads,
                             want=w_want, cell_gradient=cg, workspace=cg_ws if cg else None,
                             persistent_scatter=p)
                bwd()
                torch.cuda.synchronize()
                t = timed(bwd)
                times[pk][int(p)] = min(t, times[pk].get(int(p), t))
        # the persistent form unless the one-tile form is more than 1% faster:
        # its gain grows with the launch (1024^3 FP16: equal on 4 views of
        # 2048^2, 3.4% faster on all 32), and a caller may tune on a few views
        tp = times[pk]
        ps = 1 in tp and (0 not in tp or tp[1] <= 1.01 * tp[0])
        del cells, sc, cg_ws
    result = {"width": best_f, "adjoint_width": best_b, "cells": int(use_cells), "cell_gradient": bool(cg),
              "persistent_scatter": ps,
              "ms": {n: {str(k): round(v, 4) for k, v in t.items()} for n, t in times.items()}}
    _cache[key] = result
    if cache_file:
        try:
            with open(cache_file, "w") as f:
                json.dump(_cache, f, indent=1)
        except OSError:
            pass
    return result
