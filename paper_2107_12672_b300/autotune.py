"""Autotuner for the ray tiling of the march kernels.

A warp marches a tile of `width x (32 / width)` pixels; which shape touches
the fewest cache sectors per gather depends on the view direction and the
volume layout, so the tuner times forward + adjoint passes of the caller's
own workload for each candidate width and keeps the fastest (the choice
never changes results: every ray is computed the same way). Choices are
cached per device and workload signature for the life of the process, and
optionally in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from . import _abi
from .binding import Scene, backward, forward

CANDIDATES = (4, 8, 16, 32)
_cache: dict = {}


def signature(scene: Scene, want) -> str:
    vols = ";".join(f"{tuple(v.shape)}:{v.dtype}" for v in scene.volumes)
    views = ";".join(f"{w.width}x{w.height}:{int(bool(w.ortho))}" for w in scene.views)
    tf = "" if scene.tf is None else f"{tuple(scene.tf.shape)}:{scene.tf.dtype}"
    dev = torch.cuda.get_device_name(scene.volumes[0].device)
    return f"{dev}|m{scene.model}|{vols}|{tf}|{views}|{','.join(sorted(want))}"


def set_tile_width(width: int) -> None:
    _abi.check(_abi.load().dvr_set_tile_width(int(width)), "dvr_set_tile_width")


def get_tile_width() -> int:
    return int(_abi.load().dvr_get_tile_width())


def autotune(scene: Scene, eye, step_voxels, *, want=("tf", "eye"), reps: int = 5,
             candidates=CANDIDATES, cache_file: str | None = None) -> dict:
    """Time forward + adjoint for each tile width, set the fastest, and
    return {"width": best, "ms": {width: ms}}. Cached per signature."""
    key = signature(scene, want)
    if key not in _cache and cache_file and os.path.exists(cache_file):
        try:
            _cache.update(json.load(open(cache_file)))
        except (OSError, ValueError):
            pass
    if key in _cache:
        set_tile_width(_cache[key]["width"])
        return _cache[key]
    dev = scene.volumes[0].device
    image = torch.empty((scene.pixels, scene.channels), device=dev)
    aux = torch.empty((scene.pixels, 2), device=dev)
    seed = torch.full_like(image, 1e-3)
    grads = {}
    if "volume" in want:
        grads["volume"] = [torch.zeros(v.shape, device=dev) for v in scene.volumes]
    if "tf" in want and scene.tf is not None:
        grads["tf"] = torch.zeros((scene.tf.shape[0], 4), device=dev)
    if "eye" in want:
        grads["eye"] = torch.zeros((len(scene.views), 3), device=dev)
    w_want = tuple(grads.keys())
    times = {}
    for width in candidates:
        set_tile_width(width)

        def once():
            forward(None, None, None, None, eye, step_voxels, scene=scene, image=image, aux=aux)
            backward(None, None, None, None, eye, step_voxels, aux, seed, scene=scene, grads=grads, want=w_want)

        once()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record()
        for _ in range(reps):
            once()
        end.record()
        torch.cuda.synchronize()
        times[width] = start.elapsed_time(end) / reps
    best = min(times, key=times.get)
    set_tile_width(best)
    result = {"width": best, "ms": {str(k): round(v, 4) for k, v in times.items()}}
    _cache[key] = result
    if cache_file:
        try:
            with open(cache_file, "w") as f:
                json.dump(_cache, f, indent=1)
        except OSError:
            pass
    return result
