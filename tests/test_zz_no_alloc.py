"""dvr_backward_noalloc: the adjoint for callers that cannot allocate device
memory (a plugin whose host application owns the whole device-memory
budget, or a loop that must not call cudaMalloc because it can synchronise
the device). It keeps its tile-queue counters in a fixed array inside the
library instead of a caller workspace.

The GPU test calls it through the C ABI twice in a row (the second call
finds the counters the first one left behind) and checks each result
against dvr_backward with a workspace, within the gradient tolerance of the
other GPU tests. The oversize check needs no GPU: a call with more views
than the fixed array serves is refused before anything is launched.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2107_12672_b300 import _abi
from paper_2107_12672_b300 import synthetic as syn

GRAD_RTOL = 1e-3      # the gradient tolerance of the GPU parity tests


def _args(sc, eye, step, aux, seed, grads):
    gv = None
    if "volume" in grads:
        gv = (ctypes.c_void_p * len(sc.volumes))(*[t.data_ptr() for t in grads["volume"]])

    def p(k):
        return grads[k].data_ptr() if k in grads else None

    return (sc.vol_desc, len(sc.volumes), sc.tf_ref(), sc.model, sc.view_desc, len(sc.views),
            eye.data_ptr(), float(step), aux.data_ptr(), seed.data_ptr(), gv, p("tf"), p("eye"), p("step"), 0)


def _zero_grads(sc, want):
    dev = sc.volumes[0].device
    g = {}
    if "volume" in want:
        g["volume"] = [torch.zeros(v.shape, device=dev) for v in sc.volumes]
    if "tf" in want:
        g["tf"] = torch.zeros((sc.tf.shape[0], 4), device=dev)
    if "eye" in want:
        g["eye"] = torch.zeros((len(sc.views), 3), device=dev)
    if "step" in want:
        g["step"] = torch.zeros(1, device=dev)
    return g


def _close(got, ref, what):
    got = got.double().cpu()
    ref = ref.double().cpu()
    scale = float(ref.abs().max())
    err = float(((got - ref).abs() / (ref.abs() + scale)).max()) if scale > 0 else float(got.abs().max())
    assert err <= GRAD_RTOL, f"{what}: relative difference {err:.3e}"


@pytest.mark.gpu
@pytest.mark.parametrize("want", [("tf", "eye", "step"), ("volume", "tf", "eye")])
def test_noalloc_matches_workspace_entry_point_twice(want):
    from paper_2107_12672_b300.binding import Scene, forward
    lib = _abi.load()
    vol = torch.as_tensor(syn.value_noise(40, seed=11)).cuda()
    tf = torch.as_tensor(syn.random_tf(16, seed=12)).cuda()
    views = [syn.View(45, 37), syn.View(30, 52)]
    eye = torch.as_tensor(2.5 * syn.fibonacci_sphere(5)[[1, 3]], dtype=torch.float32).cuda().contiguous()
    step = 0.5
    sc = Scene.make([vol], tf, "emission_absorption", views)
    image, aux = forward(None, None, None, None, eye, step, scene=sc)
    rng = np.random.default_rng(13)
    seed = torch.as_tensor(rng.normal(size=tuple(image.shape)), dtype=torch.float32).cuda().contiguous()
    ws = torch.empty(int(lib.dvr_backward_workspace_bytes(len(views))), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        ref = _zero_grads(sc, want)
        got = _zero_grads(sc, want)
        _abi.check(lib.dvr_backward(*_args(sc, eye, step, aux, seed, ref), None, 0, ws.data_ptr(), ws.numel(),
                                    stream), "dvr_backward")
        _abi.check(lib.dvr_backward_noalloc(*_args(sc, eye, step, aux, seed, got), stream),
                   "dvr_backward_noalloc")
        torch.cuda.synchronize()
        for k in want:
            r = ref[k][0] if k == "volume" else ref[k]
            g = got[k][0] if k == "volume" else got[k]
            assert float(r.abs().max()) > 0, f"call {call}: {k} gradient is all zero"
            _close(g, r, f"call {call}: {k}")


def test_noalloc_refuses_more_views_than_its_scratch_serves():
    lib = _abi.load()
    n = 1025           # three launches of up to 512 views: three counters, the array holds two
    vol = _abi.DvrVolume(8, 8, 8, _abi.DVR_F32, 4096)
    views = (_abi.DvrView * n)(*[_abi.DvrView(4, 4, 0, 0, 0.4, 0, 16 * i) for i in range(n)])
    rc = lib.dvr_backward_noalloc(ctypes.byref(vol), 1, None, _abi.DVR_ABSORPTION, views, n, 4096, 0.5,
                                  4096, 4096, None, None, 4096, None, 0, None)
    assert rc == -1
    msg = lib.dvr_last_error().decode()
    assert "at most 1024 views" in msg and "dvr_backward_noalloc" in msg
