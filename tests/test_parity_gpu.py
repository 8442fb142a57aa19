"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Inputs come from the seeded generators only; the adjoint seeds dL/d(image)
are seeded random arrays given to both sides. Tolerances (per element,
relative to the element or to the array's scale): images 1e-5, gradients
1e-3. Sample counts are integers decided by the same binary32 ray setup on
both sides and must match exactly.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2107_12672_b300 as dvr
from paper_2107_12672_b300 import synthetic as syn
from tests.gpu_helpers import (FP32_MARGIN, GRAD_RTOL, IMAGE_RTOL, as_oracle_volume, assert_close,
                               pixel_offsets, seeded_grad_image, to_dev)

pytestmark = pytest.mark.gpu


def _run_gpu(w, vol_dtype=torch.float32, tf_dtype=torch.float32, grad_seed=5, want=("volume", "tf", "eye"),
             tf_immediate=False, persistent_scatter=False):
    vols = [to_dev(v, vol_dtype) for v in w.volumes]
    tf = to_dev(w.tf, tf_dtype) if w.tf is not None else None
    eye = to_dev(w.eye)
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    img, aux = dvr.forward(vols, tf, w.model, w.views, eye, w.step_voxels, sample_count=count)
    nc = img.shape[1]
    G = seeded_grad_image(img.shape[0], nc, grad_seed)
    g = dvr.backward(vols, tf, w.model, w.views, eye, w.step_voxels, aux, to_dev(G), want=want,
                     tf_immediate=tf_immediate, persistent_scatter=persistent_scatter)
    torch.cuda.synchronize()
    return vols, tf, img.cpu().numpy(), int(count.item()), G, g


def _oracle(w, vols, tf, G, want=("volume", "tf", "eye")):
    vols64 = [as_oracle_volume(v) for v in vols]
    tf64 = as_oracle_volume(tf) if tf is not None else None
    offs, P = pixel_offsets(w.views)
    nc = 1 if w.model == "absorption" else 4
    img = np.zeros((P, nc))
    Ntot = 0
    gv = [np.zeros(v.shape) for v in vols64]
    amb = [np.zeros(v.shape) for v in vols64]
    gt = np.zeros_like(tf64) if tf64 is not None else None
    ge = np.zeros((len(w.views), 3))
    amb_e = np.zeros((len(w.views), 3))
    for k, view in enumerate(w.views):
        n = view.width * view.height
        vol = vols64[view.volume_index]
        im, N, _ = oracle.render(vol, tf64, w.model, view, w.eye[k], w.step_voxels)
        img[offs[k]:offs[k] + n] = im
        Ntot += int(N.sum())
        ow = tuple(x for x in want if x != "step")
        g = oracle.backward(vol, tf64, w.model, view, w.eye[k], w.step_voxels, G[offs[k]:offs[k] + n], want=ow,
                            margin=FP32_MARGIN)
        if "volume" in g:
            gv[view.volume_index] += g["volume"]
            if "volume_ambiguity" in g:
                amb[view.volume_index] += g["volume_ambiguity"]
        if "tf" in g and gt is not None:
            gt += g["tf"]
        if "eye" in g:
            ge[k] = g["eye"]
            amb_e[k] = g["eye_ambiguity"]
    return img, Ntot, {"volume": gv, "tf": gt, "eye": ge, "amb": amb, "amb_eye": amb_e}


def _compare(w, gpu, ref, want, image_rtol=IMAGE_RTOL, grad_rtol=GRAD_RTOL):
    vols, tf, img, count, G, g = gpu
    rimg, rN, rg = ref
    assert count == rN, "sample counts differ: the ray setup is not bit-identical"
    errs = {"image": assert_close(img, rimg, image_rtol, "image")}
    if "volume" in want:
        for i, (a, b) in enumerate(zip(g["volume"], rg["volume"])):
            errs[f"volume{i}"] = assert_close(a.cpu().numpy(), b, grad_rtol, f"grad volume {i}",
                                              slack=rg["amb"][i])
    if "tf" in want and tf is not None:
        errs["tf"] = assert_close(g["tf"].cpu().numpy(), rg["tf"], grad_rtol, "grad tf")
    if "eye" in want:
        errs["eye"] = assert_close(g["eye"].cpu().numpy(), rg["eye"], grad_rtol, "grad eye",
                                   slack=rg["amb_eye"])
    return errs


# ------------------------------------------------------------------ workloads
def test_absorption_64_full_size():
    """64^3 Gaussian blobs, ortho +z, 64x64, step 0.5: image and the
    gradient w.r.t. all 262144 densities at full size."""
    w = syn.workload("absorption_64")
    want = ("volume", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


@pytest.mark.parametrize("scale,size", [(0.25, None), (0.25, (131, 97)), (0.125, (8, 4)), (0.125, (1, 1))])
def test_ea_reduced(scale, size):
    """Emission-absorption value noise with a 16-row TF and a perspective
    camera, at sizes spanning several tiles and ragged tails."""
    w = syn.workload("ea_256", scale=scale)
    if size is not None:
        w.views = [syn.View(size[0], size[1])]
    want = ("volume", "tf", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


def test_ea_256_full_size():
    """The 256^3 / 512^2 emission-absorption workload at full size: every
    pixel, and the TF and eye gradients (global sums over all rays)."""
    w = syn.workload("ea_256")
    want = ("tf", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


def test_multiview_uneven_one_launch():
    """64 Fibonacci views of uneven sizes and two volumes in one launch."""
    w = syn.workload("tomo_256x64", scale=1 / 16)
    w.volumes.append(syn.gaussian_blobs(w.volumes[0].shape[0], 4, seed=44))
    for k, v in enumerate(w.views):
        v.volume_index = k % 2
    want = ("volume", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


@pytest.mark.parametrize("case", ["multiview", "ea_ragged_fp16"])
def test_persistent_scatter_against_oracle(case):
    """The volume-gradient adjoint as a persistent launch
    (DVR_FLAG_PERSISTENT_SCATTER: as many blocks as are resident, each warp
    taking ray tiles from the launch's queue) against the oracle, element
    by element: 64 uneven views of two absorption volumes in one launch
    (volume and eye gradients), and one ragged 131 x 97 emission-absorption
    view of an FP16 volume (volume, TF and eye gradients)."""
    if case == "multiview":
        w = syn.workload("tomo_256x64", scale=1 / 16)
        w.volumes.append(syn.gaussian_blobs(w.volumes[0].shape[0], 4, seed=45))
        for k, v in enumerate(w.views):
            v.volume_index = k % 2
        want, vdt = ("volume", "eye"), torch.float32
    else:
        w = syn.workload("ea_256", scale=0.25)
        w.views = [syn.View(131, 97)]
        want, vdt = ("volume", "tf", "eye"), torch.float16
    gpu = _run_gpu(w, vol_dtype=vdt, want=want, persistent_scatter=True)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


def test_persistent_forward_over_several_launches():
    """More views than one launch takes (600 > 512: two launches, each with
    its own tile-queue counter in the workspace): the persistent forward
    writes every pixel of a NaN-filled image with the bits of the launch
    with one tile per warp, and counts the same samples; with the cell
    layout in 4^3 bricks as well."""
    import ctypes
    from paper_2107_12672_b300 import _abi
    w = syn.workload("ea_256", scale=0.0625)
    vol, tf = to_dev(w.volumes[0], torch.float16), to_dev(w.tf)
    sizes = [(1 + k % 9, 1 + (k * 7) % 11) for k in range(600)]
    views = [syn.View(a, b) for a, b in sizes]
    eye = to_dev(2.3 * syn.fibonacci_sphere(len(views)))
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    for cells in (None, [dvr.make_cells(vol, brick=4)]):
        sc = dvr.Scene.make([vol], tf, w.model, views, cells=cells, cells_brick=4)
        out = []
        for ws in (None, sc.workspace(lib)):
            img = torch.full((sc.pixels, 4), float("nan"), device="cuda")
            aux = torch.full((sc.pixels, 2), float("nan"), device="cuda")
            count = torch.zeros(1, dtype=torch.int64, device="cuda")
            rc = lib.dvr_forward(sc.vol_desc, 1, sc.tf_ref(), sc.model, sc.view_desc, len(views), eye.data_ptr(),
                                 ctypes.c_float(w.step_voxels), img.data_ptr(), aux.data_ptr(), count.data_ptr(),
                                 None, 0, None if ws is None else ws.data_ptr(), 0 if ws is None else ws.numel(),
                                 stream)
            _abi.check(rc, "dvr_forward")
            torch.cuda.synchronize()
            out.append((img, aux, int(count.item())))
        assert not torch.isnan(out[1][0]).any() and not torch.isnan(out[1][1]).any()
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
        assert out[0][2] == out[1][2] > 0


def test_persistent_scatter_over_several_launches():
    """More views than one launch takes (600 > 512: two adjoint launches,
    each with its own tile-queue counter in the workspace): the persistent
    volume-gradient adjoint of an FP16 volume gives the volume, TF and eye
    gradients of the launch with one tile per warp, for every view, from the
    volume's array and from its cell layout with the per-cell gradient."""
    w = syn.workload("ea_256", scale=0.0625)
    vol, tf = to_dev(w.volumes[0], torch.float16), to_dev(w.tf)
    views = [syn.View(1 + k % 9, 1 + (k * 7) % 11) for k in range(600)]
    eye = to_dev(2.3 * syn.fibonacci_sphere(len(views)))
    want = ("volume", "tf", "eye")
    for cells, cg in ((None, False), ([dvr.make_cells(vol, brick=4)], True)):
        sc = dvr.Scene.make([vol], tf, w.model, views, cells=cells, cells_brick=4)
        _, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
        G = to_dev(seeded_grad_image(sc.pixels, 4, 12))
        a = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=want, cell_gradient=cg)
        b = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=want, cell_gradient=cg,
                         persistent_scatter=True)
        torch.cuda.synchronize()
        lit = a["eye"].abs().sum(dim=1) > 0                     # views whose rays change the loss
        assert float(lit[:512].float().mean()) > 0.9 and float(lit[512:].float().mean()) > 0.9
        assert_close(b["volume"][0].cpu().numpy(), a["volume"][0].cpu().numpy(), 1e-4, "volume")
        for k in ("tf", "eye"):
            assert_close(b[k].cpu().numpy(), a[k].cpu().numpy(), 1e-4, k)


@pytest.mark.parametrize("vdt,tdt", [(torch.bfloat16, torch.float16), (torch.float16, torch.float32)])
def test_reduced_precision_storage(vdt, tdt):
    """BF16/FP16 volume and FP16 TF storage with FP32 arithmetic: the oracle
    takes the same rounded values, so FP32 tolerances hold."""
    w = syn.workload("ea_bf16_512", scale=1 / 8)
    w.views = w.views[:3]
    w.eye = w.eye[:3]
    want = ("volume", "tf", "eye")
    gpu = _run_gpu(w, vol_dtype=vdt, tf_dtype=tdt, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("eye,ortho", [
    ((0.0, 2.4, 0.0), False),          # looking straight down -y: fixed right vector
    ((0.12, -0.08, 0.2), False),       # camera inside the volume
    ((0.0, 0.0, 3.0), True),           # axis-aligned ortho: N exactly integral
    ((5.0, 0.0, 0.0), False),          # far camera, grazing rays at the box faces
    ((0.0, 0.0, -0.9), True),          # ortho from -z
])
def test_camera_edge_cases(eye, ortho):
    w = syn.workload("ea_256", scale=0.0625)
    w.views = [syn.View(37, 29, ortho=ortho, ortho_height=1.2)]
    w.eye = np.array([eye], dtype=np.float32)
    want = ("volume", "tf", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


def test_rays_that_miss_the_volume():
    """An orthographic image plane four times wider than the box: most rays
    miss (N = 0, zero pixel, no gradient), the rest match the oracle."""
    w = syn.workload("ea_256", scale=0.0625)
    w.views = [syn.View(24, 20, ortho=True, ortho_height=4.0)]
    w.eye = np.array([[0.3, 0.2, 2.5]], dtype=np.float32)
    want = ("volume", "tf", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)
    img = gpu[2]
    assert (np.abs(img).sum(1) == 0).mean() > 0.5


def test_tf_immediate_equals_delayed():
    """The adjoint-immediate and adjoint-delayed TF accumulations (Sec. 5.2)
    give the same gradient."""
    w = syn.workload("ea_256", scale=0.125)
    a = _run_gpu(w, want=("tf",))
    b = _run_gpu(w, want=("tf",), tf_immediate=True)
    # binary32 sums of ~10^5 contributions per entry, added in different
    # orders: equal to 1e-4 per element (both are checked against the oracle
    # at the gradient bar elsewhere)
    assert_close(b[5]["tf"].cpu().numpy(), a[5]["tf"].cpu().numpy(), 1e-4, "immediate vs delayed")


def test_step_gradient():
    """dL/d(step_voxels) against central differences of the oracle (N fixed)."""
    w = syn.workload("ea_256", scale=0.125)
    step = 0.53
    w.step_voxels = step
    vols = [to_dev(w.volumes[0])]
    tf = to_dev(w.tf)
    eye = to_dev(w.eye)
    img, aux = dvr.forward(vols, tf, w.model, w.views, eye, step)
    G = seeded_grad_image(img.shape[0], 4, 9)
    g = dvr.backward(vols, tf, w.model, w.views, eye, step, aux, to_dev(G), want=("step",))
    gs = float(g["step"].item())
    ref = oracle.backward(as_oracle_volume(vols[0]), as_oracle_volume(tf), w.model, w.views[0], w.eye[0],
                          step, G, want=("step",))["step"]
    assert abs(gs - ref) <= GRAD_RTOL * abs(ref)


def test_orbit_camera_kernels():
    rng = np.random.default_rng(0)
    prm = np.stack([rng.uniform(-3, 3, 50), rng.uniform(-1.4, 1.4, 50), rng.uniform(1, 4, 50)], 1)
    prm = prm.astype(np.float32)
    eye = dvr.orbit_eye(to_dev(prm)).cpu().numpy()
    np.testing.assert_allclose(eye, oracle.orbit_eye(prm), rtol=2e-6, atol=2e-6)
    ge = rng.normal(size=(50, 3)).astype(np.float32)
    gp = dvr.orbit_eye_backward(to_dev(prm), to_dev(ge)).cpu().numpy()
    np.testing.assert_allclose(gp, oracle.orbit_eye_backward(prm, ge), rtol=1e-5, atol=2e-5)


def test_loss_l2_kernel():
    rng = np.random.default_rng(1)
    for n in (1, 7, 4096, 100003):
        x = rng.normal(size=n).astype(np.float32)
        y = rng.normal(size=n).astype(np.float32)
        loss = torch.zeros(1, device="cuda")
        g = dvr.loss_l2(to_dev(x), to_dev(y), 0.25, loss=loss).cpu().numpy()
        np.testing.assert_allclose(g, 0.5 * (x.astype(np.float64) - y), rtol=1e-6, atol=1e-7)
        ref = 0.25 * ((x.astype(np.float64) - y) ** 2).sum()
        assert abs(loss.item() - ref) <= 1e-5 * ref


def test_autograd_render_matches_raw_backward():
    """render() as a torch.autograd.Function: gradients equal dvr.backward."""
    w = syn.workload("ea_256", scale=0.125)
    vol = to_dev(w.volumes[0]).requires_grad_(True)
    tf = to_dev(w.tf).requires_grad_(True)
    eye = to_dev(w.eye).requires_grad_(True)
    img = dvr.render(vol, tf, eye, w.views, w.step_voxels, w.model)
    G = to_dev(seeded_grad_image(img.shape[0], 4, 3))
    (img * G).sum().backward()
    _, aux = dvr.forward([vol.detach()], tf.detach(), w.model, w.views, eye.detach(), w.step_voxels)
    g = dvr.backward([vol.detach()], tf.detach(), w.model, w.views, eye.detach(), w.step_voxels, aux, G)
    for a, b in ((vol.grad, g["volume"][0]), (tf.grad, g["tf"]), (eye.grad, g["eye"])):
        assert_close(a.cpu().numpy(), b.cpu().numpy(), 1e-5, "autograd")


def test_autograd_render_with_cell_layout_and_persistent_scatter():
    """render() with the fast options of the 16-bit workloads (an FP16
    volume gathered from its 4^3-brick cell layout, the volume gradient per
    cell, the persistent scatter): the image of the plain call bit for bit,
    and the gradients of the raw dvr.backward on the volume's array (the
    volume gradient rounded to the volume's FP16 by autograd)."""
    w = syn.workload("ea_256", scale=0.125)
    vol = to_dev(w.volumes[0], torch.float16).requires_grad_(True)
    tf = to_dev(w.tf).requires_grad_(True)
    eye = to_dev(w.eye).requires_grad_(True)
    img = dvr.render(vol, tf, eye, w.views, w.step_voxels, w.model, cells=4, cell_gradient=True,
                     persistent_scatter=True)
    G = to_dev(seeded_grad_image(img.shape[0], 4, 7))
    (img * G).sum().backward()
    v0 = vol.detach()
    ref_img, aux = dvr.forward([v0], tf.detach(), w.model, w.views, eye.detach(), w.step_voxels)
    assert torch.equal(img.detach(), ref_img)
    g = dvr.backward([v0], tf.detach(), w.model, w.views, eye.detach(), w.step_voxels, aux, G)
    assert vol.grad.dtype == torch.float16
    assert_close(vol.grad.float().cpu().numpy(), g["volume"][0].half().float().cpu().numpy(), 2e-3, "volume")
    for a, b in ((tf.grad, g["tf"]), (eye.grad, g["eye"])):
        assert_close(a.cpu().numpy(), b.cpu().numpy(), 1e-4, "autograd")


def test_orbit_chain_gradient():
    """Gradient w.r.t. (yaw, pitch, distance) through the orbit kernels and the
    renderer, against the oracle's chain of the same two maps. The eye is
    rounded differently on both sides, so a ray whose N sits on a rounding
    boundary may differ; the camera gradient sums all rays and stays within
    the gradient tolerance."""
    w = syn.workload("ea_256", scale=0.25)
    prm = to_dev(w.orbit.astype(np.float32)).requires_grad_(True)
    vol = to_dev(w.volumes[0])
    tf = to_dev(w.tf)
    eye = dvr.orbit_camera(prm)
    img = dvr.render(vol, tf, eye, w.views, w.step_voxels, w.model)
    G = seeded_grad_image(img.shape[0], 4, 21)
    (img * to_dev(G)).sum().backward()
    p64 = w.orbit.astype(np.float32).astype(np.float64)
    e64 = oracle.orbit_eye(p64)[0]
    ge = oracle.backward(as_oracle_volume(vol), as_oracle_volume(tf), w.model, w.views[0], e64,
                         w.step_voxels, G, fp32=False, want=("eye",))["eye"]
    ref = oracle.orbit_eye_backward(p64, ge[None])[0]
    assert_close(prm.grad.cpu().numpy()[0], ref, GRAD_RTOL, "orbit chain")


def test_memory_constant_in_step_count():
    """The adjoint keeps no per-step state: peak device memory of a
    forward+backward is the same at step 0.5, 0.25 and 0.125 voxel."""
    w = syn.workload("ea_256", scale=0.25)
    vols = [to_dev(w.volumes[0])]
    tf = to_dev(w.tf)
    eye = to_dev(w.eye)
    peaks = []
    for step in (0.5, 0.25, 0.125):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        img, aux = dvr.forward(vols, tf, w.model, w.views, eye, step)
        G = torch.ones_like(img)
        dvr.backward(vols, tf, w.model, w.views, eye, step, aux, G, want=("volume", "tf", "eye"))
        torch.cuda.synchronize()
        peaks.append(torch.cuda.max_memory_allocated())
        del img, aux, G
    assert peaks[0] == peaks[1] == peaks[2]
    # device-wide (cudaMemGetInfo sees every allocation of the process, the
    # library's included): with the outputs allocated beforehand, forward +
    # adjoint change nothing at any step size
    scene = dvr.Scene.make(vols, tf, w.model, w.views)
    img = torch.empty((scene.pixels, 4), device="cuda")
    aux = torch.empty((scene.pixels, 2), device="cuda")
    G = torch.ones_like(img)
    grads = {"volume": [torch.zeros_like(vols[0])], "tf": torch.zeros_like(tf), "eye": torch.zeros_like(eye)}

    def run(step):
        dvr.forward(None, None, None, None, eye, step, scene=scene, image=img, aux=aux)
        dvr.backward(None, None, None, None, eye, step, aux, G, scene=scene, grads=grads,
                     want=("volume", "tf", "eye"))
        torch.cuda.synchronize()

    for step in (0.5, 0.25, 0.125):
        run(step)
    used = []
    for step in (0.5, 0.25, 0.125):
        free0, total = torch.cuda.mem_get_info()
        run(step)
        free1, _ = torch.cuda.mem_get_info()
        used.append((total - free0, total - free1))
    assert len({u for pair in used for u in pair}) == 1, used


# ------------------------------------------------------- pre-shaded colour volume
@pytest.mark.parametrize("vdt", [torch.float32, torch.float16, torch.bfloat16])
def test_color_volume_parity(vdt):
    """Colour volume (Sec. 5.4; r, g, b, tau per vertex): image, 4-channel
    volume gradient and eye gradient against the oracle."""
    n = 24
    cv = syn.color_volume(n, seed=31)
    w = syn.Workload("color", "color", [cv], None, [syn.View(45, 37)],
                     np.array([[0.9, -0.7, 1.9]], dtype=np.float32), None, 0.5, ("volume", "camera"))
    want = ("volume", "eye")
    gpu = _run_gpu(w, vol_dtype=vdt, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


def test_color_volume_equals_ea_for_affine_tf_gpu():
    """On the GPU too: a colour volume holding an affine TF of the densities
    renders as the EA model with that TF, and the TF-space gradients agree."""
    n = 20
    v = syn.value_noise(n, seed=8)
    tf = np.array([[0.1, 0.7, 0.3, 1.5], [0.9, 0.2, 0.6, 6.0]], dtype=np.float32)
    cv = (tf[0][None, None, None, :] * (1 - v[..., None]) + tf[1][None, None, None, :] * v[..., None]).astype(np.float32)
    views = [syn.View(33, 29)]
    eye = to_dev(np.array([[0.7, 0.8, 1.6]], dtype=np.float32))
    a, _ = dvr.forward([to_dev(v)], to_dev(tf), "emission_absorption", views, eye, 0.5)
    b, _ = dvr.forward([to_dev(cv)], None, "color", views, eye, 0.5)
    assert_close(b.cpu().numpy(), a.cpu().numpy(), 2e-6, "colour vs EA")


# ------------------------------------------------ forward-mode tangents (Sec. 4.2)
@pytest.mark.parametrize("model,ortho", [("emission_absorption", False), ("emission_absorption", True),
                                         ("absorption", False)])
def test_forward_tangent(model, ortho):
    """d(image)/d(eye) from the forward-mode kernel: contracted with a seed it
    equals the adjoint's eye gradient (Sec. 5.1: same gradients up to
    rounding) and the oracle's; per pixel it matches the oracle's dual
    numbers (N from the same binary32 decision)."""
    if model == "absorption":
        w = syn.workload("absorption_64", scale=0.5)
        w.views = [syn.View(41, 35, ortho=ortho, ortho_height=1.3)]
        w.eye = np.array([[0.9, 0.7, 1.8]], dtype=np.float32)
    else:
        w = syn.workload("ea_256", scale=0.125)
        w.views = [syn.View(41, 35, ortho=ortho, ortho_height=1.3)]
    vols = [to_dev(w.volumes[0])]
    tf = to_dev(w.tf) if w.tf is not None else None
    eye = to_dev(w.eye)
    sc = dvr.Scene.make(vols, tf, w.model, w.views)
    img_t, tan = dvr.forward_tangent(None, None, None, None, eye, w.step_voxels, scene=sc)
    img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
    assert torch.equal(img_t, img)
    G = to_dev(seeded_grad_image(img.shape[0], img.shape[1], 17))
    g_fwd = dvr.tangent_contract(sc, tan, G)
    g_adj = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=("eye",))["eye"]
    # two binary32 evaluations of the same derivative (tangents summed over
    # pixels vs adjoints summed along rays): 1e-4 per element, including a
    # small component of the eye gradient next to a large one
    assert_close(g_fwd.cpu().numpy(), g_adj.cpu().numpy(), 1e-4, "forward mode vs adjoint")
    vol64 = as_oracle_volume(vols[0])
    tf64 = as_oracle_volume(tf) if tf is not None else None
    ref = oracle.backward(vol64, tf64, w.model, w.views[0], w.eye[0], w.step_voxels, G.cpu().numpy(),
                          want=("eye",), margin=FP32_MARGIN)
    assert_close(g_fwd.cpu().numpy()[0], ref["eye"], GRAD_RTOL, "forward mode vs oracle",
                 slack=ref["eye_ambiguity"])
    _, dref = oracle.render_dual(vol64, tf64, w.model, w.views[0], w.eye[0], w.step_voxels, n_fp32=True)
    t = tan.cpu().numpy().astype(np.float64)
    scale = np.abs(dref).max()
    err = np.abs(t - dref) / (np.abs(dref) + scale)
    # single samples next to a TF control point or a cell face may take the
    # other one-sided derivative in binary32 (the dual-number oracle takes
    # the binary64 ray geometry, within ~1e-7 of the kernel's, so samples
    # near a kink can land on the other side): most pixels agree tightly
    assert np.quantile(err, 0.99) < 3e-4, np.quantile(err, 0.99)
    assert err.max() < 5e-2, err.max()


# ------------------------------------------------------ optimisation-side kernels
def test_priors_losses_and_resampling():
    """Smoothing priors (Eq. tf-loss, 3D form of Sec. 5.3), L1 loss and
    resampling kernels against their oracle definitions."""
    rng = np.random.default_rng(3)
    v = rng.normal(size=(37, 29, 41)).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    g = torch.zeros(v.shape, device="cuda")
    from paper_2107_12672_b300 import binding as b
    lib = b._abi.load()
    b._abi.check(lib.dvr_volume_prior(to_dev(v).data_ptr(), 41, 29, 37, 0.5, g.data_ptr(), loss.data_ptr(), None),
                 "prior")
    torch.cuda.synchronize()
    rl, rg = oracle.volume_prior(v)
    assert abs(loss.item() - 0.5 * rl) <= 1e-5 * abs(0.5 * rl)
    # per element, the prior's gradient 2 lambda sum (v_i - v_j) is a
    # difference of binary32 values: 1e-4 (1e-7 of the largest element)
    assert_close(g.cpu().numpy(), 0.5 * rg, 1e-4, "volume prior gradient")
    tf = rng.uniform(0, 1, (16, 4)).astype(np.float32)
    l2, g2 = dvr.tf_prior(to_dev(tf), 0.4)
    rl, rg = oracle.tf_prior(tf)
    assert abs(l2.item() - 0.4 / 60 * rl) <= 1e-5 * abs(0.4 / 60 * rl)
    assert_close(g2.cpu().numpy(), 0.4 / 60 * rg, 1e-5, "tf prior gradient")
    x = rng.normal(size=10001).astype(np.float32)
    y = rng.normal(size=10001).astype(np.float32)
    l1 = torch.zeros(1, device="cuda")
    g1 = dvr.loss_l1(to_dev(x), to_dev(y), 0.25, loss=l1).cpu().numpy()
    np.testing.assert_array_equal(g1, 0.25 * np.sign(x - y))
    assert abs(l1.item() - 0.25 * np.abs(x.astype(np.float64) - y).sum()) <= 1e-5 * l1.item()
    src = rng.uniform(0, 1, (17, 17, 17)).astype(np.float32)
    up = dvr.resample(to_dev(src), (33, 33, 33)).cpu().numpy()
    # binary32 trilinear values of unit scale: 1e-4 per element, i.e. 1e-7
    # absolute below the floor (about one rounding of the unit-scale values)
    assert_close(up, oracle.resample(src, (33, 33, 33)), 1e-4, "resample")


def test_multiresolution_reconstruction():
    """The schedule of Sec. 5.3 on the synthetic tomography workload: start at
    17^3, refine by resampling to 33^3 and 65^3, Adam on the densities with
    the L2 image loss plus the 3D smoothing prior; the loss at the finest
    level ends well below its start."""
    w = syn.workload("tomo_256x64", scale=0.25)       # 64^3 target, 64 views
    eye = to_dev(w.eye)
    target_vol = to_dev(syn.gaussian_blobs(65, 32, seed=4))
    with torch.no_grad():
        target = dvr.render(target_vol, None, eye, w.views, w.step_voxels, "absorption")
    x = torch.zeros((17, 17, 17), device="cuda")
    first = last = None
    for level, n in enumerate((17, 33, 65)):
        if n != x.shape[0]:
            x = dvr.resample(x.contiguous(), (n, n, n))
        x = x.detach().requires_grad_(True)
        opt = torch.optim.Adam([x], lr=0.05)
        for it in range(30):
            opt.zero_grad()
            img = dvr.render(x, None, eye, w.views, w.step_voxels * (n - 1) / 64, "absorption")
            loss = ((img - target) ** 2).mean() + dvr.volume_smoothness(x, 0.01)
            loss.backward()
            opt.step()
            if first is None:
                first = float(loss.detach())
        last = float(loss.detach())
    assert last < first / 5, (first, last)


# ------------------------------------------------------------ ray tiling
def test_tile_width_changes_nothing_and_autotuner_picks_one():
    """Every warp tile shape gives bit-identical images (each ray is computed
    the same way) and gradients equal up to the order of atomic additions;
    the autotuner selects one of the candidates and leaves it set."""
    from paper_2107_12672_b300 import autotune
    w = syn.workload("ea_256", scale=0.25)
    w.views = [syn.View(100, 77)]
    vols = [to_dev(w.volumes[0])]
    tf = to_dev(w.tf)
    eye = to_dev(w.eye)
    sc = dvr.Scene.make(vols, tf, w.model, w.views)
    G = to_dev(seeded_grad_image(100 * 77, 4, 4))
    ref = None
    old, old_adj = autotune.get_tile_width(), autotune.get_tile_width(adjoint=True)
    try:
        for width in (1, 2, 4, 8, 16, 32):
            autotune.set_tile_width(width)
            img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
            g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc,
                             want=("volume", "tf", "eye"))
            torch.cuda.synchronize()
            cur = (img.cpu(), g["volume"][0].cpu().numpy(), g["tf"].cpu().numpy(), g["eye"].cpu().numpy())
            if ref is None:
                ref = cur
                continue
            assert torch.equal(cur[0], ref[0]), width
            # gradients: binary32 sums in another order (atomics, other
            # warps per tile), equal to 1e-4 per element
            for a, b in zip(cur[1:], ref[1:]):
                assert_close(a, b, 1e-4, f"width {width}")
        # forward and adjoint widths set apart give the same results
        autotune.set_tile_width(32, 2)
        img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
        g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=("volume", "tf", "eye"))
        torch.cuda.synchronize()
        assert torch.equal(img.cpu(), ref[0])
        for a, b in zip((g["volume"][0].cpu().numpy(), g["tf"].cpu().numpy(), g["eye"].cpu().numpy()), ref[1:]):
            assert_close(a, b, 1e-4, "widths 32 / 2")
        res = autotune.autotune(sc, eye, w.step_voxels, want=("tf", "eye"), reps=2)
        assert res["width"] in autotune.CANDIDATES and autotune.get_tile_width() == res["width"]
        assert res["adjoint_width"] in autotune.CANDIDATES
        assert autotune.get_tile_width(adjoint=True) == res["adjoint_width"]
        # timed pass by pass with a buffer overwritten before each
        autotune._cache.clear()
        res = autotune.autotune(sc, eye, w.step_voxels, want=("tf", "eye"), reps=2,
                                l2_flush=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
        assert set(res["ms"]["forward|cells=0"]) == set(res["ms"]["adjoint|cells=0|cell_gradient=0"]) == \
            {str(c) for c in autotune.CANDIDATES}
        assert autotune.get_tile_width(adjoint=True) == res["adjoint_width"]
        assert res["cells"] == 0 and res["cell_gradient"] is False
        # with the gather layout and the scatter among the choices (volume gradient)
        autotune._cache.clear()
        res = autotune.autotune(sc, eye, w.step_voxels, want=("volume", "tf", "eye"), reps=1,
                                candidates=(8, 16), layouts=(0, 1, 4, 8), cell_gradients=(False, True))
        assert {f"forward|cells={c}" for c in (0, 1, 4, 8)} | \
            {f"adjoint|cells={c}|cell_gradient={g}" for c in (0, 1, 4, 8) for g in (0, 1)} == set(res["ms"])
        assert res["width"] in (8, 16) and res["adjoint_width"] in (8, 16)
        assert res["cells"] in (0, 1, 4, 8) and isinstance(res["cell_gradient"], bool)
        # the launch form of the volume-gradient adjoint: not a choice for a
        # binary32 volume, timed both ways for a 16-bit one
        autotune._cache.clear()
        res = autotune.autotune(sc, eye, w.step_voxels, want=("volume", "tf", "eye"), reps=1, candidates=(8,),
                                persistent=(False, True))
        assert res["persistent_scatter"] is False and not any(k.endswith("|persistent") for k in res["ms"])
        sc16 = dvr.Scene.make([to_dev(w.volumes[0], torch.float16)], tf, w.model, w.views)
        res = autotune.autotune(sc16, eye, w.step_voxels, want=("volume", "tf", "eye"), reps=1, candidates=(8,),
                                layouts=(4,), cell_gradients=(True,), persistent=(False, True))
        pk = "adjoint|cells=4|cell_gradient=1|width=8|persistent"
        assert set(res["ms"][pk]) == {"0", "1"} and isinstance(res["persistent_scatter"], bool)
    finally:
        autotune.set_tile_width(old, old_adj)


# ------------------------------------------------ inversion ablation (Sec. 4.4)
def test_inversion_ablation_at_high_opacity():
    """Opacity recovery before each sample, on the full 256^3 / 512^2 EA
    workload (tau up to 50 per unit: many rays reach A = 1 in binary32).
    The optical-depth form (default) and the alpha form with its division in
    binary64 above A = 0.99 meet the gradient tolerance; the alpha form in
    binary32 (Eq. inv-blend-forward as printed) loses the gradient of every
    sample in front of a saturated pixel and is much worse."""
    w = syn.workload("ea_256")
    vols = [to_dev(w.volumes[0])]
    tf = to_dev(w.tf)
    eye = to_dev(w.eye)
    img, aux = dvr.forward(vols, tf, w.model, w.views, eye, w.step_voxels)
    G = seeded_grad_image(img.shape[0], 4, 23)
    errs = {}
    ref = oracle.backward(as_oracle_volume(vols[0]), w.tf, w.model, w.views[0], w.eye[0], w.step_voxels, G,
                          want=("tf", "eye"), margin=FP32_MARGIN)
    for mode in ("depth", "alpha64", "alpha32"):
        g = dvr.backward(vols, tf, w.model, w.views, eye, w.step_voxels, aux, to_dev(G), want=("tf", "eye"),
                         inversion=mode)
        torch.cuda.synchronize()
        from tests.gpu_helpers import rel_err
        errs[mode] = rel_err(g["tf"].cpu().numpy(), ref["tf"])
    assert errs["depth"] <= GRAD_RTOL, errs
    assert errs["alpha64"] <= GRAD_RTOL, errs
    assert errs["alpha32"] > 10 * errs["depth"], errs


# ------------------------------------------------------------- volume shapes
@pytest.mark.parametrize("shape,model", [((24, 40, 33), "emission_absorption"),   # nz, ny, nx: non-cubic box
                                         ((7, 2, 5), "emission_absorption"),      # two vertices along y
                                         ((17, 9, 30), "absorption")])
def test_non_cubic_volumes(shape, model):
    """Boxes whose axes differ (the longest has length 1, the others shorter,
    as for the paper's 256 x 256 x 161 tooth) and a 2-vertex axis."""
    rng = np.random.default_rng(sum(shape))
    vol = rng.uniform(0.05, 0.95, shape).astype(np.float32)
    tf = syn.random_tf(9, seed=7, tau_max=12.0) if model == "emission_absorption" else None
    w = syn.Workload("shape", model, [vol], tf, [syn.View(37, 31), syn.View(20, 23, ortho=True, ortho_height=1.1)],
                     np.array([[0.7, 0.9, 1.6], [-1.2, 0.3, 0.8]], dtype=np.float32), None, 0.45,
                     ("volume", "tf", "camera"))
    want = ("volume", "tf", "eye") if tf is not None else ("volume", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    _compare(w, gpu, ref, want)


# ------------------------------------------------------------- TF row counts
@pytest.mark.parametrize("R", [2, 33, 1024])
def test_tf_sizes_at_the_limits(R):
    """The smallest TF (one segment), the first size past the per-lane
    shared-memory copies (R = 33: per-warp copies with register runs) and the
    largest (R = 1024 rows staged in shared memory). The rows sample one
    smooth TF, as a high-resolution TF does: with independent random rows the
    slope grows with R, and at R = 1024 the binary32 rounding of the density
    alone moves pixels by ~6e-5, beyond the image tolerance."""
    rng = np.random.default_rng(R)
    vol = rng.uniform(0.02, 0.98, (14, 13, 12)).astype(np.float32)
    x = np.linspace(0.0, 1.0, R)
    tf = np.stack([0.5 + 0.4 * np.sin(2 * np.pi * (x + 0.1)), 0.5 + 0.4 * np.cos(3 * np.pi * x),
                   x, 10.0 * (1.0 + np.sin(5 * np.pi * x + 0.3))], axis=1).astype(np.float32)
    w = syn.Workload("tf_rows", "emission_absorption", [vol], tf, [syn.View(23, 17), syn.View(9, 30)],
                     np.array([[0.9, 0.5, 1.7], [-1.3, 0.8, -1.1]], dtype=np.float32), None, 0.4,
                     ("volume", "tf", "camera"))
    want = ("volume", "tf", "eye")
    gpu = _run_gpu(w, want=want)
    ref = _oracle(w, gpu[0], gpu[1], gpu[4], want=want)
    if R < 1024:
        _compare(w, gpu, ref, want)
        return
    # At R = 1024 each row's gradient gathers the samples of a density band
    # 2/1023 wide, and some entries are ill-conditioned: moving every stored
    # density by one binary32 ulp (random signs) moves the oracle's own
    # binary64 result by up to ~1% on such rows. A binary32 evaluation
    # cannot do better than that, so those entries may differ by what one
    # ulp of the volume makes (four times the largest of five such moves).
    _compare(w, gpu, ref, ("volume", "eye"))
    vol32 = w.volumes[0]
    moves = []
    for t in range(5):
        sign = np.random.default_rng(100 + t).choice([-1.0, 1.0], size=vol32.shape)
        vp = np.where(sign > 0, np.nextafter(vol32, np.float32(2)), np.nextafter(vol32, np.float32(-1)))
        wp = syn.Workload(w.name, w.model, [vp.astype(np.float32)], w.tf, w.views, w.eye, None, w.step_voxels,
                          w.grads)
        moves.append(np.abs(_oracle(wp, [to_dev(vp.astype(np.float32))], gpu[1], gpu[4], want=("tf",))[2]["tf"]
                            - ref[2]["tf"]))
    slack = 4.0 * np.max(moves, axis=0)
    assert_close(gpu[5]["tf"].cpu().numpy(), ref[2]["tf"], GRAD_RTOL, "grad tf", slack=slack)


# ------------------------------------------------------------------ probes
def test_bandwidth_probes_run_and_count():
    """The roofline probes run; the reduction probe adds exactly `reps` to
    every word of a power-of-two buffer (its scattered order is a
    permutation of the words)."""
    from paper_2107_12672_b300 import _abi
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    sink = torch.zeros(1, device="cuda")
    buf = torch.zeros(1 << 20, device="cuda")            # 4 MiB, 2^20 words
    _abi.check(lib.dvr_probe(_abi.DVR_PROBE_L2_RED, buf.data_ptr(), buf.numel() * 4, 3, sink.data_ptr(), stream),
               "dvr_probe")
    torch.cuda.synchronize()
    assert torch.equal(buf, torch.full_like(buf, 3.0))
    for kind in (_abi.DVR_PROBE_L2_READ, _abi.DVR_PROBE_L1_READ):
        _abi.check(lib.dvr_probe(kind, buf.data_ptr(), buf.numel() * 4, 2, sink.data_ptr(), stream), "dvr_probe")
    torch.cuda.synchronize()
    assert float(sink.item()) == 0.0


# ------------------------------------------------------------ tile order
@pytest.mark.parametrize("width", [1, 8, 32])
def test_tile_order_changes_nothing(width):
    """With the centre-out tile order of dvr_tile_order and a persistent
    launch (warps taking tiles from the workspace's queue), dvr_forward
    writes every pixel of a NaN-filled image, counts the same samples (a
    tile taken twice would count twice) and gives the same bits as the fixed
    order with one tile per warp; the adjoint's gradients agree up to the
    order of atomic additions."""
    import ctypes
    from paper_2107_12672_b300 import _abi, autotune
    w = syn.workload("ea_256", scale=0.125)
    views = [syn.View(37, 29), syn.View(1, 1), syn.View(64, 3), syn.View(3, 64), syn.View(50, 50)]
    eye = to_dev(2.5 * syn.fibonacci_sphere(9)[:len(views)])
    vol, tf = to_dev(w.volumes[0]), to_dev(w.tf)
    sc = dvr.Scene.make([vol], tf, w.model, views)
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    old = autotune.get_tile_width(), autotune.get_tile_width(adjoint=True)
    out = []
    try:
        autotune.set_tile_width(width)
        for use_order in (False, True):
            # the second pass also runs the forward persistent (tile queue)
            order, n = sc.tile_order(lib, adjoint=False) if use_order else (None, 0)
            wsf = sc.workspace(lib) if use_order else None
            img = torch.full((sc.pixels, 4), float("nan"), device="cuda")
            aux = torch.full((sc.pixels, 2), float("nan"), device="cuda")
            count = torch.zeros(1, dtype=torch.int64, device="cuda")
            rc = lib.dvr_forward(sc.vol_desc, 1, sc.tf_ref(), sc.model, sc.view_desc, len(views), eye.data_ptr(),
                                 ctypes.c_float(w.step_voxels), img.data_ptr(), aux.data_ptr(), count.data_ptr(),
                                 None if order is None else order.data_ptr(), n,
                                 None if wsf is None else wsf.data_ptr(), 0 if wsf is None else wsf.numel(), stream)
            _abi.check(rc, "dvr_forward")
            G = to_dev(seeded_grad_image(sc.pixels, 4, 3))
            ordered, n_b = sc.tile_order(lib, adjoint=True) if use_order else (None, 0)
            grads = {"tf": torch.zeros((w.tf.shape[0], 4), device="cuda"), "eye": torch.zeros((len(views), 3), device="cuda")}
            ws = sc.workspace(lib)
            rc = lib.dvr_backward(sc.vol_desc, 1, sc.tf_ref(), sc.model, sc.view_desc, len(views), eye.data_ptr(),
                                  ctypes.c_float(w.step_voxels), aux.data_ptr(), G.data_ptr(), None,
                                  grads["tf"].data_ptr(), grads["eye"].data_ptr(), None, 0,
                                  None if ordered is None else ordered.data_ptr(), n_b, ws.data_ptr(), ws.numel(),
                                  stream)
            _abi.check(rc, "dvr_backward")
            torch.cuda.synchronize()
            out.append((img.cpu(), aux.cpu(), int(count.item()), grads["tf"].cpu().numpy(), grads["eye"].cpu().numpy()))
    finally:
        autotune.set_tile_width(*old)
    (i0, a0, c0, t0, e0), (i1, a1, c1, t1, e1) = out
    assert not torch.isnan(i1).any() and not torch.isnan(a1).any()
    assert c0 == c1 > 0
    assert torch.equal(i0, i1) and torch.equal(a0, a1)
    assert_close(t1, t0, 1e-5, "grad tf")
    assert_close(e1, e0, 1e-5, "grad eye")


# ------------------------------------------- per-K-step opacity checkpoints
def test_checkpoints_bound_the_alpha_form_drift():
    """The paper's alpha-form opacity recovery restarted from the forward's
    value every K samples (Sec. 4.4 ablation): on the 256^3 / 512^2 EA
    workload (tau up to 50 per unit) its TF-gradient error against the FP64
    oracle falls with K; with a checkpoint at every sample (K = 1) both the
    binary32 form and the binary64-guarded one meet the gradient tolerance,
    and so does the guarded one at K = 16. The checkpointed forward's image
    is the forward's, bit for bit, and slot 0 of every hit ray holds 1."""
    from tests.gpu_helpers import rel_err
    w = syn.workload("ea_256")
    vols = [to_dev(w.volumes[0])]
    tf = to_dev(w.tf)
    eye = to_dev(w.eye)
    sc = dvr.Scene.make(vols, tf, w.model, w.views)
    img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
    G = seeded_grad_image(img.shape[0], 4, 23)
    ref = oracle.backward(as_oracle_volume(vols[0]), w.tf, w.model, w.views[0], w.eye[0], w.step_voxels, G,
                          want=("tf", "eye"), margin=FP32_MARGIN)
    errs = {}
    for mode in ("alpha32", "alpha64"):
        g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, to_dev(G), scene=sc, want=("tf",),
                         inversion=mode)
        torch.cuda.synchronize()
        errs[(mode, None)] = rel_err(g["tf"].cpu().numpy(), ref["tf"])
        for k in (256, 16, 1):
            slots = dvr.checkpoint_slots(sc, w.step_voxels, k)
            ck = torch.full((sc.pixels, slots), -1.0, device="cuda")
            img_k, aux_k = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc, checkpoints=(ck, k))
            g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux_k, to_dev(G), scene=sc, want=("tf",),
                             inversion=mode, checkpoints=(ck, k))
            torch.cuda.synchronize()
            assert torch.equal(img_k, img) and torch.equal(aux_k, aux)
            hit = img[:, 3].cpu() > 0
            assert torch.all(ck[:, 0].cpu()[hit] == 1.0)
            errs[(mode, k)] = rel_err(g["tf"].cpu().numpy(), ref["tf"])
    print({f"{m}/K={k}": f"{e:.2e}" for (m, k), e in errs.items()})
    assert errs[("alpha32", 1)] <= GRAD_RTOL and errs[("alpha64", 1)] <= GRAD_RTOL, errs
    assert errs[("alpha32", 16)] <= errs[("alpha32", 256)] <= errs[("alpha32", None)], errs
    assert errs[("alpha32", 16)] < 0.1 * errs[("alpha32", None)], errs
    assert errs[("alpha64", 16)] <= GRAD_RTOL, errs


def test_tile_order_across_launches():
    """More than 512 views make several launches; the binding's centre-out
    tile order is one array whose part for each launch starts after the
    previous launch's tiles. The adjoint with it equals the adjoint in the
    fixed order (dvr_backward_noalloc takes no order) up to the order of
    atomic additions: every view's eye gradient and the step gradient."""
    import ctypes
    from paper_2107_12672_b300 import _abi
    n = 600
    w = syn.workload("absorption_64", scale=0.25)
    views = [syn.View(3 + k % 5, 2 + k % 7) for k in range(n)]
    eye = to_dev(2.5 * syn.fibonacci_sphere(n))
    vol = to_dev(w.volumes[0])
    sc = dvr.Scene.make([vol], None, "absorption", views)
    img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
    G = to_dev(seeded_grad_image(sc.pixels, 1, 8))
    # the binding passes its tile order to adjoints without a density gradient
    g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=("eye", "step"))
    lib = _abi.load()
    ref_e = torch.zeros((n, 3), device="cuda")
    ref_s = torch.zeros(1, device="cuda")
    rc = lib.dvr_backward_noalloc(sc.vol_desc, 1, None, _abi.DVR_ABSORPTION, sc.view_desc, n, eye.data_ptr(),
                                  ctypes.c_float(w.step_voxels), aux.data_ptr(), G.data_ptr(), None, None,
                                  ref_e.data_ptr(), ref_s.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    _abi.check(rc, "dvr_backward_noalloc")
    torch.cuda.synchronize()
    assert int((ref_e.abs().sum(1) > 0).sum()) > n // 2
    assert_close(g["eye"].cpu().numpy(), ref_e.cpu().numpy(), 1e-5, "grad eye")
    assert_close(g["step"].cpu().numpy(), ref_s.cpu().numpy(), 1e-5, "grad step")


# ------------------------------------------------ opacity entropy (Sec. 5.1)
@pytest.mark.parametrize("channels", [1, 4])
def test_loss_entropy_matches_oracle(channels):
    """Per view (uneven sizes, one with unlit pixels, one of a single pixel):
    the loss scale * sum(-H) and the opacity gradient match the oracle's
    binary64 definition; the colour channels of the gradient are zero."""
    rng = np.random.default_rng(11 + channels)
    views = [syn.View(37, 23), syn.View(1, 1), syn.View(64, 50), syn.View(9, 4)]
    sc_views = dvr.Scene.make([to_dev(np.zeros((4, 4, 4), np.float32))], None, "absorption", views)
    P = sc_views.pixels
    img = rng.uniform(0.0, 1.0, (P, channels)).astype(np.float32)
    off = sc_views.offsets
    img[off[2]:off[2] + 500, channels - 1] = 0.0          # unlit pixels
    scale = 0.7
    loss = torch.zeros(1, device="cuda")
    g = dvr.loss_entropy(to_dev(img), sc_views, scale, loss=loss)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    ref_loss, ref_g = 0.0, np.zeros((P, channels))
    for k, v in enumerate(views):
        n = v.width * v.height
        H, dH = oracle.opacity_entropy(img[off[k]:off[k] + n, channels - 1].astype(np.float64))
        ref_loss += -scale * H
        ref_g[off[k]:off[k] + n, channels - 1] = -scale * dH
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    assert np.all(g[:, :channels - 1] == 0.0)
    assert_close(g, ref_g, 1e-5, "entropy gradient")


def test_viewpoint_entropy_gradient_end_to_end():
    """Sec. 5.1 on the GPU: orbit camera -> forward -> opacity-entropy seed ->
    adjoint (eye) -> orbit adjoint gives dH/d(yaw, pitch, distance) equal to
    central differences of the rendered entropy, and five normalised ascent
    steps along it raise the entropy.

    H is differentiable in the camera only where moving it adds or drops no
    opacity: a sample appears or vanishes at a ray's exit, and a pixel's ray
    enters or leaves the box, in jumps the gradient does not see. So the TF's
    absorption is zero at density 0 and the blobs are narrow enough that the
    density at the box faces is near zero; with a random TF (absorption up to
    30 at density 0) the jumps dominate any difference quotient."""
    vol = to_dev(syn.gaussian_blobs(32, 6, seed=21, sigma=(4.0, 6.0)))
    x = np.linspace(0.0, 1.0, 12)
    tf = to_dev(np.stack([0.2 + 0.8 * x, 0.9 - 0.7 * x, 0.5 + 0.4 * np.sin(3 * x), 12.0 * x * x],
                         axis=1).astype(np.float32))
    views = [syn.View(48, 40)]
    sc = dvr.Scene.make([vol], tf, "emission_absorption", views)
    step = 0.5

    def entropy(params, want_grad=False):
        eye = dvr.orbit_eye(params)
        img, aux = dvr.forward(None, None, None, None, eye, step, scene=sc)
        loss = torch.zeros(1, device="cuda")
        g_img = dvr.loss_entropy(img, sc, -1.0, loss=loss)   # scale -1: loss = +H, seed = dH/dA
        if not want_grad:
            torch.cuda.synchronize()
            return float(loss.item())
        g = dvr.backward(None, None, None, None, eye, step, aux, g_img, scene=sc, want=("eye",))
        gp = dvr.orbit_eye_backward(params, g["eye"])
        torch.cuda.synchronize()
        return float(loss.item()), gp.cpu().numpy()[0]

    params = torch.tensor([[0.7, 0.35, 2.2]], device="cuda")
    H0, grad = entropy(params, True)
    assert np.abs(grad).max() > 1e-2, grad
    h = 5e-3
    for a in range(3):
        pp, pm = params.clone(), params.clone()
        pp[0, a] += h
        pm[0, a] -= h
        fd = (entropy(pp) - entropy(pm)) / (2 * h)
        assert abs(fd - grad[a]) <= 0.03 * np.abs(grad).max() + 1e-4, (a, fd, grad)
    for _ in range(5):
        _, grad = entropy(params, True)
        params = params + torch.as_tensor(0.03 * grad / np.linalg.norm(grad), device="cuda").float()[None, :]
    assert entropy(params) > H0 + 1e-3, (H0, entropy(params))
