"""The cell layout of a volume (dvr_make_cells): per cell its 8 corner
values side by side, which the march kernels gather with one or two 16-byte
loads. Its contents against their definition, and every march with it
against the same march on the volume's own array: images, optical depths
and forward-mode tangents bit for bit (the same corner values enter the
same arithmetic), gradients up to the order of atomic additions."""
import numpy as np
import pytest
import torch

import paper_2107_12672_b300 as dvr
from paper_2107_12672_b300 import synthetic as syn
from tests.gpu_helpers import assert_close, seeded_grad_image, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [torch.float32, torch.float16, torch.bfloat16]


def _bits(t):
    return t.view(torch.int16) if t.element_size() == 2 else t.view(torch.int32)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("brick", [1, 4, 8])
def test_cell_layout_contents(dtype, brick):
    """Cell (i, j, k) holds V(i,j,k), V(i,j,k+1), V(i+1,j,k), V(i+1,j,k+1),
    V(i,j+1,k), V(i,j+1,k+1), V(i+1,j+1,k), V(i+1,j+1,k+1), bit for bit, at
    record i + (nx-1)(j + (ny-1)k) (row order) or B^3 (bi + bx (bj + by bk))
    + (i % B) + B (j % B) + B^2 (k % B) (bricks of B^3 cells, B = 4 or 8,
    (bi, bj, bk) = (i, j, k) / B), on a box with three different sizes that
    are no multiples of 4 or 8 (one size above 8)."""
    v = to_dev(np.random.default_rng(1).normal(size=(7, 6, 11)).astype(np.float32), dtype)
    c = dvr.make_cells(v, brick=brick).view(-1, 8)
    ref = torch.stack([v[:-1, :-1, :-1], v[1:, :-1, :-1], v[:-1, :-1, 1:], v[1:, :-1, 1:],
                       v[:-1, 1:, :-1], v[1:, 1:, :-1], v[:-1, 1:, 1:], v[1:, 1:, 1:]], dim=-1)   # [k][j][i][8]
    nz, ny, nx = 6, 5, 10                                                                        # cells per axis
    k, j, i = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
    if brick == 1:
        rec = i + nx * (j + ny * k)
    else:
        B = brick
        bx, by = (nx + B - 1) // B, (ny + B - 1) // B
        rec = B ** 3 * (i // B + bx * (j // B + by * (k // B))) + (i % B) + B * (j % B) + B * B * (k % B)
        assert c.shape[0] == bx * by * ((nz + B - 1) // B) * B ** 3
    got = c[rec.reshape(-1).to(c.device)]
    assert torch.equal(_bits(got.contiguous()), _bits(ref.reshape(-1, 8).contiguous()))


def _march(w, vols, tf, cells, G, want, brick=1):
    sc = dvr.Scene.make(vols, tf, w.model, w.views, cells=cells, cells_brick=brick)
    eye = to_dev(w.eye)
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc, sample_count=count)
    g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=want)
    torch.cuda.synchronize()
    return img, aux, int(count.item()), g


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("model", ["emission_absorption", "absorption"])
@pytest.mark.parametrize("brick", [1, 4, 8])
def test_cells_equal_linear(dtype, model, brick):
    """Forward and adjoint (volume, TF and eye gradients) of several views of
    uneven sizes over two non-cubic volumes, ragged tiles included, with and
    without the cell layout."""
    rng = np.random.default_rng(7)
    vols = [to_dev(syn.value_noise(n, seed=s)[:, :n - 3, :], dtype) for n, s in ((33, 2), (24, 3))]
    vols = [v.contiguous() for v in vols]
    tf = to_dev(syn.random_tf(16, seed=4)) if model == "emission_absorption" else None
    views = [syn.View(37, 29), syn.View(20, 21, volume_index=1), syn.View(16, 11, ortho=True, ortho_height=1.2)]
    eye = (syn.fibonacci_sphere(3) * 2.2).astype(np.float32)
    w = syn.Workload("cells", model, vols, tf, views, eye, None, 0.4, ("volume", "tf", "camera"))
    nc = 4 if model == "emission_absorption" else 1
    G = to_dev(seeded_grad_image(sum(v.width * v.height for v in views), nc, 9))
    want = ("volume", "tf", "eye") if tf is not None else ("volume", "eye")
    a = _march(w, vols, tf, None, G, want)
    cells = [dvr.make_cells(v, brick=brick) for v in vols]
    b = _march(w, vols, tf, cells, G, want, brick)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and a[2] == b[2]
    for i in range(len(vols)):
        assert_close(b[3]["volume"][i].cpu().numpy(), a[3]["volume"][i].cpu().numpy(), 1e-4, f"volume {i}")
    if tf is not None:
        assert_close(b[3]["tf"].cpu().numpy(), a[3]["tf"].cpu().numpy(), 1e-4, "tf")
    assert_close(b[3]["eye"].cpu().numpy(), a[3]["eye"].cpu().numpy(), 1e-4, "eye")


def test_cells_forward_tangent_bit_identical():
    """The forward-mode pass reads the cell layout too: same image and
    tangents bit for bit."""
    w = syn.workload("ea_256", scale=0.125)
    vol = to_dev(w.volumes[0], torch.float16)
    tf = to_dev(w.tf)
    eye = to_dev(w.eye)
    out = []
    for brick, cells in ((1, None), (1, [dvr.make_cells(vol)]), (4, [dvr.make_cells(vol, brick=4)]),
                         (8, [dvr.make_cells(vol, brick=8)])):
        sc = dvr.Scene.make([vol], tf, w.model, w.views, cells=cells, cells_brick=brick)
        img, tan = dvr.forward_tangent(None, None, None, None, eye, w.step_voxels, scene=sc)
        torch.cuda.synchronize()
        out.append((img, tan))
    for o in out[1:]:
        assert torch.equal(out[0][0], o[0]) and torch.equal(out[0][1], o[1])


def test_cells_full_size_1024():
    """The 1024^3 FP16 volume (value noise + 32 blobs) on two of its 2048^2
    views: images bit for bit, volume and TF gradients to the order of
    atomics, with a cell layout of 16 GiB."""
    w = syn.workload("ea_fp16_1024")
    vol = syn.large_volume(w.target["n"]).to(torch.float16)
    tf = to_dev(w.tf)
    w.views, w.eye = w.views[:2], w.eye[:2]
    G = torch.zeros((sum(v.width * v.height for v in w.views), 4), device="cuda")
    G[::97] = 1.0
    a = _march(w, [vol], tf, None, G, ("volume", "tf"))
    cells = [dvr.make_cells(vol, brick=4)]
    b = _march(w, [vol], tf, cells, G, ("volume", "tf"), brick=4)
    assert torch.equal(a[0], b[0]) and a[2] == b[2]
    diff = (a[3]["volume"][0] - b[3]["volume"][0]).abs().max().item()
    assert diff <= 1e-5 * a[3]["volume"][0].abs().max().item(), diff
    assert_close(b[3]["tf"].cpu().numpy(), a[3]["tf"].cpu().numpy(), 1e-4, "tf")


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("model", ["emission_absorption", "absorption"])
def test_cell_gradient_equals_vertex_scatter(dtype, model):
    """DVR_FLAG_CELL_GRADIENT (each cell run as two vector reductions into
    a cell-major array, then a pass adding each vertex's 8 cell entries)
    gives the volume gradient of the vertex scatter up to the order of the
    additions, for two volumes of different shapes; the other gradients are
    unchanged, with and without the cell layout for the gathers."""
    vols = [to_dev(syn.value_noise(n, seed=s)[:, :n - 3, :], dtype).contiguous() for n, s in ((33, 2), (24, 3))]
    tf = to_dev(syn.random_tf(16, seed=4)) if model == "emission_absorption" else None
    views = [syn.View(37, 29), syn.View(20, 21, volume_index=1), syn.View(16, 11, ortho=True, ortho_height=1.2)]
    eye = to_dev((syn.fibonacci_sphere(3) * 2.2).astype(np.float32))
    nc = 4 if model == "emission_absorption" else 1
    G = to_dev(seeded_grad_image(sum(v.width * v.height for v in views), nc, 9))
    want = ("volume", "tf", "eye") if tf is not None else ("volume", "eye")
    for brick, cells in ((1, None), (1, [dvr.make_cells(v) for v in vols]),
                         (4, [dvr.make_cells(v, brick=4) for v in vols]), (8, [dvr.make_cells(v, brick=8) for v in vols])):
        sc = dvr.Scene.make(vols, tf, model, views, cells=cells, cells_brick=brick)
        _, aux = dvr.forward(None, None, None, None, eye, 0.4, scene=sc)
        a = dvr.backward(None, None, None, None, eye, 0.4, aux, G, scene=sc, want=want)
        b = dvr.backward(None, None, None, None, eye, 0.4, aux, G, scene=sc, want=want, cell_gradient=True)
        torch.cuda.synchronize()
        for i in range(len(vols)):
            assert_close(b["volume"][i].cpu().numpy(), a["volume"][i].cpu().numpy(), 1e-4, f"volume {i}")
        for k in want[1:]:
            assert_close(b[k].cpu().numpy(), a[k].cpu().numpy(), 1e-4, k)


@pytest.mark.parametrize("dtype", DTYPES)
def test_persistent_scatter_equals_one_tile_per_warp(dtype):
    """DVR_FLAG_PERSISTENT_SCATTER (the volume-gradient adjoint with as
    many blocks as are resident, warps taking tiles from a queue) gives the
    gradients of the launch with one tile per warp, up to the order of the
    additions, for two volumes and three views: from the volume's array and
    from its cell layout in 4^3 bricks, with the vertex scatter and with the
    per-cell gradient."""
    vols = [to_dev(syn.value_noise(n, seed=s)[:, :n - 3, :], dtype).contiguous() for n, s in ((33, 5), (24, 6))]
    tf = to_dev(syn.random_tf(16, seed=7))
    views = [syn.View(37, 29), syn.View(20, 21, volume_index=1), syn.View(16, 11, ortho=True, ortho_height=1.2)]
    eye = to_dev((syn.fibonacci_sphere(3) * 2.2).astype(np.float32))
    G = to_dev(seeded_grad_image(sum(v.width * v.height for v in views), 4, 10))
    want = ("volume", "tf", "eye")
    for brick, cells in ((1, None), (4, [dvr.make_cells(v, brick=4) for v in vols])):
        sc = dvr.Scene.make(vols, tf, "emission_absorption", views, cells=cells, cells_brick=brick)
        _, aux = dvr.forward(None, None, None, None, eye, 0.4, scene=sc)
        for cg in (False, True):
            a = dvr.backward(None, None, None, None, eye, 0.4, aux, G, scene=sc, want=want, cell_gradient=cg)
            b = dvr.backward(None, None, None, None, eye, 0.4, aux, G, scene=sc, want=want, cell_gradient=cg,
                             persistent_scatter=True)
            torch.cuda.synchronize()
            for i in range(len(vols)):
                assert_close(b["volume"][i].cpu().numpy(), a["volume"][i].cpu().numpy(), 1e-4, f"volume {i}")
            for k in want[1:]:
                assert_close(b[k].cpu().numpy(), a[k].cpu().numpy(), 1e-4, k)


def test_cell_gradient_accumulates_and_full_size():
    """The cell-gradient pass adds into the caller's gradient (Alg. 2's +=)
    and zeroes its cell array on every call: two calls give twice one call.
    At full size (1024^3 FP16, two 2048^2 views, a 34 GB cell array) it
    equals the vertex scatter."""
    w = syn.workload("ea_fp16_1024")
    vol = syn.large_volume(w.target["n"]).to(torch.float16)
    tf = to_dev(w.tf)
    w.views, w.eye = w.views[:2], w.eye[:2]
    eye = to_dev(w.eye)
    sc = dvr.Scene.make([vol], tf, w.model, w.views)
    _, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=sc)
    G = torch.zeros((sc.pixels, 4), device="cuda")
    G[::97] = 1.0
    ws = torch.empty(dvr.cell_workspace_bytes(sc), dtype=torch.uint8, device="cuda")
    a = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=("volume",))["volume"][0]
    g = {"volume": [torch.zeros_like(a)]}
    for _ in range(2):
        dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=sc, want=("volume",), grads=g,
                     cell_gradient=True, workspace=ws)
    torch.cuda.synchronize()
    b = g["volume"][0]
    scale = a.abs().max().item()
    assert scale > 0
    assert (b - 2 * a).abs().max().item() <= 1e-5 * scale
