"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each test checks it against a
closed form, an exact identity, brute-force finite differences, or an
independently derived forward-mode result, chosen so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2107_12672_b300 import synthetic as syn


def _ortho(n=64, W=None, H=None):
    return syn.View(W or n, H or n, ortho=True, ortho_height=1.0)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("sigma", [0.3, 1.3, 7.0])
def test_beer_lambert_constant_density(sigma):
    """Absorption-only, constant density: 1 - A = exp(-sigma N dt) (Sec. 3.1,
    Beer-Lambert segment opacity). Ortho +z through a 64^3 box: L = 1 and
    N = 126 at step 0.5 voxel."""
    n = 64
    sigma = float(np.float32(sigma))
    vol = np.full((n, n, n), sigma, np.float32)
    img, N, S = oracle.render(vol, None, "absorption", _ortho(), [0, 0, 2.0], 0.5)
    assert (N == 126).all()
    dt = float(np.float32(0.5 / 63))
    np.testing.assert_allclose(img[:, 0], 1 - np.exp(-sigma * 126 * dt), rtol=1e-13)
    np.testing.assert_allclose(S, sigma * 126 * dt, rtol=1e-13)


def test_beer_lambert_perspective_every_pixel():
    """Same closed form per pixel for a perspective camera: each ray's
    opacity is 1 - exp(-sigma N_ray dt) whatever its length."""
    n = 16
    sigma = 2.0
    vol = np.full((n, n, n), sigma, np.float32)
    view = syn.View(23, 17)
    img, N, S = oracle.render(vol, None, "absorption", view, [0.7, 0.9, 1.8], 0.37)
    dt = float(np.float32(np.float32(0.37) / np.float32(15)))
    assert N.max() > 0 and (N == 0).any()
    np.testing.assert_allclose(img[:, 0], 1 - np.exp(-sigma * N * dt), rtol=1e-13, atol=1e-15)


def test_constant_tf_closed_form():
    """Emission-absorption with constant density and a constant TF row
    (rgb, tau): the Riemann sum of Eq. 1 with premultiplied emission gives
    C = rgb (1 - exp(-tau N dt)) and A = 1 - exp(-tau N dt)."""
    n = 12
    vol = np.full((n, n, n), 0.37)
    row = np.array([0.2, 0.5, 0.9, 3.0])
    tf = np.tile(row, (7, 1))
    view = syn.View(9, 11)
    img, N, _ = oracle.render(vol, tf, "emission_absorption", view, [1.1, -0.4, 1.6], 0.5)
    dt = float(np.float32(np.float32(0.5) / np.float32(11)))
    A = 1 - np.exp(-row[3] * N * dt)
    np.testing.assert_allclose(img[:, 3], A, rtol=1e-13, atol=1e-15)
    for ch in range(3):
        np.testing.assert_allclose(img[:, ch], row[ch] * A, rtol=1e-13, atol=1e-15)


def test_front_to_back_order_two_layers():
    """Two slabs of different colour along the view axis: front-to-back
    blending (Eq. blend-forward) makes the front slab's colour dominate:
    C = c_f (1 - e_f) + e_f c_b (1 - e_b), with e = exp(-tau N dt) per slab."""
    n = 9  # box [-0.5, 0.5], spacing 1/8; vertices z = 0.5 .. -0.5
    vol = np.zeros((n, n, n), np.float32)
    vol[5:, :, :] = 1.0      # z >= 1/8 (front half as seen from +z) -> density 1
    vol[:5, :, :] = 0.0
    # TF: density 0 -> blue, tau 2; density 1 -> red, tau 5 (R = 2)
    tf = np.array([[0, 0, 1, 2.0], [1, 0, 0, 5.0]])
    view = syn.View(1, 1, ortho=True, ortho_height=0.5)
    img, N, _ = oracle.render(vol, tf, "emission_absorption", view, [0, 0, 3.0], 0.5)
    dt = float(np.float32(np.float32(0.5) / np.float32(8)))
    # samples at z = 0.5 - i dt, i = 0..N-1; density along z (trilinear in z)
    z = 0.5 - np.arange(N[0]) * dt
    g = (z + 0.5) * 8
    d = np.clip(g - 4, 0, 1)             # 0 below vertex 4, ramps to 1 at vertex 5
    col = np.outer(1 - d, tf[0]) + np.outer(d, tf[1])
    a = 1 - np.exp(-dt * col[:, 3])
    C = np.zeros(3)
    T = 1.0
    for i in range(N[0]):
        C += T * a[i] * col[i, :3]
        T *= 1 - a[i]
    np.testing.assert_allclose(img[0, :3], C, rtol=1e-13)
    np.testing.assert_allclose(img[0, 3], 1 - T, rtol=1e-13)
    assert img[0, 0] > img[0, 2]  # front (red) dominates


def test_linear_ramp_riemann_sum():
    """Density linear in z, ortho camera along -z: the optical depth is the
    Riemann sum dt * sum_i d(z_i) with z_i = 1/2 - i dt (samples start at the
    entry face and advance by dt, Alg. 1)."""
    n = 33
    zs = np.linspace(-0.5, 0.5, n)
    a, b = 1.7, 0.4
    vol = np.broadcast_to((a * zs + b)[:, None, None], (n, n, n)).astype(np.float64)
    img, N, S = oracle.render(vol, None, "absorption", _ortho(n, 5, 5), [0, 0, 4.0], 0.7)
    dt = float(np.float32(np.float32(0.7) / np.float32(32)))
    Nn = int(N[0])
    expect = dt * (Nn * (a * 0.5 + b) - a * dt * Nn * (Nn - 1) / 2)
    np.testing.assert_allclose(S, expect, rtol=1e-13)


def test_trilinear_reproduces_multilinear_fields():
    """Trilinear interpolation on vertices at -ext/2 + j h reproduces any
    function of the form (a + b x)(c + d y)(e + f z) + linear exactly
    (Sec. 3.1: density at grid vertices, trilinear in between)."""
    rng = np.random.default_rng(0)
    nx, ny, nz = 9, 6, 13
    h = 1.0 / 12
    xs = -0.5 * (nx - 1) * h + np.arange(nx) * h
    ys = -0.5 * (ny - 1) * h + np.arange(ny) * h
    zs = -0.5 * (nz - 1) * h + np.arange(nz) * h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    f = lambda x, y, z: (0.3 + 1.1 * x) * (0.7 - 0.4 * y) * (1.2 + 0.9 * z) + 0.2 * x - 0.5 * z
    vol = f(X, Y, Z)
    pts = np.stack([rng.uniform(xs[0], xs[-1], 200), rng.uniform(ys[0], ys[-1], 200),
                    rng.uniform(zs[0], zs[-1], 200)], axis=1)
    d = oracle.interpolate(vol, pts)
    np.testing.assert_allclose(d, f(pts[:, 0], pts[:, 1], pts[:, 2]), rtol=1e-12, atol=1e-13)
    # a non-multilinear field is NOT reproduced (sanity of the test itself)
    d2 = oracle.interpolate(X ** 2, pts)
    assert np.abs(d2 - pts[:, 0] ** 2).max() > 1e-5


def test_ray_geometry_ortho_and_perspective():
    """Camera convention: eye on +z looks down -z with right = +x, up = +y,
    pixel row 0 at the top; perspective rays follow the pinhole formula
    w ~ (sx tan aspect, sy tan, -1)."""
    view = syn.View(8, 6, ortho=True, ortho_height=1.0)
    N, q, geo = oracle.rays((64, 64, 64), view, [0, 0, 2.0], 0.5)
    for p in [0, 5, 17, 47]:
        px, py = p % 8, p // 8
        sx = (2 * px + 1) / 8 - 1
        sy = 1 - (2 * py + 1) / 6
        np.testing.assert_allclose(geo[p, 2:5], [sx * 0.5 * 8 / 6, sy * 0.5, 0.5], rtol=1e-6)
        np.testing.assert_allclose(geo[p, 5:8], [0, 0, -1])
        np.testing.assert_allclose(geo[p, 0], 1.5, rtol=1e-7)
    t = math.tan(math.radians(30))
    view = syn.View(7, 5, tan_half_fov_y=t)
    N, q, geo = oracle.rays((16, 16, 16), view, [0, 0, 2.5], 0.5, fp32=False)
    for p in range(35):
        px, py = p % 7, p // 7
        v = np.array([((2 * px + 1) / 7 - 1) * t * 7 / 5, (1 - (2 * py + 1) / 5) * t, -1.0])
        np.testing.assert_allclose(geo[p, 5:8], v / np.linalg.norm(v), rtol=1e-13, atol=1e-15)
    # centre pixel of an odd image points at the box centre from any eye
    e = np.array([0.8, -1.3, 1.9])
    N, q, geo = oracle.rays((16, 16, 16), view, e, 0.5, fp32=False)
    np.testing.assert_allclose(geo[17, 5:8], -e / np.linalg.norm(e), rtol=1e-13)


def test_orbit_camera_convention():
    """Orbit parameters (yaw, pitch, distance): yaw = pitch = 0 puts the eye on
    +z; pitch = pi/2 on +y; |eye| = distance (Sec. 5.1 longitude/latitude)."""
    e = oracle.orbit_eye([[0, 0, 2.5], [0, math.pi / 2, 3.0], [math.pi / 2, 0, 1.0],
                          [0.3, -0.2, 2.0]])
    np.testing.assert_allclose(e[0], [0, 0, 2.5], atol=1e-15)
    np.testing.assert_allclose(e[1], [0, 3.0, 0], atol=1e-15)
    np.testing.assert_allclose(e[2], [1.0, 0, 0], atol=1e-15)
    assert abs(np.linalg.norm(e[3]) - 2.0) < 1e-14
    # finite differences of the orbit map against its adjoint
    p = np.array([[0.3, -0.2, 2.0]])
    g = np.array([[0.3, -1.2, 0.7]])
    ga = oracle.orbit_eye_backward(p, g)[0]
    for k in range(3):
        h = 1e-6
        dp = np.zeros_like(p)
        dp[0, k] = h
        fd = ((oracle.orbit_eye(p + dp) - oracle.orbit_eye(p - dp)) * g).sum() / (2 * h)
        assert abs(fd - ga[k]) < 1e-8


def test_image_orientation_right_is_plus_x():
    """A blob at +x appears in the right half of the image of a camera on +z
    (and at +y in the top rows)."""
    n = 32
    vol = syn.gaussian_blobs(n, 1, seed=0, centre=(30, 30), scale_to=32, sigma=(2, 3))
    # the single blob is centred at voxel ~ (30,30,30) of 32: +x, +y, +z corner
    img, _, _ = oracle.render(vol, None, "absorption", syn.View(16, 16, ortho=True), [0, 0, 2], 0.5)
    A = img[:, 0].reshape(16, 16)
    assert A[:, 8:].sum() > 10 * A[:, :8].sum()
    assert A[:8, :].sum() > 10 * A[8:, :].sum()


# ---------------------------------------------------------- exact identities
def test_absorption_transpose_identity():
    """Absorption-only: the optical depth S = P v is linear in the volume
    (Sec. 5.3: a linear problem). The adjoint with dL/dA = w / T_N returns
    P^T w, so <P r, w> = <r, grad> for any volume r (dot-product test)."""
    rng = np.random.default_rng(7)
    n = 10
    v = rng.uniform(0, 2, (n, n, n))
    r = rng.normal(size=(n, n, n))
    view = syn.View(13, 11)
    eye = [0.9, 0.5, 1.7]
    imgv, Nv, Sv = oracle.render(v, None, "absorption", view, eye, 0.6)
    _, _, Sr = oracle.render(r, None, "absorption", view, eye, 0.6)
    w = rng.normal(size=Sv.shape)
    T = 1 - imgv[:, 0]
    g = oracle.backward(v, None, "absorption", view, eye, 0.6, (w / np.where(T > 0, T, 1))[:, None],
                        want=("volume",))["volume"]
    lhs = float(np.dot(Sr, w))
    rhs = float(np.sum(r * g))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_inversion_equals_tape():
    """Sec. 4.4: reconstructing (A_i, C_i) with Eq. inv-blend-forward gives the
    same gradients as storing them, up to rounding, for moderate opacity."""
    rng = np.random.default_rng(3)
    n = 10
    v = rng.uniform(0, 1, (n, n, n))
    tf = syn.random_tf(6, seed=9, tau_max=4.0).astype(np.float64)
    view = syn.View(9, 8)
    eye = [0.6, 0.4, 1.9]
    G = rng.normal(size=(72, 4))
    a = oracle.backward(v, tf, "emission_absorption", view, eye, 0.5, G, invert=False)
    b = oracle.backward(v, tf, "emission_absorption", view, eye, 0.5, G, invert=True)
    for k in ("volume", "tf", "eye"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-9, atol=1e-12 * np.abs(a[k]).max())


# ------------------------------------------------ brute-force finite differences
def _loss(img, G):
    return float(np.sum(img * G))


def _fd_setup(model, ortho=False, eye=(0.9, 0.6, 1.7), seed=11, R=5):
    rng = np.random.default_rng(seed)
    n = 8
    v = rng.uniform(0.05, 0.95, (n, n, n))
    tf = None
    if model == "emission_absorption":
        tf = rng.uniform(0.1, 1.0, (R, 4))
        tf[:, 3] *= 6.0
    view = syn.View(6, 5, ortho=ortho, ortho_height=1.3) if ortho else syn.View(6, 5)
    nc = 4 if model == "emission_absorption" else 1
    G = rng.normal(size=(30, nc))
    return v, tf, view, np.array(eye), G


@pytest.mark.parametrize("model", ["absorption", "emission_absorption"])
def test_fd_volume_every_voxel(model):
    """Central differences of L = <G, image> w.r.t. every voxel of an 8^3
    volume equal the adjoint gradient (Alg. 2; Eq. simpleadjoint)."""
    v, tf, view, eye, G = _fd_setup(model)
    g = oracle.backward(v, tf, model, view, eye, 0.5, G, fp32=False, want=("volume",))["volume"]
    h = 1e-6
    fd = np.zeros_like(v)
    for idx in np.ndindex(v.shape):
        vp = v.copy(); vp[idx] += h
        vm = v.copy(); vm[idx] -= h
        fd[idx] = (_loss(oracle.render(vp, tf, model, view, eye, 0.5, fp32=False)[0], G)
                   - _loss(oracle.render(vm, tf, model, view, eye, 0.5, fp32=False)[0], G)) / (2 * h)
    scale = np.abs(g).max()
    assert scale > 0
    assert np.abs(fd - g).max() <= 1e-6 * scale
    assert np.count_nonzero(np.abs(g) > 1e-3 * scale) > 50


def test_fd_tf_every_entry():
    """Central differences w.r.t. every TF entry (r, g, b, tau of each of the
    R control points) equal the adjoint's T^ (Alg. 2, f_TF line)."""
    model = "emission_absorption"
    v, tf, view, eye, G = _fd_setup(model, R=5)
    g = oracle.backward(v, tf, model, view, eye, 0.5, G, fp32=False, want=("tf",))["tf"]
    h = 1e-6
    fd = np.zeros_like(tf)
    for idx in np.ndindex(tf.shape):
        tp = tf.copy(); tp[idx] += h
        tm = tf.copy(); tm[idx] -= h
        fd[idx] = (_loss(oracle.render(v, tp, model, view, eye, 0.5, fp32=False)[0], G)
                   - _loss(oracle.render(v, tm, model, view, eye, 0.5, fp32=False)[0], G)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7 * np.abs(g).max())


@pytest.mark.parametrize("model,ortho,eye", [
    ("absorption", False, (0.9, 0.6, 1.7)),
    ("emission_absorption", False, (0.9, 0.6, 1.7)),
    ("emission_absorption", True, (-1.2, 0.5, 1.4)),
    ("emission_absorption", False, (0.0, 2.2, 0.0)),      # looking along -y (fixed right)
    ("emission_absorption", False, (0.1, 0.15, 0.3)),     # camera inside the box
])
def test_fd_eye(model, ortho, eye):
    """Central differences w.r.t. the eye position equal the adjoint's camera
    gradient, including the entry point's dependence on the camera."""
    v, tf, view, eye, G = _fd_setup(model, ortho=ortho, eye=eye)
    g = oracle.backward(v, tf, model, view, eye, 0.5, G, fp32=False, want=("eye",))["eye"]
    h = 1e-6
    for k in range(3):
        ep = eye.copy(); ep[k] += h
        em = eye.copy(); em[k] -= h
        ip, Np, _ = oracle.render(v, tf, model, view, ep, 0.5, fp32=False)
        im, Nm, _ = oracle.render(v, tf, model, view, em, 0.5, fp32=False)
        assert (Np == Nm).all(), "N changed within the FD step: move the eye"
        fd = (_loss(ip, G) - _loss(im, G)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, np.abs(g).max()), (k, fd, g[k])


def test_fd_step():
    """Central differences w.r.t. the step size (Alg. 2: dt^ += i w.x^_i plus
    the dependence of alpha on dt), with N held fixed."""
    model = "emission_absorption"
    v, tf, view, eye, G = _fd_setup(model)
    step = 0.53
    g = oracle.backward(v, tf, model, view, eye, step, G, fp32=False, want=("step",))["step"]
    h = 1e-7
    ip, Np, _ = oracle.render(v, tf, model, view, eye, step + h, fp32=False)
    im, Nm, _ = oracle.render(v, tf, model, view, eye, step - h, fp32=False)
    assert (Np == Nm).all()
    fd = (_loss(ip, G) - _loss(im, G)) / (2 * h)
    assert abs(fd - g) <= 1e-6 * max(1.0, abs(g))


# --------------------------------------------------- forward mode vs adjoint
@pytest.mark.parametrize("model,ortho", [("absorption", False), ("emission_absorption", False),
                                         ("emission_absorption", True)])
def test_dual_numbers_match_adjoint(model, ortho):
    """Sec. 5.1: forward and adjoint differentiation give the same camera
    gradient up to rounding. The dual-number render is an independent
    derivation of d(image)/d(eye)."""
    v, tf, view, eye, G = _fd_setup(model, ortho=ortho, eye=(1.1, -0.7, 1.5))
    img, dimg = oracle.render_dual(v, tf, model, view, eye, 0.5)
    img64, _, _ = oracle.render(v, tf, model, view, eye, 0.5, fp32=False)
    np.testing.assert_allclose(img, img64, rtol=1e-13, atol=1e-15)
    fwd = np.einsum("pc,pck->k", G, dimg)
    adj = oracle.backward(v, tf, model, view, eye, 0.5, G, fp32=False, want=("eye",))["eye"]
    np.testing.assert_allclose(adj, fwd, rtol=1e-10, atol=1e-12 * np.abs(fwd).max())


def test_fp32_setup_close_to_fp64():
    """The binary32 ray setup differs from the binary64 one by rounding only
    (images agree to ~1e-6 where N agrees)."""
    w = syn.workload("ea_256", scale=0.125)
    img32, N32, _ = oracle.render(w.volumes[0], w.tf, w.model, w.views[0], w.eye[0], 0.5, fp32=True)
    img64, N64, _ = oracle.render(w.volumes[0], w.tf, w.model, w.views[0], w.eye[0], 0.5, fp32=False)
    same = N32 == N64
    assert same.mean() > 0.99
    assert np.abs(img32[same] - img64[same]).max() < 1e-4


def test_kink_ambiguity_bounds_one_sided_derivatives():
    """At a TF control point the derivative of f_TF jumps (piecewise-linear
    TF, Sec. 3.1). With every sample exactly on a knot (constant density
    0.5, R = 5: u = 2), the central difference w.r.t. a voxel averages the
    two one-sided derivatives, so it must lie within the reported ambiguity
    of the adjoint's one-sided value; away from knots the ambiguity is 0."""
    n = 6
    v = np.full((n, n, n), 0.5)
    tf = np.array([[0.1, 0.2, 0.3, 1.0], [0.4, 0.1, 0.9, 3.0], [0.2, 0.8, 0.5, 2.0],
                   [0.9, 0.3, 0.1, 6.0], [0.5, 0.5, 0.5, 1.5]])
    view = syn.View(4, 3)
    eye = np.array([0.7, 0.5, 1.9])
    G = np.random.default_rng(2).normal(size=(12, 4))
    g = oracle.backward(v, tf, "emission_absorption", view, eye, 0.5, G, fp32=False,
                        want=("volume",), margin=1e6)
    amb = g["volume_ambiguity"]
    assert amb.max() > 0
    h = 1e-7
    for idx in [(3, 3, 3), (2, 3, 2), (3, 2, 3)]:
        vp = v.copy(); vp[idx] += h
        vm = v.copy(); vm[idx] -= h
        fd = (_loss(oracle.render(vp, tf, "emission_absorption", view, eye, 0.5, fp32=False)[0], G)
              - _loss(oracle.render(vm, tf, "emission_absorption", view, eye, 0.5, fp32=False)[0], G)) / (2 * h)
        assert abs(fd - g["volume"][idx]) <= amb[idx] * 0.5 + 1e-6 * np.abs(g["volume"]).max()
        assert abs(fd - g["volume"][idx]) >= amb[idx] * 0.5 - 1e-6 * np.abs(g["volume"]).max()
    v2 = np.full((n, n, n), 0.4)     # u = 1.6: no knot nearby
    g2 = oracle.backward(v2, tf, "emission_absorption", view, eye, 0.5, G, fp32=False,
                         want=("volume",), margin=1.0)
    assert g2["volume_ambiguity"].max() == 0


def _kink_ray(D_shift):
    """One perspective ray in the xz-plane-ish (pixel (5, 2) of a 7 x 6 view,
    eye on the +z axis at distance D) through a 9^3 box whose vertex plane
    x = 0.125 (vertex 5) holds a kink. D is chosen so that sample 3 lies
    exactly on that plane (D_shift = 0) or shifted so that no sample lies
    on any cell face or knot. Only that one sample sits on the kink, so a
    small move of the eye along any axis takes it to one side."""
    W, H, px, py = 7, 6, 5, 2
    view = syn.View(W, H)
    lens = view.tan_half_fov_y
    su = ((2 * px + 1) / W - 1) * lens * W / H
    sv = (1 - (2 * py + 1) / H) * lens
    dl = math.sqrt(1 + su * su + sv * sv)
    dt = 0.5 / 8
    D = 0.5 + (0.125 - 3 * dt * su / dl) / su + D_shift
    return view, np.array([py * W + px]), np.array([0.0, 0.0, D])


@pytest.mark.parametrize("kind", ["cell_face", "tf_knot"])
def test_eye_kink_ambiguity_bounds_one_sided_derivatives(kind):
    """The eye-gradient kink bound (`eye_ambiguity`) against central
    differences (Sec. 3.1: trilinear density, piecewise-linear TF; Alg. 2's
    f_interpolate adjoint takes one-sided derivatives there). A sample on a
    vertex plane across which the density's x-slope jumps (cell_face:
    absorption model, d = 1/2 + |i - 5|/4), or whose density sits exactly on
    a TF control point while the density varies along x (tf_knot: d = 3/16
    + i/16, R = 5, d = 1/2 at vertex 5): the central difference w.r.t. each
    eye coordinate averages the two one-sided derivatives, so it lies
    exactly half the reported bound away from the adjoint's one-sided value
    (the x and y coordinates also turn the ray, which the bound's chain
    through the direction adjoint must carry); with the
    ray moved off the plane the bound is exactly 0 and the central
    difference equals the adjoint. All vertex values are dyadic, so slopes
    away from the kink are exact and contribute nothing."""
    n = 9
    i = np.arange(n)
    if kind == "cell_face":
        model, tf = "absorption", None
        prof = 0.5 + 0.25 * np.abs(i - 5)
        G = np.array([[1.0]])
    else:
        model = "emission_absorption"
        prof = 0.1875 + 0.0625 * i
        tf = np.array([[0.1, 0.2, 0.3, 1.0], [0.4, 0.1, 0.9, 3.0], [0.2, 0.8, 0.5, 2.0],
                       [0.9, 0.3, 0.1, 6.0], [0.5, 0.5, 0.5, 1.5]])
        G = np.array([[0.3, -0.7, 0.5, 1.1]])
    v = np.broadcast_to(prof[None, None, :], (n, n, n)).astype(np.float64).copy()
    h = 1e-6
    for shift in (0.0, 0.0123):
        view, pix, eye = _kink_ray(shift)
        g = oracle.backward(v, tf, model, view, eye, 0.5, G, fp32=False, pix=pix, want=("eye",), margin=1.0)
        amb = g["eye_ambiguity"]
        scale = np.abs(g["eye"]).max()
        for k in range(3):
            ep = eye.copy(); ep[k] += h
            em = eye.copy(); em[k] -= h
            ip, Np, _ = oracle.render(v, tf, model, view, ep, 0.5, fp32=False, pix=pix)
            im, Nm, _ = oracle.render(v, tf, model, view, em, 0.5, fp32=False, pix=pix)
            assert (Np == Nm).all() and Np[0] > 8
            fd = (_loss(ip, G) - _loss(im, G)) / (2 * h)
            dev = abs(fd - g["eye"][k])
            if shift == 0.0:
                assert abs(dev - 0.5 * amb[k]) <= 1e-6 * scale, (k, dev, amb[k])
            else:
                assert amb[k] == 0, amb
                assert dev <= 1e-8 * scale, (k, fd, g["eye"][k])
        if shift == 0.0:
            assert amb[0] > 0.05 * scale and amb[2] > 0.05 * scale


# ------------------------------------------------------- pre-shaded colour volume
def test_color_volume_equals_ea_for_affine_tf():
    """Sec. 5.4 colour volume: per-vertex (r, g, b, tau), interpolated. An
    affine TF (R = 2) commutes with trilinear interpolation for densities in
    [0, 1], so the colour volume TF(v) renders exactly as the EA model."""
    rng = np.random.default_rng(4)
    n = 9
    v = rng.uniform(0.0, 1.0, (n, n, n))
    tf = np.array([[0.1, 0.7, 0.3, 1.5], [0.9, 0.2, 0.6, 6.0]])
    cv = tf[0][None, None, None, :] * (1 - v[..., None]) + tf[1][None, None, None, :] * v[..., None]
    view = syn.View(13, 10)
    eye = [0.8, -0.6, 1.7]
    a, Na, _ = oracle.render(v, tf, "emission_absorption", view, eye, 0.5)
    b, Nb, _ = oracle.render(cv, None, "color", view, eye, 0.5)
    assert (Na == Nb).all()
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-14)


def test_color_volume_constant_closed_form():
    n = 7
    row = np.array([0.3, 0.6, 0.1, 4.0])
    cv = np.broadcast_to(row, (n, n, n, 4)).copy()
    view = syn.View(5, 6)
    img, N, _ = oracle.render(cv, None, "color", view, [0.9, 0.4, 1.8], 0.5)
    dt = float(np.float32(np.float32(0.5) / np.float32(6)))
    A = 1 - np.exp(-row[3] * N * dt)
    np.testing.assert_allclose(img[:, 3], A, rtol=1e-13, atol=1e-15)
    for ch in range(3):
        np.testing.assert_allclose(img[:, ch], row[ch] * A, rtol=1e-13, atol=1e-15)


def test_color_volume_fd_every_entry_and_eye():
    """Central differences w.r.t. every channel of every vertex of a 6^3
    colour volume and w.r.t. the eye equal the adjoint."""
    rng = np.random.default_rng(5)
    n = 6
    cv = rng.uniform(0.1, 1.0, (n, n, n, 4))
    cv[..., 3] *= 5.0
    view = syn.View(5, 4)
    eye = np.array([0.9, 0.6, 1.7])
    G = rng.normal(size=(20, 4))
    g = oracle.backward(cv, None, "color", view, eye, 0.5, G, fp32=False, want=("volume", "eye"))
    h = 1e-6
    fd = np.zeros_like(cv)
    for idx in np.ndindex(cv.shape):
        vp = cv.copy(); vp[idx] += h
        vm = cv.copy(); vm[idx] -= h
        fd[idx] = (_loss(oracle.render(vp, None, "color", view, eye, 0.5, fp32=False)[0], G)
                   - _loss(oracle.render(vm, None, "color", view, eye, 0.5, fp32=False)[0], G)) / (2 * h)
    scale = np.abs(g["volume"]).max()
    assert np.abs(fd - g["volume"]).max() <= 1e-6 * scale
    for k in range(3):
        ep = eye.copy(); ep[k] += h
        em = eye.copy(); em[k] -= h
        fd_e = (_loss(oracle.render(cv, None, "color", view, ep, 0.5, fp32=False)[0], G)
                - _loss(oracle.render(cv, None, "color", view, em, 0.5, fp32=False)[0], G)) / (2 * h)
        assert abs(fd_e - g["eye"][k]) <= 1e-6 * max(1.0, np.abs(g["eye"]).max())
    img, dimg = oracle.render_dual(cv, None, "color", view, eye, 0.5)
    np.testing.assert_allclose(g["eye"], np.einsum("pc,pck->k", G, dimg), rtol=1e-9)


# ------------------------------------------------------ optimisation-side terms
def test_volume_prior_closed_form_and_fd():
    """3D smoothing prior (Sec. 5.3): a ramp a*z has every z-difference a and
    no x/y differences, so the sum is a^2 nx ny (nz - 1); the gradient of the
    quadratic matches central differences exactly."""
    nz, ny, nx = 5, 4, 6
    a = 0.7
    ramp = np.broadcast_to((a * np.arange(nz))[:, None, None], (nz, ny, nx))
    loss, grad = oracle.volume_prior(ramp)
    assert abs(loss - a * a * nx * ny * (nz - 1)) < 1e-12
    rng = np.random.default_rng(0)
    v = rng.normal(size=(3, 4, 5))
    loss, grad = oracle.volume_prior(v)
    for idx in [(0, 0, 0), (1, 2, 3), (2, 3, 4), (1, 0, 2)]:
        vp = v.copy(); vp[idx] += 1e-4
        vm = v.copy(); vm[idx] -= 1e-4
        fd = (oracle.volume_prior(vp)[0] - oracle.volume_prior(vm)[0]) / 2e-4
        assert abs(fd - grad[idx]) < 1e-8


def test_tf_prior_closed_form():
    """Eq. tf-loss prior: rows differing by a constant c in every channel sum
    to 4 (R - 1) c^2."""
    R, c = 9, 0.3
    tf = np.arange(R)[:, None] * c + np.zeros((1, 4))
    loss, grad = oracle.tf_prior(tf)
    assert abs(loss - 4 * (R - 1) * c * c) < 1e-12
    assert np.abs(grad[1:-1]).max() < 1e-12          # interior rows: equal differences cancel


def test_resample_reproduces_linear_fields():
    """Resampling onto a finer grid over the same box keeps a linear field
    exactly (trilinear reproduction), and the identity shape is the identity."""
    n = 5
    xs = np.linspace(-0.5, 0.5, n)
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    v = 0.3 + 1.1 * X - 0.7 * Y + 0.4 * Z
    up = oracle.resample(v, (9, 9, 9))
    xs9 = np.linspace(-0.5, 0.5, 9)
    Z9, Y9, X9 = np.meshgrid(xs9, xs9, xs9, indexing="ij")
    np.testing.assert_allclose(up, 0.3 + 1.1 * X9 - 0.7 * Y9 + 0.4 * Z9, atol=1e-13)
    np.testing.assert_allclose(oracle.resample(v, v.shape), v, atol=1e-14)


# ------------------------------------------------------- opacity entropy (Sec. 5.1)
def test_opacity_entropy_extremes():
    """Normalised entropy of the alpha channel: 1 for a uniform opacity, 0
    when one pixel holds all of it, and in between otherwise."""
    H, _ = oracle.opacity_entropy(np.full(64, 0.37))
    assert abs(H - 1.0) < 1e-14
    a = np.zeros(64)
    a[17] = 0.8
    H, _ = oracle.opacity_entropy(a)
    assert H == 0.0
    a[:8] = 0.5                                 # 9 lit pixels, not all equal
    H, _ = oracle.opacity_entropy(a)
    assert 0.0 < H < np.log(9) / np.log(64)


def test_opacity_entropy_gradient():
    """The gradient matches central differences at lit pixels, and since H
    does not change when every opacity is scaled by the same factor, Euler's
    identity sum_k A_k dH/dA_k = 0 holds."""
    rng = np.random.default_rng(7)
    a = rng.uniform(0.05, 0.95, 40)
    H, g = oracle.opacity_entropy(a)
    assert abs(float((a * g).sum())) < 1e-13
    h = 1e-6
    for k in (0, 13, 39):
        ap, am = a.copy(), a.copy()
        ap[k] += h
        am[k] -= h
        fd = (oracle.opacity_entropy(ap)[0] - oracle.opacity_entropy(am)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])
    # an unlit pixel: lighting it raises the entropy (logarithm at a_min)
    a[5] = 0.0
    _, g = oracle.opacity_entropy(a)
    assert g[5] > 0 and np.isfinite(g[5])


@pytest.mark.parametrize("model", ["absorption", "emission_absorption", "color"])
def test_compact_volume_gradient_equals_dense(model):
    """The compact volume-gradient output (one entry per vertex the listed
    rays read, for volumes whose dense binary64 gradient does not fit in
    host memory) holds exactly the dense gradient's values at those
    vertices, and the dense gradient is zero everywhere else."""
    rng = np.random.default_rng(8)
    n = 10
    if model == "color":
        v = rng.uniform(0.1, 1.0, (n, n, n, 4))
        tf = None
    else:
        v = rng.uniform(0.0, 1.0, (n, n, n))
        tf = rng.uniform(0.1, 1.0, (6, 4)) if model == "emission_absorption" else None
    view = syn.View(11, 9)
    eye = np.array([0.9, -0.5, 1.6])
    pix = np.array([3, 17, 40, 41, 77, 98])
    nc = 1 if model == "absorption" else 4
    G = rng.normal(size=(pix.size, nc))
    sel = oracle.touched(v.shape, view, eye, 0.5, pix=pix)
    assert sel.size > 8 and (np.diff(sel) > 0).all()
    dense = oracle.backward(v, tf, model, view, eye, 0.5, G, pix=pix, want=("volume", "eye"), margin=2.0)
    comp = oracle.backward(v, tf, model, view, eye, 0.5, G, pix=pix, want=("volume", "eye"), margin=2.0, sel=sel)
    flat = dense["volume"].reshape((n ** 3,) + v.shape[3:])
    np.testing.assert_allclose(comp["volume"], flat[sel], rtol=1e-13, atol=1e-15)
    rest = np.ones(n ** 3, bool)
    rest[sel] = False
    assert not flat[rest].any()
    assert np.abs(flat[sel]).max() > 0
    np.testing.assert_allclose(comp["eye"], dense["eye"], rtol=1e-13)
    if model == "emission_absorption":
        np.testing.assert_allclose(comp["volume_ambiguity"], dense["volume_ambiguity"].reshape(-1)[sel],
                                   rtol=1e-13, atol=1e-15)
    with pytest.raises(ValueError):
        oracle.backward(v, tf, model, view, eye, 0.5, G, pix=pix, want=("volume",), sel=sel[1:])
