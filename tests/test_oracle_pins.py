"""Pins of the FP64 oracle against closed forms, brute force, invariances and
textbook special cases (no GPU).  Each test names the passage or the
mathematical fact it checks."""
import json
import math
import os

import numpy as np
import pytest

from paper_2606_00352_gb300.scenes import Scene, Camera, uniform_scene, look_at, tiny_workload
from oracle import project as P
from oracle import composite as C
from oracle import batched as B
from oracle import binning as BN
from oracle import sh as SH

HERE = os.path.dirname(os.path.abspath(__file__))


def one_scene(means, log_scales, quats, logits, sh0):
    n = np.asarray(means, np.float64).reshape(-1, 3).shape[0]
    return Scene(np.asarray(means, np.float32).reshape(n, 3),
                 np.asarray(log_scales, np.float32).reshape(n, 3),
                 np.asarray(quats, np.float32).reshape(n, 4),
                 np.asarray(logits, np.float32).reshape(n),
                 np.asarray(sh0, np.float32).reshape(n, 1, 3), 0)


def axis_camera(w=64, h=64, f=64.0, cx=None, cy=None):
    """Camera at the origin looking along +z (identity world->camera)."""
    return Camera(np.eye(4, dtype=np.float32), f, f, w / 2 if cx is None else cx,
                  h / 2 if cy is None else cy, w, h)


Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def test_closed_form_isotropic_gaussian():
    """Isotropic gaussian on the optical axis: Sigma2 = (f s / d)^2 I + 0.3 I,
    centre at (cx - 0.5, cy - 0.5); pixel = c min(0.99, o e^{-q/2}) inside
    q <= 9 with alpha >= 1/255 (Sec. 3.4 rules, 3DGS projection)."""
    f, d, s, o = 64.0, 4.0, 0.25, 0.8
    sh0 = 0.3
    sc = one_scene([0, 0, d], [math.log(s)] * 3, [1, 0, 0, 0], [math.log(o / (1 - o))], [sh0] * 3)
    cam = axis_camera(f=f)
    pr = P.project(sc, cam)
    var = (f * s / d) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0.0, var], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(pr["mean2d"][0], [31.5, 31.5], atol=1e-9)
    assert pr["radius"][0] == math.ceil(3.0 * math.sqrt(var + math.sqrt(0.1)))
    img = C.render(pr)
    ys, xs = np.mgrid[0:64, 0:64]
    q = ((xs - 31.5) ** 2 + (ys - 31.5) ** 2) / var
    a = np.minimum(0.99, o * np.exp(-0.5 * q))
    a = np.where((q <= 9.0) & (a >= 1.0 / 255.0), a, 0.0)
    colour = sh0 * Y00 + 0.5
    np.testing.assert_allclose(img["rgb"][..., 0], colour * a, atol=1e-6)
    np.testing.assert_allclose(img["T"], 1.0 - a, atol=1e-6)


def test_anisotropic_rotation_about_view_axis():
    """A +45 deg rotation about the optical axis (quaternion (cos 22.5, 0, 0,
    sin 22.5), order w,x,y,z) turns diag(sx^2, sy^2) into an off-diagonal
    (sx^2 - sy^2)/2 (times (f/d)^2): pins the quaternion convention."""
    f, d, sx, sy, sz = 64.0, 4.0, 0.4, 0.1, 0.2
    th = math.radians(45.0)
    quat = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    sc = one_scene([0, 0, d], np.log([sx, sy, sz]), quat, [0.0], [0, 0, 0])
    pr = P.project(sc, axis_camera(f=f))
    k = (f / d) ** 2
    a = k * (sx * sx + sy * sy) / 2 + 0.3
    b = k * (sx * sx - sy * sy) / 2
    np.testing.assert_allclose(pr["cov2d"][0], [a, b, a], rtol=1e-5)
    det = a * a - b * b
    np.testing.assert_allclose(pr["conic"][0], [a / det, -b / det, a / det], rtol=1e-5)


def test_rotation_about_x_mixes_y_and_depth_scales():
    """Rotation by th about x maps the (y, z) scales onto image y as
    cos^2 sy^2 + sin^2 sz^2 for a gaussian on the optical axis."""
    f, d, sx, sy, sz, th = 50.0, 5.0, 0.1, 0.3, 0.05, 0.7
    quat = [math.cos(th / 2), math.sin(th / 2), 0, 0]
    sc = one_scene([0, 0, d], np.log([sx, sy, sz]), quat, [0.0], [0, 0, 0])
    pr = P.project(sc, axis_camera(f=f))
    k = (f / d) ** 2
    yy = k * (math.cos(th) ** 2 * sy * sy + math.sin(th) ** 2 * sz * sz) + 0.3
    assert abs(pr["cov2d"][0, 2] - yy) < 1e-6 * yy
    # float32 inputs: log(s) and the quaternion carry ~1e-7 relative rounding
    assert abs(pr["cov2d"][0, 0] - (k * sx * sx + 0.3)) < 1e-6 * (k * sx * sx + 0.3)
    assert abs(pr["cov2d"][0, 1]) < 1e-6 * k * sy * sy


def test_jacobian_is_derivative_of_pinhole_map():
    """EWA uses J = d(pi)/dt at the camera-space mean (Sec. 4.2 front end);
    checked against central differences of the pinhole map."""
    g = np.random.default_rng(3)
    cam = axis_camera(w=200, h=100, f=150.0)
    for _ in range(5):
        t = np.array([g.uniform(-0.3, 0.3), g.uniform(-0.2, 0.2), g.uniform(1.0, 3.0)])
        sc = one_scene(t, [-3, -3, -3], [1, 0, 0, 0], [0.0], [0, 0, 0])
        pr = P.project(sc, cam)

        def pi(v):
            return np.array([cam.fx * v[0] / v[2] + cam.cx - 0.5, cam.fy * v[1] / v[2] + cam.cy - 0.5])
        h = 1e-6
        fd = np.stack([(pi(t + h * e) - pi(t - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        t32 = np.asarray(t, np.float32).astype(np.float64)
        np.testing.assert_allclose(pr["jac"][0], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
        np.testing.assert_allclose(pr["mean2d"][0], pi(t32), atol=1e-9)


def test_jacobian_clamp_far_off_axis():
    """Off-screen means clamp x/z to +-1.3 tan(fov_x / 2) inside J."""
    cam = axis_camera(w=64, h=64, f=64.0)
    sc = one_scene([3.0, 0.0, 2.0], [-3, -3, -3], [1, 0, 0, 0], [0.0], [0, 0, 0])
    pr = P.project(sc, cam)
    lim = 1.3 * 0.5 * 64 / 64.0
    assert abs(pr["jac"][0, 0, 2] - (-64.0 * lim * 2.0 / 4.0)) < 1e-9


def test_near_plane_cull():
    sc = one_scene([[0, 0, 0.15], [0, 0, 0.25]], [[-3] * 3] * 2, [[1, 0, 0, 0]] * 2, [0, 0], [[0] * 3] * 2)
    pr = P.project(sc, axis_camera())
    assert list(pr["visible"]) == [False, True]


def test_rigid_motion_invariance():
    """Moving scene and camera by the same rigid motion leaves every
    projected quantity unchanged (pins rotation order and transposes)."""
    scene, cams = tiny_workload()
    sub = scene.subset(np.arange(400))
    cam = cams[0]
    g = np.random.default_rng(7)
    qm = g.standard_normal(4)
    qm /= np.linalg.norm(qm)
    rm = P.quat_to_rot(qm[None])[0]
    tr = g.standard_normal(3)
    moved = sub.copy()
    moved.means = (sub.means.astype(np.float64) @ rm.T + tr).astype(np.float32)
    w0, x0, y0, z0 = qm
    q = sub.quats.astype(np.float64)
    w1, x1, y1, z1 = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    moved.quats = np.stack([w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1,
                            w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
                            w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1,
                            w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1], 1).astype(np.float32)
    g4 = np.eye(4)
    g4[:3, :3] = rm
    g4[:3, 3] = tr
    vm = cam.viewmat.astype(np.float64) @ np.linalg.inv(g4)
    cam2 = Camera(vm.astype(np.float32), cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    a, b = P.project(sub, cam), P.project(moved, cam2)
    ok = a["visible"] & ~a["ambiguous"]
    np.testing.assert_allclose(a["mean2d"][ok], b["mean2d"][ok], atol=2e-4)
    np.testing.assert_allclose(a["cov2d"][ok], b["cov2d"][ok], rtol=2e-4, atol=1e-4)
    np.testing.assert_allclose(a["rgb"][ok], b["rgb"][ok], atol=1e-12)


def _tiny_random(n=64, w=16, h=16, seed=0):
    g = np.random.default_rng(seed)
    means = np.stack([g.uniform(-0.5, 0.5, n), g.uniform(-0.5, 0.5, n), g.uniform(2.0, 3.0, n)], 1)
    sc = one_scene(means, g.normal(-1.6, 0.4, (n, 3)), g.standard_normal((n, 4)),
                   g.normal(1.5, 1.5, n), g.uniform(-1.5, 1.5, (n, 3)))
    return sc, axis_camera(w=w, h=h, f=20.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_render_equals_brute_force(seed):
    """Tile-pruned vectorised compositing == per-pixel loop over every
    gaussian sorted by (key, id) (Sec. 3.4 definition)."""
    sc, cam = _tiny_random(seed=seed)
    pr = P.project(sc, cam)
    img = C.render(pr, bg=(0.1, 0.2, 0.3))
    worst = 0.0
    stops = 0
    for y in range(cam.height):
        for x in range(cam.width):
            c, t, st = C.pixel_brute_force(pr, x, y, bg=(0.1, 0.2, 0.3))
            worst = max(worst, np.abs(c - img["rgb"][y, x]).max(), abs(t - img["T"][y, x]))
            assert st == img["stopped"][y, x]
            stops += st
    assert worst < 1e-12
    if seed == 0:
        assert stops > 10  # the termination rule is exercised


@pytest.mark.parametrize("seed", [0, 1])
def test_pixel_work_equals_sequential_loop(seed):
    """Per-pixel work counts of the tile-pruned oracle == an explicit loop
    over every visible gaussian in (key, id) order: contributions as the
    sequential compositing loop counts them, support evaluations (q <= 9)
    up to and including the stopping gaussian."""
    sc, cam = _tiny_random(seed=seed)
    pr = P.project(sc, cam)
    n_sup, n_con = C.pixel_work(pr)
    vis = np.nonzero(pr["visible"])[0]
    order = vis[np.lexsort((vis, pr["depth_key"][vis]))]
    stops = 0
    for y in range(cam.height):
        for x in range(cam.width):
            q, al = C.alpha_at(pr, order, np.array([float(x)]), np.array([float(y)]))
            q, al = q[:, 0], al[:, 0]
            _, _, st, nc = C.composite_sequence(al, q, pr["rgb"][order])
            t, sup = 1.0, 0
            for i in range(len(order)):
                if q[i] > 9.0:
                    continue
                sup += 1
                if al[i] < 1.0 / 255.0:
                    continue
                t *= 1.0 - al[i]
                if t < 1e-4:
                    break
            assert n_con[y, x] == nc and n_sup[y, x] == sup, (x, y)
            stops += st
    assert stops > 10 or seed != 0


def test_pixel_work_of_the_termination_stack():
    """Five alpha = 0.95 layers at the centre pixel: three are blended and
    the fourth stops the pixel, so 3 contributions and 4 support
    evaluations."""
    cam = axis_camera(w=16, h=16, f=16.0, cx=8.5, cy=8.5)
    n = 5
    sc = one_scene([[0, 0, 2.0 + 0.1 * i] for i in range(n)], [[-2] * 3] * n,
                   [[1, 0, 0, 0]] * n, [math.log(0.95 / 0.05)] * n, [[0.4, 0.4, 0.4]] * n)
    n_sup, n_con = C.pixel_work(P.project(sc, cam))
    assert n_con[8, 8] == 3 and n_sup[8, 8] == 4


def test_two_gaussian_depth_order():
    """C = c1 a1 + c2 a2 (1 - a1) with the nearer gaussian first."""
    o1, o2 = 0.6, 0.7
    sh_a, sh_b = [1.0, 0, 0], [0, 1.0, 0]
    lg = lambda o: math.log(o / (1 - o))
    cam = axis_camera(w=16, h=16, f=16.0, cx=8.5, cy=8.5)  # centre pixel (8, 8)
    for near_first in (True, False):
        z1, z2 = (2.0, 3.0) if near_first else (3.0, 2.0)
        sc = one_scene([[0, 0, z1], [0, 0, z2]], [[-2] * 3] * 2, [[1, 0, 0, 0]] * 2,
                       [lg(o1), lg(o2)], [sh_a, sh_b])
        pr = P.project(sc, cam)
        img = C.render(pr)
        c1 = np.array(sh_a) * Y00 + 0.5
        c2 = np.array(sh_b) * Y00 + 0.5
        if near_first:
            want = c1 * o1 + c2 * o2 * (1 - o1)
        else:
            want = c2 * o2 + c1 * o1 * (1 - o2)
        np.testing.assert_allclose(img["rgb"][8, 8], want, atol=1e-12)


def test_termination_stack_alpha_095():
    """Five alpha = 0.95 layers: after three T = 0.05^3 = 1.25e-4 >= 1e-4,
    the fourth would give 6.25e-6 < 1e-4 so it is excluded and the pixel
    stops: C = c (1 - 0.05^3) exactly (3DGS termination rule)."""
    cam = axis_camera(w=16, h=16, f=16.0, cx=8.5, cy=8.5)
    n = 5
    lg = math.log(0.95 / 0.05)
    sc = one_scene([[0, 0, 2.0 + 0.1 * i] for i in range(n)], [[-2] * 3] * n,
                   [[1, 0, 0, 0]] * n, [lg] * n, [[0.4, 0.4, 0.4]] * n)
    pr = P.project(sc, cam)
    img = C.render(pr)
    c = 0.4 * Y00 + 0.5
    # float32 inputs round the logit and the coefficient at ~1e-7 relative;
    # including a fourth layer would change C by 1.2e-4 relative
    np.testing.assert_allclose(img["rgb"][8, 8], c * (1 - 0.05 ** 3), rtol=1e-7)
    np.testing.assert_allclose(img["T"][8, 8], 0.05 ** 3, rtol=1e-5)
    assert img["stopped"][8, 8]


def test_termination_stack_alpha_099_is_decision_ambiguous():
    """0.01^2 lands on 1e-4 exactly: the oracle must report a ~0 margin."""
    cam = axis_camera(w=16, h=16, f=16.0, cx=8.5, cy=8.5)
    n = 4
    sc = one_scene([[0, 0, 2.0 + 0.1 * i] for i in range(n)], [[-2] * 3] * n,
                   [[1, 0, 0, 0]] * n, [math.log(0.995 / 0.005)] * n, [[0.4, 0.4, 0.4]] * n)
    img = C.render(P.project(sc, cam))
    assert img["m_T"][8, 8] < 1e-9


def test_sh_orthonormal_by_quadrature():
    """Y_k are orthonormal on the sphere (Gauss-Legendre in cos t x uniform
    azimuth, exact for these polynomial degrees)."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    y = SH.sh_basis(d, 3)
    gram = (y * w[:, None]).T @ y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_known_values_and_order():
    """Index k = l^2 + l + m with the Condon-Shortley phase:
    Y_1^1(+x) = Y_1^-1(+y) = -sqrt(3/4pi), Y_1^0(+z) = +sqrt(3/4pi),
    Y_2^-2 = (1/2) sqrt(15/pi) x y, Y_2^0 = (1/4) sqrt(5/pi) (2z^2 - x^2 - y^2)."""
    c1 = math.sqrt(3 / (4 * math.pi))
    y = SH.sh_basis(np.eye(3), 1)
    np.testing.assert_allclose(y[0, 3], -c1, atol=1e-14)
    np.testing.assert_allclose(y[1, 1], -c1, atol=1e-14)
    np.testing.assert_allclose(y[2, 2], c1, atol=1e-14)
    np.testing.assert_allclose(y[:, 0], Y00, atol=1e-14)
    d = np.array([[0.48, 0.6, 0.64]])
    y2 = SH.sh_basis(d, 2)[0]
    x_, y_, z_ = d[0]
    np.testing.assert_allclose(y2[4], 0.5 * math.sqrt(15 / math.pi) * x_ * y_, atol=1e-13)
    np.testing.assert_allclose(y2[6], 0.25 * math.sqrt(5 / math.pi) * (2 * z_ * z_ - x_ * x_ - y_ * y_), atol=1e-13)


def test_sh_degree0_is_view_independent():
    sc, cam = _tiny_random()
    pr1 = P.project(sc, cam)
    cam2 = look_at((2.0, 1.0, 0.5), target=(0, 0, 2.5), width=16, height=16)
    pr2 = P.project(sc, cam2)
    np.testing.assert_allclose(pr1["rgb"], pr2["rgb"], atol=1e-15)


def test_depth_key_orders_like_depth():
    """Positive float32 bits sort as unsigned integers (Sec. 4.3) and the key
    is the float32 depth within a few ulp of the float64 one."""
    scene, cams = tiny_workload()
    pr = P.project(scene, cams[0])
    keys = pr["depth_key"]
    dep32 = keys.view(np.float32).astype(np.float64)
    assert np.all(np.abs(dep32 - pr["depth"]) <= 4 * np.spacing(np.float32(4.0)))
    o = np.argsort(keys, kind="stable")
    assert np.all(np.diff(dep32[o]) >= 0)


@pytest.mark.parametrize("shape", [(4, 4), (8, 4), (8, 8)])
@pytest.mark.parametrize("cap", [32, 256, 1024, 1 << 30])
def test_macro_batch_invariance(shape, cap):
    """Any macro-tile shape and batch cap gives the same image as the plain
    per-pixel definition (Sec. 3.1 decoupling + Eq. 1 + replay)."""
    scene, cams = tiny_workload()
    pr = P.project(scene, cams[0])
    ref = C.render(pr)
    rgb, t, replays = B.render_batched(pr, shape[0], shape[1], cap)
    assert np.abs(rgb - ref["rgb"]).max() < 1e-12
    assert np.abs(t - ref["T"]).max() < 1e-12
    if cap == 32:
        assert replays > 0  # the exact-termination replay path is exercised


def test_compose_is_associative():
    """Eq. 1 over contiguous depth ranges is associative (Porter-Duff over)."""
    g = np.random.default_rng(0)
    parts = [(g.uniform(0, 1, (5, 3)), g.uniform(0, 1, 5)) for _ in range(4)]
    full = B.compose(parts)
    left = B.compose([B.compose(parts[:2]), B.compose(parts[2:])])
    right = B.compose([parts[0], B.compose(parts[1:])])
    for a in (left, right):
        np.testing.assert_allclose(a[0], full[0], atol=1e-14)
        np.testing.assert_allclose(a[1], full[1], atol=1e-14)


def test_rect_contains_support():
    """Every pixel with q <= 9 lies inside [x0 - r, x0 + r] x [y0 - r, y0 + r]."""
    sc, cam = _tiny_random(n=200, w=48, h=48, seed=5)
    pr = P.project(sc, cam)
    ys, xs = np.mgrid[0:48, 0:48]
    for i in np.nonzero(pr["visible"])[0]:
        q, _ = C.alpha_at(pr, np.array([i]), xs.ravel().astype(float), ys.ravel().astype(float))
        inside = q[0] <= 9.0
        x0 = math.floor(pr["mean2d"][i, 0])
        y0 = math.floor(pr["mean2d"][i, 1])
        r = pr["radius"][i]
        xi, yi = xs.ravel()[inside], ys.ravel()[inside]
        assert np.all((xi >= x0 - r) & (xi <= x0 + r) & (yi >= y0 - r) & (yi <= y0 + r))


def test_binning_matches_pixel_enumeration():
    """Segment lists == (macro-tile, gaussian) pairs found by enumerating the
    pixels of each gaussian's rectangle, and each segment is ascending in
    (key, id) (Sec. 3.2-3.3)."""
    scene, cams = tiny_workload()
    pr = P.project(scene, cams[0])
    mx, my, r, key = BN.records_f32(pr)
    seg = BN.segments([(mx, my, r, key)], [(256, 256)], 64, 32)
    gw = 4
    want = set()
    for i in np.nonzero(r > 0)[0]:
        x0, y0 = math.floor(float(mx[i])), math.floor(float(my[i]))
        for y in range(max(0, y0 - r[i]), min(255, y0 + r[i]) + 1, 1):
            for x in range(max(0, x0 - r[i]), min(255, x0 + r[i]) + 1, 8):
                want.add(((y // 32) * gw + x // 64, i))
            xe = min(255, x0 + r[i])
            if xe >= max(0, x0 - r[i]):
                want.add(((y // 32) * gw + xe // 64, i))
    got = set()
    for s in range(seg["n_seg"]):
        a, b = seg["seg_off"][s], seg["seg_off"][s + 1]
        k, ids = seg["keys"][a:b], seg["ids"][a:b]
        assert np.all((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (ids[1:] > ids[:-1])))
        got.update((s, int(i)) for i in ids)
    assert got == want


def test_plain_tile_pairs_against_pixel_enumeration_and_candidates():
    """The plain path's per-tile pair list (Sec. 2 / 5 baseline) over two
    views: each tile's (gaussian) set equals the tiles met by enumerating the
    pixels of each gaussian's rectangle, every tile's list is ascending in
    (depth key, record) and equals the compositing oracle's own rect
    candidates (an independent expression of the same rule), record ids are
    v n + i, and the ranges cover exactly the pairs of each tile."""
    scene, cams = tiny_workload()
    cam2 = look_at((0.4, 3.0, 0.6), width=72, height=40)
    cams = [cams[0], cam2]
    prs = [P.project(scene, c) for c in cams]
    views = [BN.records_f32(p) for p in prs]
    keys64, ids, ranges = BN.plain_tile_pairs(views, [(c.width, c.height) for c in cams])
    n = scene.n
    tiles_v = [(-(-c.width // 8)) * (-(-c.height // 8)) for c in cams]
    assert len(ranges) == sum(tiles_v)
    assert np.all(keys64[1:] >= keys64[:-1])
    tile = (keys64 >> np.uint64(32)).astype(np.int64)
    key = (keys64 & np.uint64(0xffffffff)).astype(np.uint32)
    base = 0
    for v, (cam, pr) in enumerate(zip(cams, prs)):
        gw, gh, off, gid = C.tile_candidates(pr, 8)
        mx, my, r, k = views[v]
        want = set()
        for i in np.nonzero(r > 0)[0]:
            x0, y0 = math.floor(float(mx[i])), math.floor(float(my[i]))
            for y in range(max(0, y0 - r[i]), min(cam.height - 1, y0 + r[i]) + 1):
                for x in range(max(0, x0 - r[i]), min(cam.width - 1, x0 + r[i]) + 1):
                    want.add((base + (y // 8) * gw + x // 8, v * n + i))
        got = set()
        for t in range(gw * gh):
            a, b = ranges[base + t]
            assert np.all(tile[a:b] == base + t)
            got.update((base + t, int(i)) for i in ids[a:b])
            assert np.array_equal(ids[a:b] - v * n, gid[off[t]:off[t + 1]])
            assert np.array_equal(key[a:b], k[gid[off[t]:off[t + 1]]])
        assert got == want
        base += gw * gh
    assert sum(int(b - a) for a, b in ranges) == len(ids)


def test_macro_pairs_never_exceed_tile_pairs():
    """Coarser binning never creates more pairs (Table 1 ordering)."""
    scene, cams = tiny_workload()
    pr = P.project(scene, cams[0])
    mx, my, r, _ = BN.records_f32(pr)
    t8 = BN.tile_pair_count(mx, my, r, 256, 256, 8)
    for bw, bh in ((32, 32), (64, 32), (64, 64)):
        assert BN.rect_ranges(mx, my, r, 256, 256, bw, bh)[4].sum() <= t8


def test_batch_split_covers_segments():
    g = np.random.default_rng(1)
    n = g.integers(0, 5000, 50)
    off = np.concatenate([[0], np.cumsum(n)])
    for cap in (256, 1024, 2048):
        tab, first = BN.batches(off, cap)
        assert len(tab) == int(np.sum(-(-n // cap)))
        for s in range(len(n)):
            rows = tab[first[s]:first[s + 1]]
            assert np.all(rows[:, 0] == s)
            assert np.all(rows[:, 2] <= cap) and np.all(rows[:, 2] > 0)
            assert rows[:, 2].sum() == n[s]
            if len(rows):
                assert rows[0, 1] == off[s]
                assert np.all(rows[1:, 1] == rows[:-1, 1] + cap)


def test_paper_arithmetic_facts():
    facts = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
    t = facts["render_tile_px"]["value"]
    mw, mh = facts["macro_shape_tiles"]["value"]
    n1080 = np.prod(BN.grid_dims(1920, 1080, mw * t, mh * t))
    n4k = np.prod(BN.grid_dims(3840, 2160, mw * t, mh * t))
    assert n1080 == 1020 and abs(n1080 - facts["macro_tiles_1080p_approx"]["value"]) < 50
    assert n4k == 4080 and abs(n4k - facts["macro_tiles_4k_approx"]["value"]) < 100
    lo, hi = facts["render_tile_hist_range"]["value"]
    t1080 = np.prod(BN.grid_dims(1920, 1080, t, t))
    t4k = np.prod(BN.grid_dims(3840, 2160, t, t))
    assert (t1080, t4k) == (32400, 129600) and lo <= t1080 and t4k <= hi
    assert mw * mh * t * t * 4 * 2 == facts["slot_bytes_fp16"]["value"]
