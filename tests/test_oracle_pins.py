"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
closed forms of the paper's equations, invariants, library special cases,
brute force on tiny inputs and central finite differences.  CPU only."""
import dataclasses

import numpy as np
import pytest

from paper_2503_06161_gb300 import synth


def _one(mean, log_scale, quat, logit, rgb_dc=None, D=3, feat=None):
    """Single-Gaussian scene (SH degree 0 when rgb_dc is given)."""
    P = len(mean)
    sh = np.zeros((P, 16, 3), np.float64)
    if rgb_dc is not None:
        c0 = 0.5 / np.sqrt(np.pi)  # Y_00 = 1/(2 sqrt(pi))
        sh[:, 0, :] = (np.asarray(rgb_dc, np.float64) - 0.5) / c0
    f = np.zeros((P, D)) if feat is None else np.asarray(feat, np.float64)
    return synth.Scene(np.asarray(mean, np.float64), np.asarray(log_scale, np.float64),
                       np.asarray(quat, np.float64), np.asarray(logit, np.float64), sh, f, sh_degree=0)


def _logit(o):
    return np.log(o / (1 - o))


# --------------------------------------------------------------------------
# Spherical harmonics (colour from SH, Sec. 3.1)
# --------------------------------------------------------------------------

def _scipy_real_sh(l, m, theta, phi):
    """Real SH keeping scipy's Condon-Shortley phase: sqrt2 Re/Im of Y_l^|m|."""
    import scipy.special as sp
    mm = abs(m)
    if hasattr(sp, "sph_harm_y"):
        Y = sp.sph_harm_y(l, mm, theta, phi)   # theta polar, phi azimuth
    else:  # older scipy
        Y = sp.sph_harm(mm, l, phi, theta)
    if m == 0:
        return Y.real
    return np.sqrt(2) * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_scipy(oracle):
    rng = np.random.default_rng(3)
    d = rng.normal(size=(1000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, _ = oracle.sh_eval(d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _scipy_real_sh(l, m, theta, phi)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12, err_msg=f"l={l} m={m}")


def test_sh_gradient_by_finite_differences(oracle):
    rng = np.random.default_rng(4)
    d = rng.normal(size=(50, 3))
    _, dY = oracle.sh_eval(d)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Yp, _ = oracle.sh_eval(d + e)
        Ym, _ = oracle.sh_eval(d - e)
        np.testing.assert_allclose(dY[:, :, a], (Yp - Ym) / (2 * h), atol=1e-7)


def test_sh_degree0_is_constant_colour(oracle):
    cam = synth.make_camera(32, 32, 40.0)
    rng = np.random.default_rng(0)
    P = 64
    mean = np.c_[rng.uniform(-1, 1, (P, 2)), rng.uniform(2, 4, P)]
    sc = _one(mean, np.full((P, 3), -2.0), np.tile([1, 0, 0, 0.], (P, 1)), np.zeros(P), rgb_dc=[0.2, 0.5, 0.9])
    g = oracle.gaussians(sc, cam)
    np.testing.assert_allclose(g["rgb"], np.tile([0.2, 0.5, 0.9], (P, 1)), atol=1e-14)


# --------------------------------------------------------------------------
# Closed forms of Eq. 1-2, 7-9
# --------------------------------------------------------------------------

def _cam(W=64, H=48, f=80.0):
    return synth.make_camera(W, H, f)


def test_alpha_at_centre_equals_opacity(oracle):
    cam = _cam()
    Z = 3.0
    x, y = 20, 17  # pixel whose centre the Gaussian projects to
    X = (x + 0.5 - cam.cx) * Z / cam.fx
    Yw = (y + 0.5 - cam.cy) * Z / cam.fy
    o = 0.7
    feat = np.array([[1.5, -2.0, 0.25]])
    sc = _one([[X, Yw, Z]], [[-2.5] * 3], [[0.3, 0.1, -0.5, 0.8]], [_logit(o)], rgb_dc=[0.1, 0.6, 0.3], feat=feat)
    bg = (0.2, 0.3, 0.4)
    r = oracle.render(sc, cam, bg=bg, pixels=[[x, y]])
    assert r["alpha"][0] == pytest.approx(o, abs=1e-12)
    np.testing.assert_allclose(r["rgb"][0], o * np.array([0.1, 0.6, 0.3]) + (1 - o) * np.array(bg), atol=1e-12)
    assert r["depth"][0] == pytest.approx(o * Z, abs=1e-12)
    np.testing.assert_allclose(r["feat"][0], o * feat[0], atol=1e-12)


def _sigma2(f, s, Z):
    return (f * s / Z) ** 2 + 0.3


@pytest.mark.parametrize("quat", [[1, 0, 0, 0], [0.2, 0.7, -0.1, 0.4]])
def test_isotropic_profile(oracle, quat):
    cam = _cam(W=48, H=48, f=60.0)
    Z, s, o = 4.0, np.exp(-2.2), 0.8
    sc = _one([[0.0, 0.0, Z]], [[np.log(s)] * 3], [quat], [_logit(o)], rgb_dc=[1, 1, 1])
    pix = oracle.all_pixels(cam.width, cam.height)
    r = oracle.render(sc, cam, pixels=pix)
    s2 = _sigma2(cam.fx, s, Z)
    d2 = (pix[:, 0] + 0.5 - cam.cx) ** 2 + (pix[:, 1] + 0.5 - cam.cy) ** 2
    alpha = np.minimum(0.99, o * np.exp(-0.5 * d2 / s2))
    lam = s2  # isotropic: both eigenvalues equal; radius uses max(0.1, ...) = 0.1
    r_px = np.ceil(3 * np.sqrt(lam + np.sqrt(0.1)))
    inside = (np.abs(pix[:, 0] + 0.5 - cam.cx) <= r_px) & (np.abs(pix[:, 1] + 0.5 - cam.cy) <= r_px)
    expect = np.where(inside & (alpha >= 1 / 255), alpha, 0.0)
    np.testing.assert_allclose(r["alpha"], expect, atol=1e-12)


def test_anisotropic_axis_aligned_and_rotation(oracle):
    cam = _cam(W=64, H=64, f=70.0)
    Z, o = 3.5, 0.6
    sx, sy = np.exp(-1.8), np.exp(-2.6)
    pix = oracle.all_pixels(cam.width, cam.height)
    dx = pix[:, 0] + 0.5 - cam.cx
    dy = pix[:, 1] + 0.5 - cam.cy
    for quat, (ax, ay) in [([1, 0, 0, 0], (sx, sy)),
                           ([np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)], (sy, sx))]:  # 90 deg about z swaps
        sc = _one([[0.0, 0.0, Z]], [[np.log(sx), np.log(sy), -3.0]], [quat], [_logit(o)], rgb_dc=[1, 1, 1])
        r = oracle.render(sc, cam, pixels=pix)
        vx, vy = _sigma2(cam.fx, ax, Z), _sigma2(cam.fy, ay, Z)
        alpha = o * np.exp(-0.5 * (dx * dx / vx + dy * dy / vy))
        mid = 0.5 * (vx + vy)
        lam = mid + np.sqrt(max(0.1, mid * mid - vx * vy))
        rr = np.ceil(3 * np.sqrt(lam))
        inside = (np.abs(dx) <= rr) & (np.abs(dy) <= rr)
        expect = np.where(inside & (alpha >= 1 / 255), alpha, 0.0)
        np.testing.assert_allclose(r["alpha"], expect, atol=1e-12)


def test_off_axis_jacobian_closed_form(oracle):
    # Isotropic Sigma = s^2 I off-axis: Sigma' = s^2 J J^T + 0.3 I with
    # J J^T = f^2/Z^2 [[1 + x^2/Z^2, xy/Z^2], [xy/Z^2, 1 + y^2/Z^2]].
    cam = _cam(W=64, H=64, f=50.0)
    pts = np.array([[0.6, -0.4, 3.0], [-1.0, 0.9, 4.0], [0.2, 0.3, 2.5]])
    s = np.exp(-2.0)
    P = len(pts)
    sc = _one(pts, np.full((P, 3), np.log(s)), np.tile([1, 0, 0, 0.], (P, 1)), np.zeros(P))
    g = oracle.gaussians(sc, cam)
    for i, (x, y, Z) in enumerate(pts):
        JJ = cam.fx ** 2 / Z ** 2 * np.array([[1 + x * x / Z ** 2, x * y / Z ** 2], [x * y / Z ** 2, 1 + y * y / Z ** 2]])
        S = s * s * JJ + 0.3 * np.eye(2)
        Mi = np.linalg.inv(S)
        np.testing.assert_allclose(g["conic"][i], [Mi[0, 0], Mi[0, 1], Mi[1, 1]], rtol=1e-12)
        np.testing.assert_allclose(g["uv"][i], [cam.fx * x / Z + cam.cx, cam.fy * y / Z + cam.cy], rtol=1e-14)
        assert g["depth"][i] == Z


def test_camera_pose_moves_centre(oracle):
    # World->camera transform: a pure translation t shifts camera coordinates
    # by t, and the view direction for colour is taken from the camera centre.
    cam0 = _cam()
    t = np.array([0.3, -0.2, 0.5])
    cam1 = synth.make_camera(cam0.width, cam0.height, cam0.fx, translation=t)
    P = 5
    rng = np.random.default_rng(2)
    mean = np.c_[rng.uniform(-0.5, 0.5, (P, 2)), rng.uniform(2, 3, P)]
    sc = dataclasses.replace(synth.make_scene(P, 2, (-1, -1, 2), (1, 1, 3), seed=1), means=mean)
    sc1 = dataclasses.replace(sc, means=mean - t)
    g0 = oracle.gaussians(sc, cam0)
    g1 = oracle.gaussians(sc1, cam1)
    np.testing.assert_allclose(g1["uv"], g0["uv"], rtol=1e-6)  # translation only: means moved by -t
    np.testing.assert_allclose(g1["depth"], g0["depth"], rtol=1e-6)
    np.testing.assert_allclose(g1["rgb"], g0["rgb"], atol=1e-6)


def test_termination_and_skip(oracle):
    cam = _cam(W=32, H=32, f=40.0)
    x, y = 10, 12
    Zs = [2.0, 2.5, 3.0, 3.5, 4.0]
    means = [[(x + 0.5 - cam.cx) * Z / cam.fx, (y + 0.5 - cam.cy) * Z / cam.fy, Z] for Z in Zs]
    o = 0.95
    cols = [[0.1, 0.2, 0.3], [0.9, 0.1, 0.4], [0.5, 0.5, 0.5], [1.0, 0.0, 1.0], [0.3, 0.3, 0.1]]
    sc = _one(means, np.full((5, 3), -1.0), np.tile([1, 0, 0, 0.], (5, 1)), np.full(5, _logit(o)),
              rgb_dc=None)
    c0 = 0.5 / np.sqrt(np.pi)
    sc.sh[:, 0, :] = (np.asarray(cols) - 0.5) / c0
    r = oracle.render(sc, cam, pixels=[[x, y]])
    # T: 1, 0.05, 0.0025, 1.25e-4; the 4th would take T to 6.25e-6 < 1e-4: stop.
    T = [1.0, 0.05, 0.0025]
    expect = sum(o * T[k] * np.asarray(cols[k]) for k in range(3))
    np.testing.assert_allclose(r["rgb"][0], expect, atol=1e-12)
    assert r["ncontrib"][0] == 3
    assert r["alpha"][0] == pytest.approx(1 - 1.25e-4, abs=1e-15)
    # A Gaussian below 1/255 is skipped entirely.
    sc2 = _one(means[:1], [[-1.0] * 3], [[1, 0, 0, 0]], [_logit(0.003)], rgb_dc=[1, 1, 1])
    r2 = oracle.render(sc2, cam, pixels=[[x, y]])
    assert r2["alpha"][0] == 0.0 and r2["ncontrib"][0] == 0


def test_weights_plus_transmittance_is_one(oracle):
    sc, cam, _ = synth.config_inputs("static_1k_64x64")
    r = oracle.render(sc, cam)
    np.testing.assert_allclose(r["sumw"] + (1 - r["alpha"]), 1.0, atol=1e-12)
    assert r["ncontrib"].max() > 5


def test_background_adds_transmittance(oracle):
    sc, cam, _ = synth.config_inputs("static_1k_64x64", P=300)
    bg = np.array([0.2, 0.3, 0.4])
    r0 = oracle.render(sc, cam)
    r1 = oracle.render(sc, cam, bg=bg)
    np.testing.assert_allclose(r1["rgb"] - r0["rgb"], (1 - r0["alpha"])[:, None] * bg, atol=1e-12)


def _permuted(scene, deform, perm):
    sc = synth.Scene(scene.means[perm], scene.log_scales[perm], scene.quats[perm],
                     scene.opacity_logits[perm], scene.sh[perm], scene.feat[perm], scene.sh_degree)
    df = None
    if deform is not None:
        df = dataclasses.replace(deform, noise=deform.noise[perm])
    return sc, df


def test_order_invariance(oracle):
    P = 400
    sc, cam, _ = synth.config_inputs("static_1k_64x64", P=P)
    df = synth.make_deform(P, C=8, R=8, bbox_min=(-1, -1, 2), bbox_max=(1, 1, 4), full_heads=True, head_std=0.05)
    perm = np.random.default_rng(9).permutation(P)
    sc2, df2 = _permuted(sc, df, perm)
    r1 = oracle.render(sc, cam, df, t=0.4)
    r2 = oracle.render(sc2, cam, df2, t=0.4)
    for k in ("rgb", "depth", "alpha", "feat"):
        assert np.array_equal(r1[k], r2[k]), k


# --------------------------------------------------------------------------
# Deformation (Sec. 3.2, Eq. 4-6; Appendix A)
# --------------------------------------------------------------------------

def _affine_planes(R, C, rng):
    """Plane k channel c holds a_kc + b_kc*i + c_kc*j: bilinear interpolation
    reproduces it exactly at any grid position (i, j)."""
    A = rng.uniform(0.5, 1.5, (6, C))
    B = rng.uniform(-0.02, 0.02, (6, C))
    Cc = rng.uniform(-0.02, 0.02, (6, C))
    i = np.arange(R)[:, None, None]
    j = np.arange(R)[None, :, None]
    planes = np.stack([A[k] + B[k] * i + Cc[k] * j for k in range(6)])
    return planes, A, B, Cc


def test_hexplane_affine_planes_exact(oracle):
    rng = np.random.default_rng(5)
    R, C = 9, 4
    planes, A, B, Cc = _affine_planes(R, C, rng)
    bmin, bmax = np.array([-2.0, -1.0, 3.0]), np.array([2.0, 1.0, 8.0])
    df = synth.Deform(planes, np.zeros((64, C)), np.zeros(64), np.zeros((64, 64)), np.zeros(64),
                      np.zeros((11, 64)), np.zeros(11), bmin, bmax, None)
    mu = bmin + (bmax - bmin) * rng.random((40, 3))
    t = 0.3
    f, _ = oracle.deform_eval(df, mu, t)
    # Grid position of a coordinate: corners of the grid at -1 and +1.
    coord = np.c_[2 * (mu - bmin) / (bmax - bmin) - 1, np.full(len(mu), 2 * t - 1)]
    gpos = (coord + 1) / 2 * (R - 1)
    pairs = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]
    expect = np.ones((len(mu), C))
    for k, (a, b) in enumerate(pairs):
        expect *= A[k] + B[k] * gpos[:, a:a + 1] + Cc[k] * gpos[:, b:b + 1]
    np.testing.assert_allclose(f, expect, rtol=1e-13)


def test_hexplane_node_values_and_clamp(oracle):
    rng = np.random.default_rng(6)
    R, C = 5, 3
    planes = rng.uniform(0.5, 1.5, (6, R, R, C))
    bmin, bmax = np.array([0.0, 0.0, 0.0]), np.array([4.0, 4.0, 4.0])  # node spacing 1
    df = synth.Deform(planes, np.zeros((64, C)), np.zeros(64), np.zeros((64, 64)), np.zeros(64),
                      np.zeros((11, 64)), np.zeros(11), bmin, bmax, None)
    nodes = np.array([[1.0, 3.0, 2.0], [0.0, 4.0, 4.0], [2.0, 2.0, 0.0]])
    t = 0.25  # -> grid position 1
    f, _ = oracle.deform_eval(df, nodes, t)
    it = 1
    for n, (x, y, z) in enumerate(nodes.astype(int)):
        idx = [(x, y), (x, z), (y, z), (x, it), (y, it), (z, it)]
        expect = np.prod([planes[k, i, j] for k, (i, j) in enumerate(idx)], axis=0)
        np.testing.assert_allclose(f[n], expect, rtol=1e-14)
    # Outside the box the position clamps to the border.
    fo, _ = oracle.deform_eval(df, np.array([[-3.0, 7.0, 2.0]]), t)
    fc, _ = oracle.deform_eval(df, np.array([[0.0, 4.0, 2.0]]), t)
    np.testing.assert_allclose(fo, fc, rtol=1e-15)


def test_mlp_wiring_permutation(oracle):
    # W1 = rows of a permutation, W2 = identity, head row k picks hidden unit
    # p(k): delta_k = f_{sigma(k)}; a transposed operand or a wrong index fails.
    rng = np.random.default_rng(7)
    R, C = 4, 8
    planes = rng.uniform(0.8, 1.2, (6, R, R, C))
    perm1 = rng.permutation(64)
    w1 = np.zeros((64, C))
    for o in range(64):
        if perm1[o] < C:
            w1[o, perm1[o]] = 1.0
    w2 = np.eye(64)
    wh = np.zeros((11, 64))
    pick = {}
    for k in range(11):
        o = int(np.where(perm1 == (k % C))[0][0])
        wh[k, o] = 1.0
        pick[k] = k % C
    bh = np.arange(11) * 0.01
    df = synth.Deform(planes, w1, np.zeros(64), w2, np.zeros(64), wh, bh, np.array([-1.0] * 3),
                      np.array([1.0] * 3), None)
    mu = rng.uniform(-1, 1, (10, 3))
    f, delta = oracle.deform_eval(df, mu, 0.5)
    for k in range(11):
        np.testing.assert_allclose(delta[:, k], f[:, pick[k]] + bh[k], rtol=1e-14)
    # A negative first-layer bias switches every unit off (ReLU): heads give bh.
    df2 = dataclasses.replace(df, b1=np.full(64, -10.0))
    _, delta2 = oracle.deform_eval(df2, mu, 0.5)
    np.testing.assert_allclose(delta2, np.tile(bh, (10, 1)), atol=0)


def test_zero_heads_reduce_to_static_render(oracle):
    P = 300
    sc, cam, _ = synth.config_inputs("static_1k_64x64", P=P)
    df = synth.make_deform(P, C=8, R=8, bbox_min=(-1, -1, 2), bbox_max=(1, 1, 4), noise=False)
    df = dataclasses.replace(df, wh=np.zeros_like(df.wh), bh=np.zeros_like(df.bh))
    r0 = oracle.render(sc, cam)
    r1 = oracle.render(sc, cam, df, t=0.7)
    for k in ("rgb", "depth", "alpha", "feat"):
        assert np.array_equal(r0[k], r1[k]), k


def test_noise_term_is_linear_in_t(oracle):
    P = 50
    sc, cam, _ = synth.config_inputs("static_1k_64x64", P=P)
    df = synth.make_deform(P, C=8, R=8, bbox_min=(-1, -1, 2), bbox_max=(1, 1, 4), noise=True)
    df = dataclasses.replace(df, wh=np.zeros_like(df.wh))
    for t in (0.0, 0.5, 1.0):
        g = oracle.gaussians(sc, cam, df, t=t)
        np.testing.assert_allclose(g["delta"][:, :3], df.noise_scale * t * df.noise, rtol=1e-6, atol=1e-12)


# --------------------------------------------------------------------------
# Integer stage: tile lists vs a pixel-level brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tw,th", [(16, 16), (8, 32), (32, 8)])
def test_tile_bin_matches_pixel_bruteforce(oracle, tw, th):
    rng = np.random.default_rng(11)
    W, H, P = 70, 50, 300
    uv = np.c_[rng.uniform(-15, W + 15, P), rng.uniform(-15, H + 15, P)].astype(np.float32)
    radius = rng.integers(0, 12, P).astype(np.int32)
    depth = rng.uniform(1, 5, P).astype(np.float32)
    depth[10:20] = depth[10]  # exact ties: broken by index
    # Keep clear of binary32 rounding at the rect edges (where the two
    # formulations could differ by one ulp).
    frac = np.abs(np.r_[uv[:, 0] - radius - 0.5, uv[:, 1] - radius - 0.5, uv[:, 0] + radius - 0.5,
                        uv[:, 1] + radius - 0.5] % 1.0)
    assert np.min(np.minimum(frac, 1 - frac)) > 1e-4
    keys, vals, ranges = oracle.tile_bin(uv, radius, depth, W, H, tw, th)
    tx_n, ty_n = (W + tw - 1) // tw, (H + th - 1) // th
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    u64 = uv.astype(np.float64)
    expect_tiles = []
    for ty in range(ty_n):
        for tx in range(tx_n):
            px = xs[tx * tw:(tx + 1) * tw]
            py = ys[ty * th:(ty + 1) * th]
            members = []
            for g in range(P):
                if radius[g] <= 0:
                    continue
                okx = np.any(np.abs(px - u64[g, 0]) <= radius[g])
                oky = np.any(np.abs(py - u64[g, 1]) <= radius[g])
                if okx and oky:
                    members.append(g)
            members.sort(key=lambda g: (depth[g].view(np.uint32), g))
            expect_tiles.append(members)
    got = [vals[ranges[t, 0]:ranges[t, 1]].tolist() for t in range(tx_n * ty_n)]
    assert got == expect_tiles
    # Keys carry (tile, depth bits).
    tile_of = keys >> np.uint64(32)
    for t in range(tx_n * ty_n):
        assert np.all(tile_of[ranges[t, 0]:ranges[t, 1]] == t)
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), depth[vals].view(np.uint32))


# --------------------------------------------------------------------------
# Analytic reverse pass vs central finite differences
# --------------------------------------------------------------------------

def _tiny(deform: bool, seed=0, P=10, D=4):
    rng = np.random.default_rng(seed)
    cam = synth.make_camera(20, 16, 18.0, rotation=synth.random_rotation(rng, 0.1),
                            translation=[0.05, -0.03, 0.1])
    sc = synth.make_scene(P, D, (-0.8, -0.6, 2.0), (0.8, 0.6, 3.0), seed=seed)
    sc = dataclasses.replace(sc, log_scales=sc.log_scales + 1.2)  # a few px wide at this focal length
    df = None
    if deform:
        df = synth.make_deform(P, C=6, R=6, bbox_min=(-1, -1, 1.5), bbox_max=(1, 1, 3.5), full_heads=True,
                               head_std=0.05, seed=seed + 1)
    return sc, cam, df


def _loss(oracle, sc, cam, df, t, bg, pix, G):
    r = oracle.render(sc, cam, df, t=t, bg=bg, pixels=pix, eps=None)
    L = (G["rgb"] * r["rgb"]).sum() + (G["depth"] * r["depth"]).sum() + (G["alpha"] * r["alpha"]).sum() \
        + (G["feat"] * r["feat"]).sum()
    return L, r["sig"]


@pytest.mark.parametrize("deform", [False, True])
def test_backward_matches_central_differences(oracle, deform):
    sc, cam, df = _tiny(deform)
    t = 0.35
    bg = (0.1, 0.2, 0.3)
    pix = oracle.all_pixels(cam.width, cam.height)
    n = len(pix)
    rng = np.random.default_rng(1)
    G = dict(rgb=rng.normal(size=(n, 3)), depth=rng.normal(size=n) * 0.1, alpha=rng.normal(size=n),
             feat=rng.normal(size=(n, sc.D)))
    grads = oracle.backward(sc, cam, df, t, bg, pix, G["rgb"], G["depth"], G["alpha"], G["feat"])
    base_L, base_sig = _loss(oracle, sc, cam, df, t, bg, pix, G)
    checked = 0
    worst = 0.0
    for name, arr in [("means", sc.means), ("log_scales", sc.log_scales), ("quats", sc.quats),
                      ("opacity_logits", sc.opacity_logits), ("sh", sc.sh), ("feat", sc.feat)]:
        ref = grads[name]
        scale = max(np.sqrt(np.mean(ref ** 2)), 1e-12)
        flat = np.asarray(arr, np.float64).reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals = []
            sigs_ok = True
            for s in (+1, -1):
                x = flat.copy()
                x[i] += s * h
                sc2 = dataclasses.replace(sc, **{name: x.reshape(np.shape(arr))})
                L, sig = _loss(oracle, sc2, cam, df, t, bg, pix, G)
                sigs_ok &= bool(np.array_equal(sig, base_sig))
                vals.append(L)
            if not sigs_ok:
                continue  # a discrete decision flipped: FD is not a derivative here
            fd = (vals[0] - vals[1]) / (2 * h)
            an = ref.reshape(-1)[i]
            err = abs(fd - an) / max(abs(fd), scale)
            worst = max(worst, err)
            assert err < 1e-4, (name, i, an, fd)
            checked += 1
    assert checked > 300
    assert worst < 1e-4


def test_deformation_gradient_reaches_means(oracle):
    # With only the grid path active (no direct path), the mean gradient must
    # equal the FD of the loss through the HexPlane grid: isolate it by
    # checking that the deformed and static gradients differ.
    sc, cam, df = _tiny(True, seed=3)
    pix = oracle.all_pixels(cam.width, cam.height)
    n = len(pix)
    g = np.ones((n, 3))
    a = oracle.backward(sc, cam, df, 0.5, (0, 0, 0), pix, g_rgb=g)
    b = oracle.backward(sc, cam, None, 0.5, (0, 0, 0), pix, g_rgb=g)
    assert np.abs(a["means"] - b["means"]).max() > 1e-6


# --------------------------------------------------------------------------
# Decoder, L1 and Adam oracles vs library routines
# --------------------------------------------------------------------------

def test_decoder_matches_conv2d_and_autograd(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    H, W, D, Co = 6, 7, 8, 16
    f = rng.normal(size=(H * W, D))
    w = rng.normal(size=(Co, D)) * 0.1
    b = rng.normal(size=Co)
    tgt = rng.normal(size=(H * W, Co))
    out = oracle.decoder_forward(f, w, b)
    ft = torch.tensor(f.T.reshape(1, D, H, W), dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(w.reshape(Co, D, 1, 1), dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    ot = torch.nn.functional.conv2d(ft, wt, bt)
    np.testing.assert_allclose(out, ot.detach().numpy().reshape(Co, H * W).T, rtol=1e-12)
    tt = torch.tensor(tgt.T.reshape(1, Co, H, W), dtype=torch.float64)
    loss_t = (ot - tt).abs().sum(1).mean()
    loss_t.backward()
    loss, dout = oracle.l1_loss_and_grad(out, tgt)
    assert loss == pytest.approx(loss_t.item(), rel=1e-12)
    df_, dw, db = oracle.decoder_backward(f, w, dout)
    np.testing.assert_allclose(df_, ft.grad.numpy().reshape(D, H * W).T, rtol=1e-10)
    np.testing.assert_allclose(dw, wt.grad.numpy().reshape(Co, D), rtol=1e-10)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-10)


def test_adam_matches_torch(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    p = rng.normal(size=50)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 4):
        g = rng.normal(size=50)
        pt.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, step, 1e-2)
        np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12)
