"""Pins of the oracle's decision overrides (``render_alternatives`` and the
``flip`` / ``gflip`` arguments of ``backward``) against facts that do not
come from the override code itself.  CPU only.

The comparison protocol reads a decision whose FP64 margin is inside the
binary32 error model as having two correct outcomes (Sec. 3.3, Eq. 7-8 fix
the recurrence but not which side of a threshold a rounded evaluation lands
on).  Each pin builds a scene where one decision sits exactly on its
threshold, and checks that the other branch equals an independently
constructed render: the scene without the Gaussian that was skipped or left
out, the scene with two equal-depth Gaussians renumbered, or, for the
gradient-only decisions, the one-sided derivative taken from a scene moved
slightly to that side of the threshold."""
import numpy as np

from paper_2503_06161_gb300 import synth

W = H = 32
F = 40.0
Y00 = 0.5 / np.sqrt(np.pi)


def _cam():
    return synth.make_camera(W, H, F)   # cx = cy = 16, identity pose


def _scene(means, log_scales, logits, rgb, feat=None, D=4):
    P = len(means)
    sh = np.zeros((P, 16, 3))
    sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / Y00
    f = np.zeros((P, D)) if feat is None else np.asarray(feat, np.float64)
    return synth.Scene(np.asarray(means, np.float64), np.asarray(log_scales, np.float64),
                       np.tile([1.0, 0, 0, 0], (P, 1)), np.asarray(logits, np.float64), sh, f, sh_degree=0)


def _logit(o):
    return np.log(o / (1 - o))


def _sub(sc, idx):
    idx = np.asarray(idx)
    return synth.Scene(sc.means[idx], sc.log_scales[idx], sc.quats[idx], sc.opacity_logits[idx], sc.sh[idx],
                       sc.feat[idx], sc.sh_degree)


PIX = np.array([[16, 16]], np.int32)    # centre (16.5, 16.5)
Z = 2.0
X_AT_PIX = 0.5 * Z / F                  # projects to u = v = 16.5


def _same(a, b, tol=1e-13):
    return all(np.abs(np.asarray(a[k]) - np.asarray(b[k])).max() <= tol for k in ("rgb", "depth", "alpha", "feat"))


def _alts(oracle, sc, pix=PIX):
    a = oracle.render_alternatives(sc, _cam(), pixels=pix)
    return [dict(rgb=a["rgb"][0, k], depth=a["depth"][0, k], alpha=a["alpha"][0, k], feat=a["feat"][0, k],
                 flip=a["flip"][0, k]) for k in range(int(a["nalts"][0]))]


def _plain(oracle, sc, pix=PIX):
    r = oracle.render(sc, _cam(), pixels=pix, eps=None)
    return dict(rgb=r["rgb"][0], depth=r["depth"][0], alpha=r["alpha"][0], feat=r["feat"][0])


def test_fp64_branch_is_the_plain_render_and_clear_pixels_have_one(oracle):
    from tests.gpu_helpers import deformed_case
    sc, cam, df = deformed_case(P=1500, W=96, H=72, seed=7)
    r = oracle.render(sc, cam, df, t=0.4)
    pix = oracle.all_pixels(cam.width, cam.height)
    a = oracle.render_alternatives(sc, cam, df, t=0.4, pixels=pix)
    flagged = (r["flags"] & oracle.VALUE_FLAGS) != 0
    assert flagged.sum() > 20
    assert np.array_equal(a["rgb"][:, 0], r["rgb"]) and np.array_equal(a["feat"][:, 0], r["feat"])
    assert np.all(a["flip"][:, 0] == 0)
    assert np.all(a["nalts"][~flagged] == 1)
    assert np.all(a["nalts"][flagged] >= 2)


def test_skip_branch_is_the_scene_without_that_gaussian(oracle):
    # Gaussian 1 sits at the pixel centre with opacity 1/255 (1 + 2e-5): its
    # alpha is on the skip threshold.
    o = (1.0 / 255.0) * (1 + 2e-5)
    sc = _scene([[0.1, -0.1, 4.0], [X_AT_PIX, X_AT_PIX, Z]], [[-1.5] * 3, [-2.5] * 3], [0.3, _logit(o)],
                [[0.2, 0.4, 0.6], [0.9, 0.1, 0.5]], feat=[[1, 2, 3, 4], [-1, 0.5, 2, 0]])
    alts = _alts(oracle, sc)
    assert len(alts) == 2
    assert _same(alts[0], _plain(oracle, sc))
    assert _same(alts[1], _plain(oracle, _sub(sc, [0])))


def test_termination_branch_stops_before_the_second_gaussian(oracle):
    # Two clamped (alpha = 0.99) Gaussians at the pixel centre: T would fall
    # to 0.01 * 0.01 = 1e-4, the termination threshold.
    sc = _scene([[X_AT_PIX, X_AT_PIX, Z], [X_AT_PIX, X_AT_PIX, Z + 0.5]], [[-2.5] * 3] * 2, [_logit(0.995)] * 2,
                [[0.2, 0.4, 0.6], [0.9, 0.1, 0.5]], feat=[[1, 2, 3, 4], [-1, 0.5, 2, 0]])
    alts = _alts(oracle, sc)
    assert len(alts) == 2
    assert _same(alts[0], _plain(oracle, sc))
    assert _same(alts[1], _plain(oracle, _sub(sc, [0])))


def test_depth_tie_branch_is_the_renumbered_scene(oracle):
    # Equal depths: the FP64 order is by index; the other branch is the
    # order of the scene with the two Gaussians' indices exchanged.
    sc = _scene([[X_AT_PIX, X_AT_PIX, Z], [X_AT_PIX + 0.01, X_AT_PIX - 0.01, Z]], [[-2.5] * 3] * 2,
                [_logit(0.6), _logit(0.7)], [[0.2, 0.4, 0.6], [0.9, 0.1, 0.5]],
                feat=[[1, 2, 3, 4], [-1, 0.5, 2, 0]])
    alts = _alts(oracle, sc)
    assert len(alts) == 2
    assert _same(alts[0], _plain(oracle, sc))
    assert _same(alts[1], _plain(oracle, _sub(sc, [1, 0])))
    assert not _same(alts[0], alts[1], tol=1e-6)


def test_inclusion_branch_is_the_scene_with_or_without_the_gaussian(oracle):
    # An isotropic Gaussian of pixel variance 3.36 (radius ceil(3 sqrt(3.36 +
    # sqrt(0.1))) = 6) whose square edge passes through the pixel centre,
    # where its alpha is 0.99 exp(-36 / 6.72) ~ 0.0047 > 1/255.
    s = np.sqrt(3.36 - 0.3) * Z / F
    sc = _scene([[0.0, 0.3, 5.0], [X_AT_PIX + 6.0 * Z / F, X_AT_PIX, Z]], [[-1.0] * 3, [np.log(s)] * 3],
                [0.5, _logit(0.99)], [[0.2, 0.4, 0.6], [0.9, 0.1, 0.5]], feat=[[1, 2, 3, 4], [-1, 0.5, 2, 0]])
    g = oracle.gaussians(sc, _cam())
    assert g["radius"][1] == 6
    alts = _alts(oracle, sc)
    assert len(alts) == 2
    # Independent references: the scene with Gaussian 1 moved a hair inside
    # its square (the FP64 test then includes it; the move changes the
    # result by O(1e-9)) and the scene without it.
    inside = _scene(sc.means - np.array([[0, 0, 0], [1e-9, 0, 0]]), sc.log_scales, sc.opacity_logits,
                    [[0.2, 0.4, 0.6], [0.9, 0.1, 0.5]], feat=sc.feat)
    want = sorted([_plain(oracle, inside), _plain(oracle, _sub(sc, [0]))], key=lambda a: a["alpha"])
    got = sorted(alts, key=lambda a: a["alpha"])
    assert _same(got[0], want[0], tol=1e-7) and _same(got[1], want[1], tol=1e-7)
    assert abs(got[1]["alpha"] - got[0]["alpha"]) > 1e-3


def _grads(oracle, sc, cam, df=None, t=0.0, gflip=None, seed=0):
    pix = oracle.all_pixels(cam.width, cam.height)
    rng = np.random.default_rng(seed)
    n = len(pix)
    G = dict(g_rgb=rng.normal(size=(n, 3)), g_depth=rng.normal(size=n) * 0.1, g_alpha=rng.normal(size=n),
             g_feat=rng.normal(size=(n, sc.D)))
    return oracle.backward(sc, cam, df, t, (0, 0, 0), pix, gflip=gflip, **G)


def test_rgb_clamp_branches_are_the_one_sided_derivatives(oracle):
    # Red channel of Gaussian 0 exactly at the clamp (raw colour 0): the two
    # branches of its SH gradient equal the gradients of the scene with the
    # colour nudged to either side.
    cam = _cam()
    sc = _scene([[X_AT_PIX, X_AT_PIX, Z], [0.2, 0.1, 3.0]], [[-2.0] * 3, [-1.8] * 3], [0.4, -0.2],
                [[0.0, 0.4, 0.6], [0.9, 0.1, 0.5]], feat=[[1, 2, 3, 4], [-1, 0.5, 2, 0]])
    g = oracle.gaussians(sc, cam)
    assert g["gndec"][0] == 1 and g["gndec"][1] == 0
    b0 = _grads(oracle, sc, cam, gflip=np.array([0, 0], np.uint64))
    b1 = _grads(oracle, sc, cam, gflip=np.array([1, 0], np.uint64))
    sides = []
    for dc in (1e-7, -1e-7):
        s2 = _scene(sc.means, sc.log_scales, sc.opacity_logits, [[dc, 0.4, 0.6], [0.9, 0.1, 0.5]], feat=sc.feat)
        sides.append(_grads(oracle, s2, cam))
    got = sorted([b0["sh"][0, 0, 0], b1["sh"][0, 0, 0]])
    want = sorted([sides[0]["sh"][0, 0, 0], sides[1]["sh"][0, 0, 0]])
    assert min(abs(x) for x in got) == 0.0 and abs(max(got, key=abs)) > 1e-3
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-12)


def test_grid_cell_branches_are_the_one_sided_derivatives(oracle):
    # A deformed Gaussian whose x coordinate lies exactly on an interior
    # HexPlane node: the two branches of its mean gradient equal the
    # gradients with the mean moved a hair to either side of the node.
    rng = np.random.default_rng(3)
    cam = _cam()
    df = synth.make_deform(1, C=32, R=5, bbox_min=(-1, -1, 1), bbox_max=(1, 1, 3), full_heads=True, head_std=0.05,
                           seed=11, noise=False)
    df.planes[:] = rng.normal(1.0, 0.3, df.planes.shape)      # a rough field: distinct cell slopes
    sc = _scene([[0.0, 0.013, 2.017]], [[-2.3] * 3], [0.8], [[0.6, 0.4, 0.3]], feat=[[1, 2, 3, 4]])
    t = 0.37
    g = oracle.gaussians(sc, cam, df, t=t)
    assert g["gndec"][0] >= 1
    # The node decisions of the x coordinate (planes xy, xz, xt) come first
    # among the grid decisions; take them together.
    ncell = int(g["gndec"][0])
    b0 = _grads(oracle, sc, cam, df, t, gflip=np.array([0], np.uint64))
    b1 = _grads(oracle, sc, cam, df, t, gflip=np.array([(1 << ncell) - 1], np.uint64))
    # At +-1e-9 the x coordinate is still within the node's margin, but with
    # no override the reverse takes the cell on the side it lies.
    sides = []
    for dx in (1e-9, -1e-9):
        s2 = _scene(sc.means + np.array([[dx, 0, 0]]), sc.log_scales, sc.opacity_logits, [[0.6, 0.4, 0.3]],
                    feat=sc.feat)
        sides.append(_grads(oracle, s2, cam, df, t))
    got = sorted([b0["means"][0, 0], b1["means"][0, 0]])
    want = sorted([sides[0]["means"][0, 0], sides[1]["means"][0, 0]])
    assert abs(got[1] - got[0]) > 1e-3 * max(abs(got[1]), 1e-12)
    np.testing.assert_allclose(got, want, rtol=1e-5)
