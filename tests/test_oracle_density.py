"""Pins of the FP64 oracle of adaptive density control and of the oracle's
screen-space centre gradient: hand-built cases with known outcomes (keep,
clone, split along a known rotation, prune; output order; optimiser state),
the quaternion rotation against scipy, the opacity reset's closed form, and
the centre gradient against central differences of the rendered loss under a
shift of the principal point (which moves every projected centre by the same
amount and nothing else)."""
import dataclasses

import numpy as np
import pytest

from oracle import density as DN
from paper_2503_06161_gb300 import synth


def test_quaternion_rotation_matches_scipy():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(0)
    q = rng.normal(size=(50, 4))
    want = Rot.from_quat(np.c_[q[:, 1:], q[:, 0]]).as_matrix()   # scipy takes (x, y, z, w)
    assert np.allclose(DN.quat_to_rot(q), want, atol=1e-12)


def _case():
    ls_small, ls_big = np.log([0.01, 0.02, 0.015]), np.log([0.3, 0.1, 0.2])
    qz = np.array([np.cos(np.pi / 4), 0.0, 0.0, np.sin(np.pi / 4)])   # 90 degrees about z
    params = dict(
        means=np.array([[0, 0, 3], [1, 0, 3], [0, 1, 4], [1, 1, 4], [-1, 0, 5]], float),
        log_scales=np.array([ls_small, ls_small, ls_big, ls_big, ls_big]),
        quats=np.array([[1, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], qz]),
        opacity_logits=np.array([0.5, 0.5, 0.5, -8.0, 0.5]),
        feat=np.arange(10, dtype=float).reshape(5, 2))
    state = dict(m=np.arange(5, dtype=float) + 1.0)
    accum = np.array([0.0001, 0.003, 0.004, 0.004, 0.009])
    count = np.array([1, 3, 2, 2, 3])
    rng = np.random.default_rng(1)
    normals = rng.normal(size=(5, 2, 3))
    return params, state, accum, count, normals


def test_keep_clone_split_prune_and_order():
    params, state, accum, count, normals = _case()
    out, st, d = DN.densify(params, state, accum, count, normals, grad_thresh=0.0002, dense_scale=0.05,
                            min_opacity=0.005)
    # g0 low gradient: kept; g1 high & small: kept + cloned; g2 high & big:
    # split; g3 transparent: pruned; g4 high & big & rotated: split.
    assert d.tolist() == [0, 1, 2, -1, 2]
    assert out["means"].shape == (2 + 1 + 4, 3)
    assert np.array_equal(out["feat"][:3], params["feat"][[0, 1, 1]])
    assert np.array_equal(out["feat"][3:], params["feat"][[2, 2, 4, 4]])
    s2, s4 = np.exp(params["log_scales"][2]), np.exp(params["log_scales"][4])
    for i in range(2):
        # identity rotation: mu + s * n
        assert np.allclose(out["means"][3 + i], params["means"][2] + s2 * normals[2, i], atol=1e-14)
        # 90 degrees about z: (x, y, z) -> (-y, x, z)
        v = s4 * normals[4, i]
        assert np.allclose(out["means"][5 + i], params["means"][4] + np.array([-v[1], v[0], v[2]]), atol=1e-14)
    assert np.allclose(np.exp(out["log_scales"][3:5]), s2 / 1.6, rtol=1e-14)
    assert np.allclose(np.exp(out["log_scales"][5:7]), s4 / 1.6, rtol=1e-14)
    assert np.array_equal(out["quats"][5:7], np.stack([params["quats"][4]] * 2))
    assert st["m"].tolist() == [1.0, 2.0, 0.0, 0.0, 0.0, 0.0, 0.0]


def test_threshold_is_on_the_mean_over_views():
    params, state, accum, count, normals = _case()
    # g1's sum 0.003 over 3 views is 0.001 per view; raise the threshold past it
    _, _, d = DN.densify(params, state, accum, count, normals, grad_thresh=0.0011, dense_scale=0.05,
                         min_opacity=0.005)
    assert d[1] == 0 and d[2] == 2        # 0.004 / 2 = 0.002 still qualifies


def test_single_precision_decision_agrees_with_the_definition():
    """The f32 decision (thresholds mapped through logit and log) equals the
    FP64 definition wherever no input lies within float32 rounding of a
    threshold, and it flips exactly at the mapped thresholds."""
    rng = np.random.default_rng(5)
    P = 20000
    ls = rng.normal(np.log(0.03), 0.8, size=(P, 3)).astype(np.float32)
    logits = rng.normal(0.0, 4.0, size=P).astype(np.float32)
    cnt = rng.integers(0, 6, size=P)
    acc = (rng.exponential(2e-4, size=P) * cnt).astype(np.float32)
    args = (None, ls, None, logits, acc, cnt, 2e-4, 0.05, 0.005)
    d64 = DN.decide(*args)
    d32 = DN.decide(*args, precision="f32")
    avg = np.where(cnt > 0, acc.astype(float) / np.maximum(cnt, 1), 0.0)
    near = (np.abs(avg - 2e-4) < 1e-10) | (np.abs(ls.max(axis=1) - np.log(0.05)) < 1e-6) \
        | (np.abs(logits - np.log(0.005 / 0.995)) < 1e-5)
    assert near.sum() < P // 1000 and len(set(d64.tolist())) == 4
    assert np.array_equal(d32[~near], d64[~near])
    # exactly at the float32 thresholds
    lmin, ldense = np.float32(np.log(0.005 / 0.995)), np.float32(np.log(0.05))
    edge_logits = np.array([lmin, np.nextafter(lmin, np.float32(-np.inf))], np.float32)
    e = DN.decide(None, np.full((2, 3), -5.0, np.float32), None, edge_logits, np.zeros(2, np.float32), np.ones(2),
                  1.0, 0.05, 0.005, precision="f32")
    assert e.tolist() == [0, -1]
    edge_ls = np.array([[ldense] * 3, [np.nextafter(ldense, np.float32(np.inf))] * 3], np.float32)
    e = DN.decide(None, edge_ls, None, np.zeros(2, np.float32), np.ones(2, np.float32), np.ones(2), 1e-3, 0.05,
                  0.005, precision="f32")
    assert e.tolist() == [1, 2]


def test_screen_stats_and_opacity_reset_closed_forms():
    d_uv = np.array([[3.0, 4.0], [1.0, 0.0], [0.0, 0.0]])
    acc, cnt = DN.screen_grad_stats(d_uv, [True, False, True], width=2, height=2)   # W/2 = H/2 = 1
    assert acc.tolist() == [5.0, 0.0, 0.0] and cnt.tolist() == [1, 0, 1]
    acc, cnt = DN.screen_grad_stats(d_uv, [True, True, True], width=4, height=2, accum=acc, count=cnt)
    assert acc[0] == pytest.approx(5.0 + np.hypot(6.0, 4.0)) and acc[1] == 2.0 and cnt.tolist() == [2, 1, 2]
    lg = np.array([-10.0, 0.0, 3.0])
    cap = np.log(0.01 / 0.99)
    assert np.allclose(DN.reset_opacity(lg), [-10.0, cap, cap])


def test_centre_gradient_matches_a_principal_point_shift(oracle):
    """u = fx x / z + cx: shifting cx by h shifts every projected centre by
    h and changes nothing else, so dL/dcx = sum over Gaussians of dL/du."""
    P, D, W, H = 6, 4, 40, 32
    sc = synth.make_scene(P, D, (-0.6, -0.5, 2.0), (0.6, 0.5, 3.0), seed=3)
    cam = synth.make_camera(W, H, 50.0)
    rng = np.random.default_rng(2)
    g_rgb = rng.normal(size=(W * H, 3))
    g_feat = rng.normal(size=(W * H, D))

    def loss(c):
        r = oracle.render(sc, c)
        return float(np.sum(g_rgb * r["rgb"]) + np.sum(g_feat * r["feat"]))

    g = oracle.backward(sc, cam, g_rgb=g_rgb, g_feat=g_feat, want_uv=True)
    assert np.abs(g["uv"]).sum() > 0
    h = 1e-5
    for axis, name in ((0, "cx"), (1, "cy")):
        lp = loss(dataclasses.replace(cam, **{name: getattr(cam, name) + h}))
        lm = loss(dataclasses.replace(cam, **{name: getattr(cam, name) - h}))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g["uv"][:, axis].sum()) <= 1e-5 * max(1.0, abs(fd))
