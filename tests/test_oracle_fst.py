"""Pins of the FP64 oracle of the full FST deformation module (Sec. 3.2,
Eq. 4-6; Appendix A) against facts that do not come from the oracle itself:
central finite differences of its forward for every gradient, exact node
values of the bilinear HexPlane sampling, a closed form of the network with
permutation weights (a transposed or misplaced layer changes it), and the
total-variation term on planes with a known answer."""
import numpy as np
import pytest

from oracle import fst as F

LV, RS, RT, CC, DD = 2, 3, 4, 4, 3       # tiny: 2 levels, 3^3 x 4 grid, 4 channels, D = 3
LO, HI = np.array([-1.0, -1.0, 2.0]), np.array([1.0, 1.0, 4.0])


def _rand_params(seed, levels=LV, rs=RS, rt=RT, c=CC, D=DD, wscale=1.0):
    rng = np.random.default_rng(seed)
    planes = [rng.normal(1.0, 0.3, s) for s in F.plane_shapes(levels, rs, rt, c)]
    layers = [(rng.normal(0.0, wscale * np.sqrt(2.0 / i), (o, i)), rng.normal(0.0, 0.1, o))
              for o, i in F.layer_shapes(levels, D, c)]
    return planes, layers


def _loss(planes, layers, mu, t, r):
    out = F.forward(planes, layers, mu, t, LO, HI, LV, RS, RT)
    return (np.sum(r[0] * out["dmu"]) + np.sum(r[1] * out["dq"]) + np.sum(r[2] * out["ds"])
            + np.sum(r[3] * out["do"]) + np.sum(r[4] * out["dz"])), out


def _setup(seed=0, P=5):
    rng = np.random.default_rng(seed + 100)
    planes, layers = _rand_params(seed)
    mu = rng.uniform(LO + 0.1, HI - 0.1, (P, 3))
    r = [rng.normal(size=(P, 3)), rng.normal(size=(P, 4)), rng.normal(size=(P, 3)), rng.normal(size=P),
         rng.normal(size=(P, DD))]
    return planes, layers, mu, 0.37, r


def test_reverse_pass_matches_central_differences():
    planes, layers, mu, t, r = _setup()
    _, out = _loss(planes, layers, mu, t, r)
    st = out["state"]
    rel, cell = F.margins(st)
    assert rel.min() > 1e-6 and cell.min() > 1e-6   # no decision within reach of the step
    g = F.backward(planes, layers, st, *r)
    h = 1e-6
    rng = np.random.default_rng(7)
    checked = 0
    # Planes: nodes with a nonzero analytic gradient and a few zero ones.
    for k in rng.choice(len(planes), 8, replace=False):
        nz = np.argwhere(np.abs(g["planes"][k]) > 0)
        picks = [tuple(nz[i]) for i in rng.choice(len(nz), min(3, len(nz)), replace=False)] if len(nz) else []
        picks.append(tuple(rng.integers(0, s) for s in planes[k].shape))
        for idx in picks:
            old = planes[k][idx]
            planes[k][idx] = old + h
            lp, _ = _loss(planes, layers, mu, t, r)
            planes[k][idx] = old - h
            lm, _ = _loss(planes, layers, mu, t, r)
            planes[k][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g["planes"][k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx)
            checked += 1
    # Every layer: a few weights and one bias.
    for j, (w, b) in enumerate(layers):
        for _ in range(3):
            o, i = rng.integers(0, w.shape[0]), rng.integers(0, w.shape[1])
            old = w[o, i]
            w[o, i] = old + h
            lp, _ = _loss(planes, layers, mu, t, r)
            w[o, i] = old - h
            lm, _ = _loss(planes, layers, mu, t, r)
            w[o, i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g["layers"][j][0][o, i]) <= 1e-6 * max(1.0, abs(fd)), (j, o, i)
        o = rng.integers(0, b.shape[0])
        old = b[o]
        b[o] = old + h
        lp, _ = _loss(planes, layers, mu, t, r)
        b[o] = old - h
        lm, _ = _loss(planes, layers, mu, t, r)
        b[o] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g["layers"][j][1][o]) <= 1e-6 * max(1.0, abs(fd)), (j, "bias")
        checked += 4
    # The canonical mean through the HexPlane coordinates.
    for p in range(mu.shape[0]):
        for a in range(3):
            m = mu.copy()
            m[p, a] += h
            lp, _ = _loss(planes, layers, m, t, r)
            m[p, a] -= 2 * h
            lm, _ = _loss(planes, layers, m, t, r)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g["mu"][p, a]) <= 1e-6 * max(1.0, abs(fd)), (p, a)
    assert checked > 80


def test_clamped_coordinates_have_zero_mean_gradient():
    planes, layers, mu, t, r = _setup(seed=1, P=3)
    mu[0] = HI + 0.5            # outside the box on every axis: all positions clamp
    _, out = _loss(planes, layers, mu, t, r)
    g = F.backward(planes, layers, out["state"], *r)
    assert np.all(g["mu"][0] == 0.0) and np.any(g["mu"][1] != 0.0)


def test_bilinear_samples_are_exact_at_grid_nodes():
    rt = 5   # time nodes at t = 0, 1/4, ..., 1: every coordinate below is exact in binary64
    planes, layers = _rand_params(2, levels=1, rt=rt)
    # Node (i, j, k) of the 3^3 spatial grid and node m of the 5 time nodes.
    idx = [(0, 1, 2, 3), (2, 2, 0, 0), (1, 0, 1, 4)]
    mu = np.array([[LO[a] + (HI[a] - LO[a]) * n[a] / (RS - 1) for a in range(3)] for n in idx])
    ts = [n[3] / (rt - 1) for n in idx]
    for p, n in enumerate(idx):
        out = F.forward(planes, layers, mu[p:p + 1], ts[p], LO, HI, 1, RS, rt)
        want = np.ones(CC)
        for k, (a, b) in enumerate(F.PAIRS):
            want = want * planes[k][n[a], n[b]]
        assert np.array_equal(out["state"]["f"][0], want)


def test_second_level_doubles_the_spatial_resolution_only():
    """Level 1 samples a grid of 2 RS spatial nodes per axis and the same RT
    time nodes, and its features follow level 0's in f."""
    rt = 5
    planes, layers = _rand_params(4, levels=2, rt=rt)
    r1 = 2 * RS
    idx = [(0, 3, 5, 1), (4, 1, 2, 4)]
    mu = np.array([[LO[a] + (HI[a] - LO[a]) * n[a] / (r1 - 1) for a in range(3)] for n in idx])
    for p, n in enumerate(idx):
        out = F.forward(planes, layers, mu[p:p + 1], n[3] / (rt - 1), LO, HI, 2, RS, rt)
        want = np.ones(CC)
        for k, (a, b) in enumerate(F.PAIRS):
            assert planes[6 + k].shape[:2] == ((r1, rt)[a == 3], (r1, rt)[b == 3])
            want = want * planes[6 + k][n[a], n[b]]
        # mu / (r1 - 1) is not exact in binary64: the sample is the node value
        # up to a few ulps of the fraction.
        assert np.allclose(out["state"]["f"][0, CC:], want, rtol=1e-12, atol=0)


def _perm(rng, o, i):
    """A 0/1 selection matrix [o, i]: output r copies input sel[r]."""
    sel = rng.permutation(max(o, i))[:o] % i
    m = np.zeros((o, i))
    m[np.arange(o), sel] = 1.0
    return m, sel


def test_permutation_network_closed_form():
    """With selection weights, zero biases and positive planes every ReLU
    passes its input, so each output is one entry of f chosen by the
    composition of the selections; a transposed layer or a wrong branch or
    concatenation order selects another entry."""
    rng = np.random.default_rng(3)
    levels, c, D = 2, 32, 8
    planes = [rng.uniform(0.5, 1.5, s) for s in F.plane_shapes(levels, RS, RT, c)]
    layers, sels = [], []
    for o, i in F.layer_shapes(levels, D, c):
        m, s = _perm(rng, o, i)
        layers.append((m, np.zeros(o)))
        sels.append(s)
    mu = rng.uniform(LO + 0.1, HI - 0.1, (4, 3))
    out = F.forward(planes, layers, mu, 0.6, LO, HI, levels, RS, RT)
    f = out["state"]["f"]
    # h index -> f index through F_out
    h_src = np.arange(F.W)
    for j in range(F.DEPTH - 1, -1, -1):
        h_src = sels[j][h_src]
    names = ["dmu", "dq", "ds", "do"]
    hg_src = []
    for g in range(4):
        e1, e2, hd = sels[F.DEPTH + 3 * g:F.DEPTH + 3 * g + 3]
        hsrc_g = h_src[e1[e2]]               # h_g index -> f index
        hg_src.append(hsrc_g)
        want = f[:, hsrc_g[hd]]
        got = out[names[g]].reshape(len(mu), -1)
        assert np.array_equal(got, want), names[g]
    u_src = np.concatenate(hg_src)           # u = [h_mu, h_R, h_S, h_o]
    z1, z2 = sels[F.DEPTH + 12], sels[F.DEPTH + 13]
    assert np.array_equal(out["dz"], f[:, u_src[z1[z2]]])


def test_tv_loss_on_linear_ramps():
    """A plane that rises by s per node along its first axis and is constant
    along the second has TV = s^2 (mean of squared steps along the first
    axis, zero along the second); its gradient is 2 s / n at the last row,
    -2 s / n at the first and zero inside (n = number of steps)."""
    shapes = F.plane_shapes(1, 4, 5, 2)
    planes, slopes = [], []
    for k, (ra, rb, c) in enumerate(shapes):
        s = 0.1 * (k + 1)
        planes.append(np.broadcast_to((s * np.arange(ra))[:, None, None], (ra, rb, c)).copy())
        slopes.append(s)
    loss, grads = F.tv_loss(planes, 1)
    assert loss == pytest.approx(sum(s * s for s in slopes), rel=1e-12)
    for (ra, rb, c), s, g in zip(shapes, slopes, grads):
        n = (ra - 1) * rb * c
        assert np.allclose(g[0], -2 * s / n) and np.allclose(g[-1], 2 * s / n)
        assert np.allclose(g[1:-1], 0.0)


def test_tv_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    planes = [rng.normal(size=s) for s in F.plane_shapes(1, 3, 4, 2)]
    _, grads = F.tv_loss(planes, 1)
    h = 1e-6
    for k in range(6):
        idx = tuple(rng.integers(0, s) for s in planes[k].shape)
        old = planes[k][idx]
        planes[k][idx] = old + h
        lp, _ = F.tv_loss(planes, 1)
        planes[k][idx] = old - h
        lm, _ = F.tv_loss(planes, 1)
        planes[k][idx] = old
        assert abs((lp - lm) / (2 * h) - grads[k][idx]) < 1e-7
