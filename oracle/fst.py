"""FP64 oracle of the full FST deformation module (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module; the
product path never touches it and it imports nothing from the product
package.

What it computes, by passage of arXiv 2503.06161 (FeatureEndo-4DGS):
  * Multi-resolution HexPlane encoding of (mu, t) (Sec. 3.2; Appendix A:
    grid dimension 2, input dimension 4, 32 output channels, base
    resolution [64, 64, 64, 100], levels [1, 2, 4, 8]).
  * The HexPlane decoder MLP F_out, width W = 64 and depth 8 (Appendix A),
    giving h (Sec. 3.2).
  * Four branches g in {mu, R, S, o}: a feature extractor of two linear
    layers down to W/2 and a head of output size d_g = 3, 4, 3, 1 (Eq. 4;
    Appendix A).
  * The semantic updater F_feat of two linear layers on the concatenated
    branch features, giving dz in R^D (Eq. 5; Appendix A).
  * The hand-derived reverse pass of all of the above: gradients of the
    planes, of every weight and bias, and of the canonical mean through the
    HexPlane coordinates.

Readings where the paper is silent (restated at each use below):
  * Levels scale the three spatial resolutions only (64 * 2^l); the time
    resolution stays 100.  Features of the levels are concatenated
    (f in R^{L*C}); within a level the six plane samples are multiplied
    channel by channel.
  * Coordinates: mu normalised to [-1, 1] by the scene box, t in [0, 1]
    mapped to [-1, 1]; grid corners at +-1 (align-corners); positions
    clamped to the border (a clamped coordinate has zero gradient).
  * Layer order: F_out is Linear(L*C -> W) then seven blocks of
    ReLU -> Linear(W -> W); every later layer applies ReLU to its input
    first: extractor ReLU -> Linear(W -> W/2), ReLU -> Linear(W/2 -> W/2)
    giving h_g; head ReLU -> Linear(W/2 -> d_g); F_feat ReLU ->
    Linear(4 * W/2 -> W), ReLU -> Linear(W -> D).  The paper writes
    u_all in R^{4W}; with extractors that end at W/2 it has 4 * W/2 = 2W
    entries.
  * ReLU'(0) = 0 (the gradient passes where the input is > 0).

Parameter layout (the interface shared with the library, restated here):
planes level-major then plane-major (xy, xz, yz, xt, yt, zt), each
[R_a, R_b, C] channels-last; the MLP as one flat float array in the order
F_out (W [W, L*C], b [W]; 7 x (W [W, W], b [W])); for each branch mu, R, S, o
(E1 W [W/2, W], b; E2 W [W/2, W/2], b; head W [d_g, W/2], b); F_feat
(Z1 W [W, 2W], b [W]; Z2 W [D, W], b [D]).
"""
from __future__ import annotations

import numpy as np

W = 64          # hidden width (Appendix A)
DEPTH = 8       # F_out linear layers (Appendix A)
C = 32          # channels per plane (Appendix A, output coordinate dimension)
HALF = W // 2   # extractor width (Appendix A)
BRANCH_OUT = (3, 4, 3, 1)   # d_mu, d_R, d_S, d_o (Eq. 4)
PAIRS = ((0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3))   # xy xz yz xt yt zt


def plane_shapes(levels: int, rs: int, rt: int, c: int = C):
    """[(R_a, R_b, C)] for every (level, plane), level-major."""
    out = []
    for lv in range(levels):
        res = (rs << lv, rs << lv, rs << lv, rt)
        for a, b in PAIRS:
            out.append((res[a], res[b], c))
    return out


def layer_shapes(levels: int, D: int, c: int = C):
    """[(out, in)] of every linear layer in the flat order of the MLP blob."""
    out = [(W, levels * c)] + [(W, W)] * (DEPTH - 1)
    for d in BRANCH_OUT:
        out += [(HALF, W), (HALF, HALF), (d, HALF)]
    out += [(W, 4 * HALF), (D, W)]
    return out


def unpack_planes(blob, levels, rs, rt, c=C):
    blob = np.asarray(blob, np.float64).ravel()
    planes, off = [], 0
    for shp in plane_shapes(levels, rs, rt, c):
        n = shp[0] * shp[1] * shp[2]
        planes.append(blob[off:off + n].reshape(shp))
        off += n
    assert off == blob.size, "plane blob size"
    return planes


def unpack_mlp(blob, levels, D, c=C):
    """[(weight [out, in], bias [out])] in the flat order."""
    blob = np.asarray(blob, np.float64).ravel()
    layers, off = [], 0
    for o, i in layer_shapes(levels, D, c):
        w = blob[off:off + o * i].reshape(o, i)
        off += o * i
        b = blob[off:off + o]
        off += o
        layers.append((w, b))
    assert off == blob.size, "mlp blob size"
    return layers


def _relu(x):
    return np.where(x > 0, x, 0.0)


def _grid(coord, R):
    """Continuous grid position of a [-1, 1] coordinate on R nodes, clamped
    to the border; cell index i (0..R-2), fraction, clamp flag."""
    g = (coord + 1.0) * 0.5 * (R - 1)
    clamped = (g < 0) | (g > R - 1)
    g = np.clip(g, 0.0, R - 1)
    i = np.minimum(np.floor(g).astype(np.int64), R - 2)
    return g, i, g - i, clamped


def forward(planes, layers, mu, t, bbox_min, bbox_max, levels, rs, rt):
    """Deformation offsets of every Gaussian and the state the reverse pass
    needs.  Returns dict(dmu [P,3], dq [P,4], ds [P,3], do [P], dz [P,D],
    state)."""
    mu = np.asarray(mu, np.float64)
    P = mu.shape[0]
    lo, hi = np.asarray(bbox_min, np.float64), np.asarray(bbox_max, np.float64)
    coord = np.empty((P, 4))
    coord[:, :3] = 2.0 * (mu - lo) / (hi - lo) - 1.0
    coord[:, 3] = 2.0 * float(t) - 1.0
    samples, cells = [], []
    feats = []
    for lv in range(levels):
        res = (rs << lv, rs << lv, rs << lv, rt)
        f_lv = np.ones((P, planes[0].shape[2]))
        for k, (a, b) in enumerate(PAIRS):
            pl = planes[lv * 6 + k]
            ga, ia, fa, ca = _grid(coord[:, a], res[a])
            gb, ib, fb, cb = _grid(coord[:, b], res[b])
            p00, p10 = pl[ia, ib], pl[ia + 1, ib]
            p01, p11 = pl[ia, ib + 1], pl[ia + 1, ib + 1]
            wa, wb = fa[:, None], fb[:, None]
            s = (1 - wa) * (1 - wb) * p00 + wa * (1 - wb) * p10 + (1 - wa) * wb * p01 + wa * wb * p11
            samples.append(s)
            cells.append((ia, ib, fa, fb, ca, cb, res[a], res[b], p00, p10, p01, p11))
            f_lv = f_lv * s
        feats.append(f_lv)
    f = np.concatenate(feats, axis=1)
    # F_out: the first layer acts on f directly, later ones on relu(.)
    pre = []
    x = f
    for j in range(DEPTH):
        w, b = layers[j]
        z = (x if j == 0 else _relu(x)) @ w.T + b
        pre.append(z)
        x = z
    h = x
    deltas, e1s, hgs = [], [], []
    for g in range(4):
        (w1, b1), (w2, b2), (wh, bh) = layers[DEPTH + 3 * g:DEPTH + 3 * g + 3]
        e1 = _relu(h) @ w1.T + b1
        hg = _relu(e1) @ w2.T + b2
        deltas.append(_relu(hg) @ wh.T + bh)
        e1s.append(e1)
        hgs.append(hg)
    u = np.concatenate(hgs, axis=1)
    (z1w, z1b), (z2w, z2b) = layers[DEPTH + 12], layers[DEPTH + 13]
    v = _relu(u) @ z1w.T + z1b
    dz = _relu(v) @ z2w.T + z2b
    state = dict(coord=coord, samples=samples, cells=cells, f=f, pre=pre, e1=e1s, hg=hgs, u=u, v=v,
                 levels=levels, rs=rs, rt=rt, lo=lo, hi=hi)
    return dict(dmu=deltas[0], dq=deltas[1], ds=deltas[2], do=deltas[3][:, 0], dz=dz, state=state)


def backward(planes, layers, st, g_dmu, g_dq, g_ds, g_do, g_dz):
    """Reverse pass from the gradients of the offsets.  Returns dict(planes
    [list like planes], layers [list of (dW, db)], mu [P,3])."""
    def lin_back(dz, x_in, w):
        """dz: gradient of the layer output; x_in: the layer's input after its
        input activation.  Returns (dW, db, d x_in)."""
        return dz.T @ x_in, dz.sum(axis=0), dz @ w

    n_layers = len(layers)
    d_layers = [None] * n_layers
    # F_feat
    (z1w, _), (z2w, _) = layers[DEPTH + 12], layers[DEPTH + 13]
    g_dz = np.asarray(g_dz, np.float64)
    dW, db, d_rv = lin_back(g_dz, _relu(st["v"]), z2w)
    d_layers[DEPTH + 13] = (dW, db)
    d_v = d_rv * (st["v"] > 0)
    dW, db, d_ru = lin_back(d_v, _relu(st["u"]), z1w)
    d_layers[DEPTH + 12] = (dW, db)
    d_u = d_ru * (st["u"] > 0)
    # Branches
    g_out = [np.asarray(g_dmu, np.float64), np.asarray(g_dq, np.float64), np.asarray(g_ds, np.float64),
             np.asarray(g_do, np.float64).reshape(-1, 1)]
    h = st["pre"][-1]
    d_rh = np.zeros_like(h)
    for g in range(4):
        (w1, _), (w2, _), (wh, _) = layers[DEPTH + 3 * g:DEPTH + 3 * g + 3]
        e1, hg = st["e1"][g], st["hg"][g]
        dW, db, d_rhg = lin_back(g_out[g], _relu(hg), wh)
        d_layers[DEPTH + 3 * g + 2] = (dW, db)
        d_hg = d_rhg * (hg > 0) + d_u[:, g * HALF:(g + 1) * HALF]
        dW, db, d_re1 = lin_back(d_hg, _relu(e1), w2)
        d_layers[DEPTH + 3 * g + 1] = (dW, db)
        d_e1 = d_re1 * (e1 > 0)
        dW, db, d_rh_g = lin_back(d_e1, _relu(h), w1)
        d_layers[DEPTH + 3 * g] = (dW, db)
        d_rh += d_rh_g
    # F_out, last layer first: the gradient of layer j's output is d_z.
    d_z = d_rh * (h > 0)
    for j in range(DEPTH - 1, -1, -1):
        w, _ = layers[j]
        x_in = st["f"] if j == 0 else _relu(st["pre"][j - 1])
        dW, db, dx = lin_back(d_z, x_in, w)
        d_layers[j] = (dW, db)
        d_z = dx if j == 0 else dx * (st["pre"][j - 1] > 0)
    d_f = d_z
    # HexPlane: product rule within each level, then bilinear weights.
    levels, c = st["levels"], planes[0].shape[2]
    P = d_f.shape[0]
    d_planes = [np.zeros_like(pl) for pl in planes]
    d_coord = np.zeros((P, 4))
    for lv in range(levels):
        df_lv = d_f[:, lv * c:(lv + 1) * c]
        for k, (a, b) in enumerate(PAIRS):
            others = np.ones((P, c))
            for m in range(6):
                if m != k:
                    others = others * st["samples"][lv * 6 + m]
            ds = df_lv * others
            ia, ib, fa, fb, ca, cb, Ra, Rb, p00, p10, p01, p11 = st["cells"][lv * 6 + k]
            wa, wb = fa[:, None], fb[:, None]
            dp = d_planes[lv * 6 + k]
            np.add.at(dp, (ia, ib), (1 - wa) * (1 - wb) * ds)
            np.add.at(dp, (ia + 1, ib), wa * (1 - wb) * ds)
            np.add.at(dp, (ia, ib + 1), (1 - wa) * wb * ds)
            np.add.at(dp, (ia + 1, ib + 1), wa * wb * ds)
            dga = np.sum(ds * ((1 - wb) * (p10 - p00) + wb * (p11 - p01)), axis=1)
            dgb = np.sum(ds * ((1 - wa) * (p01 - p00) + wa * (p11 - p10)), axis=1)
            d_coord[:, a] += np.where(ca, 0.0, dga * 0.5 * (Ra - 1))
            d_coord[:, b] += np.where(cb, 0.0, dgb * 0.5 * (Rb - 1))
    d_mu = d_coord[:, :3] * 2.0 / (st["hi"] - st["lo"])
    return dict(planes=d_planes, layers=d_layers, mu=d_mu)


def margins(st):
    """Per Gaussian: the smallest |pre-activation| of every ReLU decision
    relative to the rms of its layer, and the smallest distance of a grid
    position to a cell edge or the clamp border (in cells).  A binary32
    evaluation may take the other side of a decision within these margins."""
    P = st["f"].shape[0]
    rel = np.full(P, np.inf)
    for z in st["pre"] + st["e1"] + st["hg"] + [st["u"], st["v"]]:
        rms = max(np.sqrt(np.mean(z * z)), 1e-300)
        rel = np.minimum(rel, np.min(np.abs(z), axis=1) / rms)
    cell = np.full(P, np.inf)
    for lv in range(st["levels"]):
        res = (st["rs"] << lv, st["rs"] << lv, st["rs"] << lv, st["rt"])
        for a in range(4):
            g = (st["coord"][:, a] + 1.0) * 0.5 * (res[a] - 1)
            d = np.abs(g - np.round(g))
            cell = np.minimum(cell, d)
    return rel, cell


def apply(mu, quats, log_scales, logits, feat, out):
    """The deformed Gaussian G_t of Eq. 6 in the parameterisation the
    renderer takes: mu + d_mu, q + d_q (normalised by the renderer),
    log s + d_s, opacity logit + d_o, z + d_z (Eq. 5)."""
    return (np.asarray(mu, np.float64) + out["dmu"], np.asarray(quats, np.float64) + out["dq"],
            np.asarray(log_scales, np.float64) + out["ds"], np.asarray(logits, np.float64) + out["do"],
            np.asarray(feat, np.float64) + out["dz"])


def tv_loss(planes, levels):
    """Total-variation smoothness of the planes (the L_TV term of Eq. 11),
    read as in the HexPlane / K-Planes lineage: for every plane the mean
    squared difference of neighbouring nodes along each of its two axes,
    summed over planes.  Returns (loss, gradients like planes)."""
    loss = 0.0
    grads = []
    for pl in planes[:6 * levels]:
        g = np.zeros_like(pl)
        for ax in (0, 1):
            d = np.diff(pl, axis=ax)
            n = d.size
            loss += np.sum(d * d) / n
            gd = 2.0 * d / n
            if ax == 0:
                g[1:] += gd
                g[:-1] -= gd
            else:
                g[:, 1:] += gd
                g[:, :-1] -= gd
        grads.append(g)
    return loss, grads
