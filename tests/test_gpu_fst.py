"""GPU parity of the full FST deformation module (Sec. 3.2, Eq. 4-6;
Appendix A) against the FP64 oracle: deformed Gaussians, the reverse pass
(canonical means through the HexPlane coordinates, plane gradients, every
weight and bias), the TV term, ragged and multi-block sizes, every D, and
the bf16 feature storage.

With exact_planes the plane gradients are exact fixed-point sums, compared
bitwise between runs and between orders of the Gaussians.

Comparison protocol: an FP32 evaluation may take the other side of a ReLU
or grid-cell decision whose FP64 margin is tiny; Gaussians with such a
decision get zero upstream gradients on both sides, so they drop out of
every reverse-pass sum (the forward is continuous and is compared for all
Gaussians)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fst as OF  # noqa: E402
from paper_2503_06161_gb300 import _lib, synth  # noqa: E402
from paper_2503_06161_gb300.fst import FSTDeform  # noqa: E402
from paper_2503_06161_gb300.raster import GaussianScene  # noqa: E402

from gpu_helpers import TOL_FEAT_REL, TOL_GRAD_REL, rel_err  # noqa: E402

LO, HI = (-2.0, -2.0, 3.0), (2.0, 2.0, 8.0)
RELU_MARGIN, CELL_MARGIN = 3e-5, 1e-4


def _case(P, levels, rs, rt, D, seed=0, bf16=False, bias_std=0.1):
    sc = synth.make_scene(P, D, LO, HI, seed=seed, bf16_storage=bf16)
    planes, mlp = synth.make_fst(levels, rs, rt, D, seed=seed + 1, plane_std=0.2, head_std=0.5, dz_std=0.5,
                                 bias_std=bias_std)
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=bf16)
    fst = FSTDeform.from_numpy(planes, mlp, levels, rs, rt, D, LO, HI, P)
    pl = OF.unpack_planes(planes, levels, rs, rt)
    ly = OF.unpack_mlp(mlp, levels, D)
    return sc, scene, fst, pl, ly


def _oracle_forward(sc, pl, ly, t, levels, rs, rt, bf16):
    feat = synth.bf16_round(sc.feat) if bf16 else sc.feat
    out = OF.forward(pl, ly, np.asarray(sc.means, np.float64), t, LO, HI, levels, rs, rt)
    return out, feat


@pytest.mark.parametrize("P,levels,rs,rt,D", [(1000, 2, 8, 6, 32), (333, 4, 8, 5, 16), (700, 3, 6, 7, 64),
                                              (257, 1, 16, 9, 128)])
def test_forward_matches_oracle(P, levels, rs, rt, D):
    sc, scene, fst, pl, ly = _case(P, levels, rs, rt, D)
    t = 0.43
    st = fst.forward(scene, t)
    torch.cuda.synchronize()
    out, feat = _oracle_forward(sc, pl, ly, t, levels, rs, rt, False)
    ref = OF.apply(sc.means, sc.quats, sc.log_scales, sc.opacity_logits, feat, out)
    got = [st.means, st.quats, st.log_scales, st.opacity_logits, st.feat]
    canon = [sc.means, sc.quats, sc.log_scales, sc.opacity_logits, feat]
    for name, gg, r, c in zip(["means", "quats", "log_scales", "logits", "feat"], got, ref, canon):
        g64 = gg.cpu().numpy().astype(np.float64)
        # offsets compared against their own scale (the canonical part is exact input)
        off_got = g64 - np.asarray(c, np.float64).reshape(g64.shape)
        off_ref = np.asarray(r, np.float64).reshape(g64.shape) - np.asarray(c, np.float64).reshape(g64.shape)
        assert rel_err(off_got, off_ref) < TOL_FEAT_REL, name
        assert np.abs(off_ref).max() > 1e-3, name   # the offsets are not trivially zero


def test_bf16_features_are_rounded_sums():
    P, levels, rs, rt, D = 500, 2, 8, 6, 32
    sc, scene, fst, pl, ly = _case(P, levels, rs, rt, D, seed=3, bf16=True)
    st = fst.forward(scene, 0.8)
    torch.cuda.synchronize()
    out, feat = _oracle_forward(sc, pl, ly, 0.8, levels, rs, rt, True)
    want = np.asarray(feat, np.float64) + out["dz"]
    got = st.feat.float().cpu().numpy().astype(np.float64)
    assert st.feat.dtype == torch.bfloat16
    # nearest-even bf16 of an FP32 sum: within half a bf16 ulp plus the FP32
    # error of the sum, which scales with the addends (they can cancel)
    ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(want), 1e-30))) - 7)
    fp32 = 1e-5 * (np.abs(np.asarray(feat, np.float64)) + np.abs(out["dz"]))
    assert np.all(np.abs(got - want) <= 0.5 * ulp + fp32 + 1e-30)


def _upstream(P, D, seed):
    rng = np.random.default_rng(seed)
    return dict(means=rng.normal(size=(P, 3)), quats=rng.normal(size=(P, 4)), log_scales=rng.normal(size=(P, 3)),
                opacity_logits=rng.normal(size=P), feat=rng.normal(size=(P, D)))


@pytest.mark.parametrize("P,levels,rs,rt,D", [(1000, 2, 8, 6, 32), (333, 4, 8, 5, 16), (700, 3, 6, 7, 64),
                                              (257, 1, 16, 9, 128), (40000, 2, 16, 10, 32)])
def test_backward_matches_oracle(P, levels, rs, rt, D):
    sc, scene, fst, pl, ly = _case(P, levels, rs, rt, D, seed=7)
    t = 0.61
    fst.forward(scene, t)
    out, _ = _oracle_forward(sc, pl, ly, t, levels, rs, rt, False)
    rel, cell = OF.margins(out["state"])
    drop = (rel < RELU_MARGIN) | (cell < CELL_MARGIN)
    assert drop.sum() < 0.1 * P   # the comparison is not emptied by the protocol
    up = _upstream(P, D, seed=P)
    for k in up:
        up[k][drop] = 0.0
    dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous() for k, v in up.items()}
    grads = dict(dev)
    grads["means"] = dev["means"].clone()
    fst.backward(scene, t, grads)
    torch.cuda.synchronize()
    ref = OF.backward(pl, ly, out["state"], up["means"], up["quats"], up["log_scales"], up["opacity_logits"],
                      up["feat"])
    # canonical means: upstream plus the HexPlane path
    got_mu = grads["means"].cpu().numpy().astype(np.float64)
    assert rel_err(got_mu, up["means"] + ref["mu"]) < TOL_GRAD_REL
    assert rel_err(got_mu - up["means"], ref["mu"]) < 1e-2      # the path alone, at its own scale
    # planes (untouched nodes exactly zero)
    got_pl = fst.d_planes.cpu().numpy().astype(np.float64)
    ref_pl = np.concatenate([x.ravel() for x in ref["planes"]])
    assert rel_err(got_pl, ref_pl) < TOL_GRAD_REL
    assert np.all(got_pl[ref_pl == 0.0] == 0.0)
    # every layer's weight and bias
    got_w = fst.d_mlp.cpu().numpy().astype(np.float64)
    off = 0
    for j, (dw, db) in enumerate(ref["layers"]):
        n = dw.size
        assert rel_err(got_w[off:off + n], dw.ravel()) < TOL_GRAD_REL, (j, "weight")
        off += n
        assert rel_err(got_w[off:off + db.size], db) < TOL_GRAD_REL, (j, "bias")
        off += db.size
    assert off == got_w.size
    print(f"dropped {int(drop.sum())} of {P} Gaussians near a decision")


def test_full_size_module_on_sampled_gaussians():
    """The training workload's module and launch configuration (200,000
    Gaussians, 4 levels of 64^3 x 100, D=32): offsets of a random sample of
    Gaussians against the oracle, and the reverse pass with upstream
    gradients on that sample only (the others contribute exact zeros), so the
    oracle's plane and weight gradients of the sample are the exact
    reference."""
    P, levels, rs, rt, D = 200_000, 4, 64, 100, 32
    sc = synth.make_scene(P, D, LO, HI, seed=0)
    planes, mlp = synth.make_fst(levels, rs, rt, D, seed=1)
    scene = GaussianScene.from_numpy(sc, "cuda")
    fst = FSTDeform.from_numpy(planes, mlp, levels, rs, rt, D, LO, HI, P)
    pl, ly = OF.unpack_planes(planes, levels, rs, rt), OF.unpack_mlp(mlp, levels, D)
    t = 0.37
    st = fst.forward(scene, t)
    rng = np.random.default_rng(21)
    idx = np.sort(rng.choice(P, 1500, replace=False))
    out = OF.forward(pl, ly, np.asarray(sc.means, np.float64)[idx], t, LO, HI, levels, rs, rt)
    torch.cuda.synchronize()
    for got, canon, off in ((st.means, sc.means, out["dmu"]), (st.feat, sc.feat, out["dz"])):
        # deformed = canonical + offset, rounded to float32 once: the offset
        # is compared at its own scale plus that rounding
        c = np.asarray(canon, np.float64)[idx]
        g = got.float().cpu().numpy().astype(np.float64)[idx] - c
        den = np.maximum(np.abs(off), np.sqrt(np.mean(off ** 2)))
        assert np.all(np.abs(g - off) <= TOL_FEAT_REL * den + 1.2e-7 * np.abs(c + off))
    rel, cell = OF.margins(out["state"])
    keep = (rel >= RELU_MARGIN) & (cell >= CELL_MARGIN)
    assert keep.sum() > 0.9 * len(idx)
    up_s = _upstream(len(idx), D, seed=5)
    for k in up_s:
        up_s[k][~keep] = 0.0
    full = {k: np.zeros((P,) + v.shape[1:]) for k, v in up_s.items()}
    for k in full:
        full[k][idx] = up_s[k]
    dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous() for k, v in full.items()}
    grads = dict(dev, means=dev["means"].clone())
    fst.backward(scene, t, grads)
    torch.cuda.synchronize()
    ref = OF.backward(pl, ly, out["state"], up_s["means"], up_s["quats"], up_s["log_scales"],
                      up_s["opacity_logits"], up_s["feat"])
    gm = grads["means"].cpu().numpy().astype(np.float64)
    assert rel_err(gm[idx], up_s["means"] + ref["mu"]) < TOL_GRAD_REL
    others = np.ones(P, bool)
    others[idx] = False
    assert np.all(gm[others] == 0.0)
    got_pl = fst.d_planes.cpu().numpy().astype(np.float64)
    ref_pl = np.concatenate([x.ravel() for x in ref["planes"]])
    # Only the sample's corners are touched (a few hundred thousand of 42.6 M
    # entries); the others must stay exactly zero.  The touched ones are
    # compared at the scale of the touched entries (the rms over all entries
    # would shrink with the sample's sparsity).
    nz = ref_pl != 0.0
    assert np.all(got_pl[~nz] == 0.0)
    assert rel_err(got_pl[nz], ref_pl[nz]) < TOL_GRAD_REL
    got_w = fst.d_mlp.cpu().numpy().astype(np.float64)
    ref_w = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in ref["layers"]])
    assert rel_err(got_w, ref_w) < TOL_GRAD_REL


def test_weight_gradients_are_reproducible():
    P, levels, rs, rt, D = 5000, 2, 8, 6, 32
    sc, scene, fst, _, _ = _case(P, levels, rs, rt, D, seed=11)
    fst.forward(scene, 0.3)
    up = _upstream(P, D, seed=1)
    res = []
    for _ in range(2):
        dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda") for k, v in up.items()}
        fst.backward(scene, 0.3, dev)
        torch.cuda.synchronize()
        res.append((fst.d_mlp.clone(), dev["means"].clone()))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


def test_exact_plane_gradients_are_independent_of_order():
    # With exact_planes the plane gradients are every Gaussian's terms summed
    # exactly in fixed point (integer atomics), then rounded once: two runs
    # give the same bits, and so does the same scene with its Gaussians in
    # another order (the per-Gaussian terms are the same; only the summation
    # order of a float sum would change).  The default float-atomic sums
    # agree with them to float rounding.
    P, levels, rs, rt, D = 6000, 2, 8, 6, 32
    sc, scene, fst, _, _ = _case(P, levels, rs, rt, D, seed=12)
    t = 0.3
    up = _upstream(P, D, seed=2)
    fst.forward(scene, t)
    dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda") for k, v in up.items()}
    fst.backward(scene, t, dev)
    torch.cuda.synchronize()
    fast = fst.d_planes.clone()
    fst = FSTDeform(fst.planes, fst.mlp, levels, rs, rt, D, LO, HI, P, exact_planes=True)

    def run(scene_, up_):
        fst.forward(scene_, t)
        dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda") for k, v in up_.items()}
        fst.backward(scene_, t, dev)
        torch.cuda.synchronize()
        return fst.d_planes.clone()

    a = run(scene, up)
    b = run(scene, up)
    assert torch.equal(a, b)
    assert int((a != 0).sum()) > 1000
    assert rel_err(fast.cpu().numpy(), a.cpu().numpy()) < 1e-5
    perm = np.random.default_rng(3).permutation(P)
    sc_p = synth.Scene(sc.means[perm], sc.log_scales[perm], sc.quats[perm], sc.opacity_logits[perm], sc.sh[perm],
                       sc.feat[perm], sc.sh_degree)
    scene_p = GaussianScene.from_numpy(sc_p, "cuda")
    c = run(scene_p, {k: v[perm] for k, v in up.items()})
    assert torch.equal(a, c)
    assert int(fst.workspace[:4].view(torch.int32).item()) == 0        # no plane-gradient term clamped


def test_tv_matches_oracle():
    levels, rs, rt, D = 2, 8, 6, 32
    planes, mlp = synth.make_fst(levels, rs, rt, D, seed=2, plane_std=0.3)
    fst = FSTDeform.from_numpy(planes, mlp, levels, rs, rt, D, LO, HI, 16)
    loss = torch.zeros(1, device="cuda")
    scratch = torch.empty(1024, device="cuda")
    fst.d_planes.fill_(0.25)
    fst.tv(0.03, loss, scratch)
    torch.cuda.synchronize()
    ref_loss, ref_g = OF.tv_loss(OF.unpack_planes(planes, levels, rs, rt), levels)
    assert abs(loss.item() - 0.03 * ref_loss) <= 1e-5 * 0.03 * ref_loss
    ref = 0.25 + 0.03 * np.concatenate([g.ravel() for g in ref_g])
    assert rel_err(fst.d_planes.cpu().numpy(), ref) < 1e-5


def test_empty_and_bad_arguments():
    levels, rs, rt, D = 1, 4, 4, 16
    planes, mlp = synth.make_fst(levels, rs, rt, D, seed=0)
    fst = FSTDeform.from_numpy(planes, mlp, levels, rs, rt, D, LO, HI, 0)
    z = torch.zeros(0, 3, device="cuda")
    scene = GaussianScene(z, z.clone(), torch.zeros(0, 4, device="cuda"), torch.zeros(0, device="cuda"),
                          torch.zeros(0, 16, 3, device="cuda"), torch.zeros(0, D, device="cuda"), 3)
    fst.forward(scene, 0.5)
    g = dict(means=z.clone(), quats=torch.zeros(0, 4, device="cuda"), log_scales=z.clone(),
             opacity_logits=torch.zeros(0, device="cuda"), feat=torch.zeros(0, D, device="cuda"))
    fst.backward(scene, 0.5, g)
    torch.cuda.synchronize()
    assert float(fst.d_mlp.abs().sum()) == 0.0 and float(fst.d_planes.abs().sum()) == 0.0
    bad = fst.struct()
    bad.D = 24
    with pytest.raises(_lib.FeError):
        _lib.fe_fst_forward(bad, 0, z, z, z, z, z, 0.5, z, z, z, z, z, fst.workspace, False)
