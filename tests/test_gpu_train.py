"""GPU checks of the training iteration: the fused Adam kernel against the
FP64 oracle's Adam, its bf16 storage copies, and one full iteration
(render, L1 RGB, decoder L1, reverse, Adam) whose update matches the
oracle's Adam applied to the iteration's own gradients."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2503_06161_gb300 import _lib, synth  # noqa: E402
from paper_2503_06161_gb300.optim import Adam  # noqa: E402
from paper_2503_06161_gb300.train import Trainer  # noqa: E402

from gpu_helpers import deformed_case  # noqa: E402

TOL_ADAM = 2e-6  # relative to the parameter scale: FP32 arithmetic of one update
# The kernel receives its hyperparameters as float32; the oracle takes those
# same values.
B1, B2, EPS = (float(np.float32(x)) for x in (0.9, 0.999, 1e-15))


def f32(x):
    return float(np.float32(x))


def test_adam_matches_oracle_with_tails_and_bf16_copies():
    rng = np.random.default_rng(0)
    sizes = [1001, 6, 64 * 3 + 1]  # tails that are not a multiple of 4
    lrs = [1e-2, 3e-3, 5e-2]
    ps = [rng.normal(size=n).astype(np.float32) for n in sizes]
    pt = [torch.tensor(p).cuda() for p in ps]
    pb = [torch.empty(n, dtype=torch.bfloat16, device="cuda") for n in sizes]
    opt = Adam([dict(param=p, lr=lr, param_bf16=b) for p, lr, b in zip(pt, lrs, pb)])
    ref = [(p.astype(np.float64), np.zeros(len(p)), np.zeros(len(p))) for p in ps]
    for step in range(1, 4):
        gs = [rng.normal(size=n).astype(np.float32) * (10.0 ** -k) for k, n in enumerate(sizes)]
        opt.step([torch.tensor(g).cuda() for g in gs])
        ref = [O.adam_step(p, g, m, v, step, f32(lr), B1, B2, EPS) for (p, m, v), g, lr in zip(ref, gs, lrs)]
        torch.cuda.synchronize()
        for k in range(len(sizes)):
            got = pt[k].cpu().numpy()
            assert np.max(np.abs(got - ref[k][0])) <= TOL_ADAM * max(1.0, np.max(np.abs(ref[k][0])))
            for j in (1, 2):  # moments: FP32 rounding relative to their scale
                got_j = opt.groups[k]["m" if j == 1 else "v"].cpu().numpy()
                assert np.max(np.abs(got_j - ref[k][j])) <= 1e-6 * np.max(np.abs(ref[k][j]))
            bits = pb[k].cpu().view(torch.int16).numpy().view(np.uint16)
            assert np.array_equal(bits, synth.bf16_bits(got))


def test_adam_rejects_bad_groups():
    p = torch.zeros(8, device="cuda")
    with pytest.raises(_lib.FeError):
        _lib.fe_adam_step([dict(param=p, grad=p, m=p, v=p, lr=1.0)], 0, 0.9, 0.999, 1e-15)   # step 0
    q = torch.zeros(9, device="cuda")[1:]  # 4-byte offset: not 16-byte aligned
    with pytest.raises(_lib.FeError):
        _lib.fe_adam_step([dict(param=q, grad=q, m=q, v=q, lr=1.0)], 1, 0.9, 0.999, 1e-15)


def _trainer(seed=0):
    sc, cam, df = deformed_case(P=3000, W=150, H=100, D=32, seed=seed)
    w, b = synth.make_decoder(32, seed=5, b_std=0.1)
    return Trainer.from_numpy(sc, cam, df, w, b, max_dups=200_000)


def test_training_iteration_updates_match_oracle_adam_on_its_gradients():
    tr = _trainer()
    H, W = tr.cam.height, tr.cam.width
    rng = np.random.default_rng(3)
    tgt_rgb = torch.tensor(rng.random((3, H, W)).astype(np.float32)).cuda()
    tgt_dec = torch.tensor(rng.normal(size=(H * W, 256)).astype(np.float32)).to(torch.bfloat16).cuda()
    before = {k: v.detach().cpu().numpy().astype(np.float64) for k, v in tr.m.items()}
    losses = tr.step(0.4, tgt_rgb, tgt_dec)
    torch.cuda.synchronize()
    assert tr.rast.stats()["device_errors"] == 0 and tr.dec.errors() == 0
    assert np.all(np.isfinite(losses.cpu().numpy()))
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in tr.grads.items()}
    for k in before:
        lr = tr.opt.groups[["means", "log_scales", "quats", "opacity_logits", "sh", "feat"].index(k)]["lr"]
        ref, _, _ = O.adam_step(before[k], g[k], 0.0, 0.0, 1, f32(lr), B1, B2, EPS)
        got = tr.m[k].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= TOL_ADAM * max(1.0, np.max(np.abs(ref))), k
    # The renderer's bf16 storage follows the masters.
    assert np.array_equal(tr.feat_store.cpu().view(torch.int16).numpy().view(np.uint16),
                          synth.bf16_bits(tr.m["feat"].cpu().numpy()))
    # The gradients reached every group (rendered Gaussians move).
    assert np.abs(g["means"]).sum() > 0 and np.abs(g["feat"]).sum() > 0 and np.abs(g["sh"]).sum() > 0


def test_training_is_deterministic():
    a, b = _trainer(), _trainer()
    H, W = a.cam.height, a.cam.width
    rng = np.random.default_rng(4)
    tgt_rgb = torch.tensor(rng.random((3, H, W)).astype(np.float32)).cuda()
    tgt_dec = torch.tensor(rng.normal(size=(H * W, 256)).astype(np.float32)).to(torch.bfloat16).cuda()
    for t in (0.1, 0.7):
        la = a.step(t, tgt_rgb, tgt_dec).clone()
        lb = b.step(t, tgt_rgb, tgt_dec).clone()
        torch.cuda.synchronize()
        assert torch.equal(la, lb)
    for k in a.m:
        assert torch.equal(a.m[k], b.m[k]), k


def test_depth_term_of_the_loss():
    """lambda_depth * L1 depth (Eq. 11): its value against an FP64 mean of the
    rendered depth, its per-pixel gradient, and its share of the parameter
    gradients (the reverse pass is linear in the image gradients, so the
    iteration with the depth term equals the one without plus a depth-only
    reverse)."""
    from paper_2503_06161_gb300.train import LAMBDA_DEPTH
    tr = _trainer(seed=1)
    H, W = tr.cam.height, tr.cam.width
    rng = np.random.default_rng(5)
    tgt_rgb = torch.tensor(rng.random((3, H, W)).astype(np.float32)).cuda()
    tgt_dec = torch.tensor(rng.normal(size=(H * W, 256)).astype(np.float32)).to(torch.bfloat16).cuda()
    tgt_depth = torch.tensor(rng.uniform(0.0, 4.0, size=(H, W)).astype(np.float32)).cuda()
    t = 0.6
    tr.forward_backward(t, tgt_rgb, tgt_dec)
    torch.cuda.synchronize()
    base = {k: v.clone() for k, v in tr.grads.items()}
    assert tr.losses[2].item() == 0.0
    tr.forward_backward(t, tgt_rgb, tgt_dec, tgt_depth)
    torch.cuda.synchronize()
    depth = tr.out[1].cpu().numpy().astype(np.float64)
    diff = depth - tgt_depth.cpu().numpy().astype(np.float64)
    ref_loss = LAMBDA_DEPTH * np.mean(np.abs(diff))
    assert abs(tr.losses[2].item() - ref_loss) <= 1e-5 * ref_loss
    inv = np.float32(1.0) / np.float32(round(H * W / LAMBDA_DEPTH))
    assert np.array_equal(tr.g_depth.cpu().numpy(), (np.sign(diff) * inv).astype(np.float32))
    full = {k: v.clone() for k, v in tr.grads.items()}
    zr, zf = torch.zeros_like(tr.g_rgb), torch.zeros_like(tr.dec_out[1])
    tr.rast.backward(tr.scene, tr.cam, tr.deform, t, zr, tr.g_depth, None, zf, grads=tr.grads)
    torch.cuda.synchronize()
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        d = tr.grads[k].cpu().numpy().astype(np.float64)
        assert np.abs(d).sum() > 0, k
        got = full[k].cpu().numpy().astype(np.float64) - base[k].cpu().numpy().astype(np.float64)
        scale = np.sqrt(np.mean(full[k].cpu().numpy().astype(np.float64) ** 2))
        assert np.max(np.abs(got - d)) <= 1e-4 * scale, k


def test_training_with_the_full_fst_module():
    """One iteration with the full FST module (Sec. 3.2) around the renderer:
    lambda_TV * L_TV against the oracle on the pre-step planes, and the
    planes / MLP / canonical-mean updates equal to the oracle's Adam on the
    iteration's own gradients (scheduled learning rates at step 0 are the
    initial ones)."""
    from oracle import fst as OF
    from paper_2503_06161_gb300.fst import FSTDeform
    from paper_2503_06161_gb300.train import LAMBDA_TV, LR
    levels, rs, rt = 2, 16, 10
    sc, cam, _ = deformed_case(P=3000, W=150, H=100, D=32, seed=4)
    planes, mlp = synth.make_fst(levels, rs, rt, 32, seed=6, plane_std=0.1, head_std=0.05)
    fst = FSTDeform.from_numpy(planes, mlp, levels, rs, rt, 32, (-1, -1, 2), (1, 1, 4), sc.P)
    w, b = synth.make_decoder(32, seed=5, b_std=0.1)
    tr = Trainer.from_numpy(sc, cam, None, w, b, max_dups=200_000, fst=fst)
    H, W = tr.cam.height, tr.cam.width
    rng = np.random.default_rng(8)
    tgt_rgb = torch.tensor(rng.random((3, H, W)).astype(np.float32)).cuda()
    tgt_dec = torch.tensor(rng.normal(size=(H * W, 256)).astype(np.float32)).to(torch.bfloat16).cuda()
    tgt_depth = torch.tensor(synth.make_depth_target(H, W, 2.0, 4.0)).cuda()
    p0, m0 = fst.planes.cpu().numpy().astype(np.float64), fst.mlp.cpu().numpy().astype(np.float64)
    mu0 = tr.m["means"].cpu().numpy().astype(np.float64)
    losses = tr.step(0.35, tgt_rgb, tgt_dec, tgt_depth)
    torch.cuda.synchronize()
    assert tr.rast.stats()["device_errors"] == 0 and tr.dec.errors() == 0
    L = losses.cpu().numpy()
    assert np.all(np.isfinite(L)) and L[2] > 0
    ref_tv, _ = OF.tv_loss(OF.unpack_planes(p0, levels, rs, rt), levels)
    assert abs(L[3] - LAMBDA_TV * ref_tv) <= 1e-5 * LAMBDA_TV * ref_tv
    for got, before, grad, lr in ((fst.planes, p0, fst.d_planes, LR["grid"]), (fst.mlp, m0, fst.d_mlp, LR["deformation"]),
                                  (tr.m["means"], mu0, tr.grads["means"], LR["means"])):
        g = grad.cpu().numpy().astype(np.float64)
        assert np.abs(g).sum() > 0
        ref, _, _ = O.adam_step(before, g, 0.0, 0.0, 1, f32(lr), B1, B2, EPS)
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= TOL_ADAM * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("use_fst", [False, True])
def test_training_with_density_control(use_fst):
    """Statistics gathered by the iterations drive clone / split / prune of
    every parameter, render copy and Adam moment (the Trainer's result equals
    the densify call on a snapshot of the same buffers); a densify that
    selects nothing is the identity; training continues on the new set with
    every P-sized buffer rebuilt; the opacity reset caps every opacity."""
    from paper_2503_06161_gb300 import density
    from paper_2503_06161_gb300.fst import FSTDeform
    sc, cam, df = deformed_case(P=3000, W=150, H=100, D=32, seed=2)
    w, b = synth.make_decoder(32, seed=5, b_std=0.1)
    kw = dict(max_dups=200_000, density_stats=True)
    if use_fst:
        planes, mlp = synth.make_fst(2, 16, 10, 32, seed=6, plane_std=0.1, head_std=0.05)
        kw["fst"] = FSTDeform.from_numpy(planes, mlp, 2, 16, 10, 32, (-1.5, -1, 1.5), (1.5, 1, 5), sc.P)
        df = None
    tr = Trainer.from_numpy(sc, cam, df, w, b, **kw)
    H, W = tr.cam.height, tr.cam.width
    rng = np.random.default_rng(9)
    tgt_rgb = torch.tensor(rng.random((3, H, W)).astype(np.float32)).cuda()
    tgt_dec = torch.tensor(rng.normal(size=(H * W, 256)).astype(np.float32)).to(torch.bfloat16).cuda()
    for t in (0.2, 0.5, 0.8):
        tr.step(t, tgt_rgb, tgt_dec)
    torch.cuda.synchronize()
    cnt = tr.stats.count.cpu().numpy()
    assert cnt.max() == 3 and (cnt > 0).sum() > 1000 and tr.stats.accum.sum().item() > 0
    # Nothing selected: the identity.
    snap = {k: v.clone() for k, v in tr.m.items()}
    mom = [(g["m"].clone(), g["v"].clone()) for g in tr.opt.groups[:6]]
    assert tr.densify_and_prune(extent=1.0, grad_thresh=1e30, min_opacity=0.0) == 3000
    for k in snap:
        assert torch.equal(snap[k], tr.m[k]), k
    for (m, v), g in zip(mom, tr.opt.groups[:6]):
        assert torch.equal(m, g["m"]) and torch.equal(v, g["v"])
    assert tr.stats.count.sum().item() == 0
    for t in (0.3, 0.6):
        tr.step(t, tgt_rgb, tgt_dec)
    # A selective densify equals the densify call on a snapshot.
    extent = 1.5
    params = {k: tr.m[k].clone() for k in Trainer.GAUSS_KEYS}
    params["sh_store"], params["feat_store"] = tr.sh_store.clone(), tr.feat_store.clone()
    state = {}
    for i, k in enumerate(Trainer.GAUSS_KEYS):
        state[k + ".m"], state[k + ".v"] = tr.opt.groups[i]["m"].clone(), tr.opt.groups[i]["v"].clone()
    st = density.DensityStats(tr.P)
    st.accum.copy_(tr.stats.accum)
    st.count.copy_(tr.stats.count)
    normals = torch.tensor(np.random.default_rng(1).normal(size=(tr.P, 2, 3)).astype(np.float32)).cuda()
    ref_p, ref_s, ref_n = density.densify(params, state, st, normals, 1e-4, 0.01 * extent, 0.02)
    n = tr.densify_and_prune(extent, normals=normals, grad_thresh=1e-4, min_opacity=0.02)
    assert n == ref_n and n != 3000
    for k in Trainer.GAUSS_KEYS:
        assert torch.equal(tr.m[k], ref_p[k]), k
        g = tr.opt.groups[Trainer.GAUSS_KEYS.index(k)]
        assert torch.equal(g["m"], ref_s[k + ".m"]) and torch.equal(g["v"], ref_s[k + ".v"]), k
    assert torch.equal(tr.sh_store, ref_p["sh_store"]) and torch.equal(tr.feat_store, ref_p["feat_store"])
    assert tr.rast.P == n and tr.stats.P == n and tr.grads["sh"].shape[0] == n
    for t in (0.25, 0.75):
        L = tr.step(t, tgt_rgb, tgt_dec)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(L.cpu().numpy())) and tr.rast.stats()["device_errors"] == 0
    assert tr.stats.count.max().item() == 2
    tr.reset_opacity(0.01)
    op = torch.sigmoid(tr.m["opacity_logits"].double()).cpu().numpy()
    assert op.max() <= 0.01 * (1 + 1e-6) and tr.opt.groups[3]["m"].abs().sum().item() == 0
