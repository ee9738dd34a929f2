"""GPU parity of adaptive density control against the FP64 oracle, through
the C ABI.

Decisions, the new Gaussian count, the output order, copied rows and
optimiser state are bit-exact (the decision is taken in float32 on both
sides; the oracle's FP64 decision agrees away from the thresholds).  Split
children's centres are within 2e-6 of the oracle (float32 rotation of the
scaled normal), their log-scales within 1e-6.  Screen-space statistics are
compared with the oracle's centre gradients at the reverse pass's bar."""
import numpy as np
import pytest
import torch

from oracle import density as DN
from oracle import oracle as O
from paper_2503_06161_gb300 import _lib, density, synth
from tests.gpu_helpers import TOL_GRAD_REL, deformed_case, gpu_backward, gpu_forward, rel_err

pytestmark = pytest.mark.gpu

THRESH, MIN_OP = 2e-4, 0.005
DENSE = 0.01 * np.sqrt(4 ** 2 + 4 ** 2 + 5 ** 2) / 2      # percent dense x half-diagonal of the scene box


def _inputs(P, D=32, seed=0):
    sc = synth.make_scene(P, D, (-2, -2, 3), (2, 2, 8), seed=seed)
    accum, count, normals = synth.make_density_stats(P, seed=seed + 6)
    params = dict(means=sc.means, log_scales=sc.log_scales - np.float32(0.6), quats=sc.quats,
                  opacity_logits=sc.opacity_logits * np.float32(3.0), sh=sc.sh.reshape(P, 16, 3), feat=sc.feat)
    rng = np.random.default_rng(seed + 9)
    state = dict(m_means=rng.normal(size=(P, 3)).astype(np.float32), v_sh=rng.random((P, 16, 3)).astype(np.float32))
    return params, state, accum, count, normals


def _gpu(params, state, accum, count, normals, thresh=THRESH, dense=DENSE, min_op=MIN_OP, feat_bf16=False):
    dev = "cuda"
    t = {k: torch.as_tensor(v, device=dev).contiguous() for k, v in params.items()}
    if feat_bf16:
        t["feat"] = t["feat"].to(torch.bfloat16)
    s = {k: torch.as_tensor(v, device=dev).contiguous() for k, v in state.items()}
    st = density.DensityStats(len(accum), dev)
    st.accum.copy_(torch.as_tensor(accum))
    st.count.copy_(torch.as_tensor(count))
    p2, s2, n = density.densify(t, s, st, torch.as_tensor(normals, device=dev), thresh, dense, min_op)
    torch.cuda.synchronize()
    return ({k: v.float().cpu().numpy() for k, v in p2.items()}, {k: v.cpu().numpy() for k, v in s2.items()}, n,
            t, s)


def _check(params, state, accum, count, normals, got_p, got_s, n, thresh=THRESH, dense=DENSE, min_op=MIN_OP):
    ref_p, ref_s, d = DN.densify(params, state, accum, count, normals, thresh, dense, min_op, precision="f32")
    assert n == ref_p["means"].shape[0]
    nk = int(((d == 0) | (d == 1)).sum() + (d == 1).sum())       # rows before the split children
    for k in params:
        g, r = got_p[k], ref_p[k]
        assert g.shape == r.shape, k
        if k == "means":
            assert np.array_equal(g[:nk], r[:nk])
            assert np.abs(g[nk:] - r[nk:]).max(initial=0) < 2e-6
        elif k == "log_scales":
            assert np.array_equal(g[:nk], r[:nk])
            assert np.abs(g[nk:] - r[nk:]).max(initial=0) < 1e-6
        else:
            assert np.array_equal(g, r), k
    for k in state:
        assert np.array_equal(got_s[k], ref_s[k]), k
    return d


@pytest.mark.parametrize("P", [1, 257, 5000, 200_000, 300_001])
def test_densify_matches_oracle(P):
    params, state, accum, count, normals = _inputs(P)
    got_p, got_s, n, _, _ = _gpu(params, state, accum, count, normals)
    d = _check(params, state, accum, count, normals, got_p, got_s, n)
    if P >= 5000:
        assert set(np.unique(d).tolist()) == {-1, 0, 1, 2}        # every branch taken
        d64 = DN.decide(None, params["log_scales"], None, params["opacity_logits"], accum, count, THRESH, DENSE,
                        MIN_OP)
        assert (d64 != d).sum() <= P // 10000                       # the FP64 definition agrees


@pytest.mark.parametrize("raw_handle", [False, True])
def test_densify_on_a_side_stream_while_the_current_stream_is_busy(raw_handle):
    # The inputs are written on the current stream, which is then kept busy;
    # densify runs on another stream (a torch stream or its raw handle) and
    # must see the finished inputs and return the right count and rows.
    P = 20_000
    params, state, accum, count, normals = _inputs(P, seed=4)
    dev = "cuda"
    src = {k: torch.as_tensor(v, device=dev).contiguous() for k, v in list(params.items()) + list(state.items())}
    src_a, src_c = torch.as_tensor(accum, device=dev), torch.as_tensor(count, device=dev)
    t = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}
    s = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in state.items()}
    st = density.DensityStats(P, dev)
    big = torch.randn(4096, 4096, device=dev)
    torch.cuda.synchronize()
    for _ in range(20):          # keep the current stream busy
        big = big @ big
        big = big / big.norm()
    # The inputs land (device to device, on the current stream) after the busy work.
    for k in t:
        t[k].copy_(src[k])
    for k in s:
        s[k].copy_(src[k])
    st.accum.copy_(src_a)
    st.count.copy_(src_c)
    side = torch.cuda.Stream()
    p2, s2, n = density.densify(t, s, st, torch.as_tensor(normals, device=dev), THRESH, DENSE, MIN_OP,
                                stream=side.cuda_stream if raw_handle else side)
    torch.cuda.synchronize()
    got_p = {k: v.float().cpu().numpy() for k, v in p2.items()}
    got_s = {k: v.cpu().numpy() for k, v in s2.items()}
    _check(params, state, accum, count, normals, got_p, got_s, n)


def test_densify_bf16_rows_are_copied_bitwise():
    params, state, accum, count, normals = _inputs(3000)
    got_p, _, n, t, _ = _gpu(params, state, accum, count, normals, feat_bf16=True)
    p64 = dict(params, feat=t["feat"].float().cpu().numpy())       # the bf16 values as the oracle's input
    ref_p, _, _ = DN.densify(p64, {}, accum, count, normals, THRESH, DENSE, MIN_OP, precision="f32")
    assert np.array_equal(got_p["feat"], ref_p["feat"])


def test_densify_every_access_width():
    """Streams whose rows take every access width of the scatter: 16-byte
    (SH), 8-byte (float32 pairs, four bf16), 4-byte (odd float32 widths,
    including one wider than a block pass of 256 units), 2-byte (three bf16);
    copies and optimiser state bit-exact against the oracle."""
    P = 3001
    params, state, accum, count, normals = _inputs(P, seed=5)
    rng = np.random.default_rng(11)
    params["pair"] = rng.normal(size=(P, 2)).astype(np.float32)
    params["wide"] = rng.normal(size=(P, 257)).astype(np.float32)
    state["s_pair"] = rng.normal(size=(P, 2)).astype(np.float32)
    state["s_wide"] = rng.normal(size=(P, 257)).astype(np.float32)
    dev = "cuda"
    t = {k: torch.as_tensor(v, device=dev).contiguous() for k, v in params.items()}
    bf = {"b3": torch.randn(P, 3, generator=torch.Generator().manual_seed(1)).to(torch.bfloat16),
          "b4": torch.randn(P, 4, generator=torch.Generator().manual_seed(2)).to(torch.bfloat16)}
    t.update({k: v.to(dev) for k, v in bf.items()})
    s = {k: torch.as_tensor(v, device=dev).contiguous() for k, v in state.items()}
    st = density.DensityStats(P, dev)
    st.accum.copy_(torch.as_tensor(accum))
    st.count.copy_(torch.as_tensor(count))
    p2, s2, n = density.densify(t, s, st, torch.as_tensor(normals, device=dev), THRESH, DENSE, MIN_OP)
    torch.cuda.synchronize()
    ref_in = dict(params, **{k: v.float().numpy() for k, v in bf.items()})
    ref_p, ref_s, d = DN.densify(ref_in, state, accum, count, normals, THRESH, DENSE, MIN_OP, precision="f32")
    assert n == ref_p["means"].shape[0] and set(np.unique(d).tolist()) == {-1, 0, 1, 2}
    for k in ("pair", "wide", "b3", "b4", "quats", "opacity_logits", "sh", "feat"):
        assert np.array_equal(p2[k].float().cpu().numpy(), ref_p[k]), k
    for k in state:
        assert np.array_equal(s2[k].cpu().numpy(), ref_s[k]), k


@pytest.mark.parametrize("case", ["all_pruned", "all_split", "all_cloned", "none_selected"])
def test_densify_degenerate_cases(case):
    P = 1000
    params, state, accum, count, normals = _inputs(P, seed=3)
    kw = dict(all_pruned=dict(min_op=1.0), all_split=dict(thresh=0.0, dense=0.0, min_op=0.0),
              all_cloned=dict(thresh=0.0, dense=1e9, min_op=0.0), none_selected=dict(thresh=1e9, min_op=0.0))[case]
    got_p, got_s, n, _, _ = _gpu(params, state, accum, count, normals, **kw)
    _check(params, state, accum, count, normals, got_p, got_s, n, **kw)
    assert n == dict(all_pruned=0, all_split=2 * P, all_cloned=2 * P, none_selected=P)[case]


def test_densify_empty_and_deterministic():
    params, state, accum, count, normals = _inputs(0)
    _, _, n, _, _ = _gpu(params, state, accum, count, normals)
    assert n == 0
    params, state, accum, count, normals = _inputs(20000, seed=4)
    a = _gpu(params, state, accum, count, normals)
    b = _gpu(params, state, accum, count, normals)
    assert a[2] == b[2]
    for k in a[0]:
        assert np.array_equal(a[0][k], b[0][k])


def test_reset_opacity_matches_oracle():
    rng = np.random.default_rng(1)
    lg = rng.normal(-3.0, 3.0, 100_003).astype(np.float32)
    t = torch.as_tensor(lg, device="cuda")
    density.reset_opacity(t, 0.01)
    got = t.cpu().numpy()
    ref = DN.reset_opacity(lg, 0.01)
    below = lg < np.float32(np.log(0.01 / 0.99))
    assert below.sum() > 1000 and (~below).sum() > 1000
    assert np.array_equal(got[below], lg[below])
    assert np.array_equal(got[~below], ref[~below].astype(np.float32))


def test_screen_grad_stats_match_oracle_over_two_views():
    sc, cam, df = deformed_case(P=1500, W=96, H=72, D=32, seed=7)
    W, H = cam.width, cam.height
    pix = O.all_pixels(W, H)
    stats = density.DensityStats(sc.P)
    acc, cnt = None, None
    risky = np.zeros(sc.P, bool)
    for view, t in enumerate((0.4, 0.7)):
        run = gpu_forward(sc, cam, df, t=t)
        fl = O.render(sc, cam, df, t=t)["flags"]
        rng = np.random.default_rng(view)
        G = dict(rgb=rng.normal(size=(len(pix), 3)), feat=rng.normal(size=(len(pix), sc.D)))
        G["rgb"][fl != 0] = 0
        G["feat"][fl != 0] = 0
        gpu_backward(run, t, G["rgb"], None, None, G["feat"])
        stats.record(run.rast)
        ref = O.backward(sc, cam, df, t, (0.0, 0.0, 0.0), pix, G["rgb"], None, None, G["feat"], want_uv=True)
        g = O.gaussians(sc, cam, df, t=t)
        r = g["rect"]
        vis = (g["radius"] > 0) & (r[:, 0] <= W - 1) & (r[:, 2] >= 0) & (r[:, 1] <= H - 1) & (r[:, 3] >= 0) & \
            (r[:, 0] <= r[:, 2]) & (r[:, 1] <= r[:, 3])
        u, v, rad = g["uv"][:, 0], g["uv"][:, 1], g["radius"]
        near = lambda x: np.abs(x - np.round(x)) < 1e-4
        risky |= (g["gflags"] != 0) | (g["rmargin"] < 1e-5) | near(u - rad - 0.5) | near(u + rad - 0.5) | \
            near(v - rad - 0.5) | near(v + rad - 0.5)
        acc, cnt = DN.screen_grad_stats(ref["uv"], vis, W, H, acc, cnt)
    torch.cuda.synchronize()
    got_acc, got_cnt = stats.accum.cpu().numpy(), stats.count.cpu().numpy()
    ok = ~risky
    assert ok.sum() > 0.9 * sc.P and (cnt[ok] == 2).sum() > 100 and (cnt[ok] == 0).sum() > 10
    assert np.array_equal(got_cnt[ok], cnt[ok])
    assert rel_err(got_acc[ok], acc[ok]) < TOL_GRAD_REL
