"""GPU parity of the tensor-core decoder (Sec. 3.3, loss of Eq. 10) against the
FP64 oracle, through the C ABI.

Inputs are rounded to bf16 first and the oracle consumes the rounded values,
so the comparison measures only the kernel's FP32 accumulation.  The L1
gradient takes a sign decision per element: elements whose FP64 margin
|out - target| is below MARGIN are counted; pixels holding one are left out
of the d_feat comparison and the weight/bias gradients get the largest
change those decisions can make added to their bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2503_06161_gb300 import synth  # noqa: E402
from paper_2503_06161_gb300.decoder import Decoder  # noqa: E402

from gpu_helpers import rel_err  # noqa: E402

MARGIN = 1e-5      # FP32 accumulation error of <= 64 bf16 products + bias: ~1e-6 at these magnitudes
TOL_OUT = 1e-5     # relative to max(|ref|, rms)
TOL_GRAD = 1e-3


def _inputs(HW, D, seed=0, b_std=0.1, target_dtype=torch.bfloat16):
    rng = np.random.default_rng(seed)
    feat = synth.bf16_round(rng.normal(0.0, 1.0, (HW, D)).astype(np.float32))
    w, b = synth.make_decoder(D, seed=seed + 1, b_std=b_std)
    tgt = rng.normal(0.0, 1.0, (HW, 256)).astype(np.float32)
    if target_dtype == torch.bfloat16:
        tgt = synth.bf16_round(tgt)
    dec = Decoder(torch.tensor(w).to(torch.bfloat16).cuda(), torch.tensor(b).cuda())
    ft = torch.tensor(feat).to(torch.bfloat16).cuda()
    tt = torch.tensor(tgt).to(target_dtype).cuda()
    return feat, w, b, tgt, dec, ft, tt


def _l1_check(feat, w, b, tgt, got, rows=None):
    """Compare (loss, d_feat, d_w, d_b) with the oracle; returns the number of
    undecided sign elements."""
    HW = feat.shape[0]
    out = O.decoder_forward(feat, w, b)
    loss, dout = O.l1_loss_and_grad(out, tgt)
    dfeat, dw, db = O.decoder_backward(feat, w, dout)
    g_loss, g_dfeat, g_dw, g_db = (x.cpu().numpy().astype(np.float64) for x in got)
    assert abs(g_loss[0] - loss) <= 1e-5 * abs(loss)
    undecided = np.abs(out - tgt) < MARGIN
    n_und = int(undecided.sum())
    ok_rows = ~undecided.any(1)
    if rows is not None:
        ok_rows &= np.isin(np.arange(HW), rows)
    assert rel_err(g_dfeat[ok_rows], dfeat[ok_rows]) <= TOL_GRAD
    # Largest change of dW / db the undecided elements can make: 2/HW each.
    p_idx, c_idx = np.nonzero(undecided)
    corr_w = np.zeros_like(dw)
    np.add.at(corr_w, c_idx, 2.0 / HW * np.abs(feat[p_idx]))
    corr_b = np.bincount(c_idx, minlength=256) * 2.0 / HW
    for g, r, corr in ((g_dw, dw, corr_w), (g_db, db, corr_b)):
        scale = max(np.sqrt(np.mean(r ** 2)), 1e-30)
        bound = TOL_GRAD * np.maximum(np.abs(r), scale) + corr
        assert np.all(np.abs(g - r) <= bound), float(np.max(np.abs(g - r) / np.maximum(np.abs(r), scale)))
    return n_und


@pytest.mark.parametrize("D", [16, 32, 64, 128])
def test_decoder_forward_matches_oracle(D):
    HW = 1000  # 7 full 128-pixel tiles and a ragged tail of 104
    feat, w, b, tgt, dec, ft, tt = _inputs(HW, D)
    out = dec.forward(ft)
    torch.cuda.synchronize()
    assert dec.errors() == 0
    ref = O.decoder_forward(feat, w, b)
    assert rel_err(out.cpu().numpy(), ref) <= TOL_OUT


@pytest.mark.parametrize("D,tdtype", [(16, torch.bfloat16), (32, torch.bfloat16), (64, torch.bfloat16),
                                      (128, torch.bfloat16), (16, torch.float32), (32, torch.float32),
                                      (64, torch.float32), (128, torch.float32)])
def test_decoder_l1_matches_oracle(D, tdtype):
    HW = 1000
    feat, w, b, tgt, dec, ft, tt = _inputs(HW, D, seed=D, target_dtype=tdtype)
    got = dec.l1(ft, tt)
    torch.cuda.synchronize()
    assert dec.errors() == 0
    n_und = _l1_check(feat, w, b, tgt, got)
    assert n_und <= 1e-4 * HW * 256  # ~2 * MARGIN * density of out - target near 0


@pytest.mark.parametrize("D", [16, 32, 128])
def test_decoder_l1_many_tiles_per_cta(D):
    # More tiles than SMs: every CTA walks several tiles, so the weight and
    # bias gradients accumulate across tiles in tensor memory.
    HW = 128 * 400 + 77
    feat, w, b, tgt, dec, ft, tt = _inputs(HW, D, seed=5)
    got = dec.l1(ft, tt)
    torch.cuda.synchronize()
    assert dec.errors() == 0
    _l1_check(feat, w, b, tgt, got)


def test_decoder_full_size_config():
    # The 640x512 feature map of the BF16 workload, D=32 -> 256, bf16 targets.
    HW = 640 * 512
    feat, w, b, tgt, dec, ft, tt = _inputs(HW, 32, seed=11, b_std=0.0)
    got = dec.l1(ft, tt)
    torch.cuda.synchronize()
    assert dec.errors() == 0
    rows = np.random.default_rng(0).choice(HW, 4096, replace=False)
    n_und = _l1_check(feat, w, b, tgt, got, rows=rows)
    assert n_und < 1e-4 * HW * 256
    out = dec.forward(ft)
    ref = O.decoder_forward(feat[rows], w, b)
    assert rel_err(out[torch.tensor(rows).cuda()].cpu().numpy(), ref) <= TOL_OUT


def test_decoder_deterministic_and_empty():
    HW = 3000
    feat, w, b, tgt, dec, ft, tt = _inputs(HW, 64, seed=3)
    a = [x.clone() for x in dec.l1(ft, tt)]
    c = dec.l1(ft, tt)
    torch.cuda.synchronize()
    for x, y in zip(a, c):
        assert torch.equal(x, y)
    e = dec.l1(ft[:0], tt[:0])
    torch.cuda.synchronize()
    assert e[0].item() == 0.0 and not e[2].any() and not e[3].any()


def test_render_writes_bf16_feature_map_for_the_decoder():
    # The compositing pass's optional bf16 copy of the feature map is the
    # nearest-even rounding of its fp32 map (numpy rounding, bit for bit),
    # and feeding it to the fused decoder loss matches the oracle decoder on
    # those same bf16 values.
    from gpu_helpers import deformed_case
    from paper_2503_06161_gb300.raster import DeformField, GaussianScene, Rasterizer, camera_struct
    sc, cam, df = deformed_case(P=3000, W=150, H=100, D=32)
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=True)
    deform = DeformField.from_numpy(df, "cuda")
    rast = Rasterizer(sc.P, sc.D, cam.width, cam.height, auto_grow=True)
    fb = torch.empty(cam.width * cam.height, sc.D, dtype=torch.bfloat16, device="cuda")
    _, _, _, feat = rast.forward(scene, camera_struct(cam), deform, 0.3, feat_bf16=fb)
    torch.cuda.synchronize()
    f32 = feat.cpu().numpy()
    got_bits = fb.cpu().view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got_bits, synth.bf16_bits(f32))
    w, b = synth.make_decoder(sc.D, seed=4, b_std=0.1)
    dec = Decoder(torch.tensor(w).to(torch.bfloat16).cuda(), torch.tensor(b).cuda())
    tgt = synth.bf16_round(np.random.default_rng(1).normal(size=(f32.shape[0], 256)).astype(np.float32))
    got = dec.l1(fb, torch.tensor(tgt).to(torch.bfloat16).cuda())
    torch.cuda.synchronize()
    _l1_check(synth.bf16_round(f32).astype(np.float64), w, b, tgt, got)
