"""GPU checks of the batched multi-view form: views of mixed resolution and
time rendered forward and backward in one CUDA-graph launch, gradients summed
over the views.  The autotuned tile shapes must not change any result; the
summed gradients match (bit for bit) the per-view renders summed in the same
order, and the oracle's sum over views within the gradient bar."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2503_06161_gb300 import synth  # noqa: E402
from paper_2503_06161_gb300.batch import Autotuner, BatchRenderer, View  # noqa: E402
from paper_2503_06161_gb300.raster import DeformField, GaussianScene, Rasterizer, camera_struct  # noqa: E402

from gpu_helpers import TOL_GRAD_REL, rel_err  # noqa: E402


def _case(P=3000, D=32, seed=0):
    rng = np.random.default_rng(seed + 7)
    sc = synth.make_scene(P, D, (-1.2, -0.8, 2.0), (1.2, 0.8, 4.5), seed=seed)
    df = synth.make_deform(P, C=32, R=16, bbox_min=(-1.5, -1.0, 1.5), bbox_max=(1.5, 1.0, 5.0), full_heads=True,
                           head_std=0.02, seed=seed + 1)
    cams, ts = [], []
    for k, (W, H, f) in enumerate([(150, 100, 120.0), (75, 50, 60.0), (150, 100, 120.0), (72, 56, 60.0)]):
        cams.append(synth.make_camera(W, H, f, rotation=synth.random_rotation(rng, 0.05),
                                      translation=[0.02 * k, -0.01, 0.05]))
        ts.append(k / 3.0)
    return sc, df, cams, ts


def _views(sc, cams, ts, dev="cuda"):
    rng = np.random.default_rng(11)
    views = []
    for cam, t in zip(cams, ts):
        H, W = cam.height, cam.width
        views.append(View(camera_struct(cam), t, torch.tensor(rng.random((3, H, W)).astype(np.float32)).to(dev),
                          torch.tensor(rng.normal(size=(H * W, sc.D)).astype(np.float32)).to(dev)))
    return views


def test_batched_graph_matches_per_view_sum_and_oracle():
    sc, df, cams, ts = _case()
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, deform, views, Autotuner(), streams=2)
    assert br.S == 2
    br.capture()
    br.replay()
    torch.cuda.synchronize()
    assert br.device_errors() == 0
    got = {k: v.clone() for k, v in br.grads.items()}
    # Replaying again gives the same bits (the first view overwrites).
    br.replay()
    torch.cuda.synchronize()
    for k in got:
        assert torch.equal(got[k], br.grads[k]), k
    # Per-view renders with the same tile shapes, summed in the batch's
    # order: within each stream in view order, then the streams in order.
    per_stream = [None] * br.S
    for k, (v, b, shape) in enumerate(zip(views, br.bufs, br.tile_shapes)):
        r = Rasterizer(sc.P, sc.D, v.cam.width, v.cam.height, tile=shape, auto_grow=True)
        r.forward(scene, v.cam, deform, v.t)
        g = r.backward(scene, v.cam, deform, v.t, b["g_rgb"], None, None, b["g_feat"])
        s = br.stream_of[k]
        per_stream[s] = ({n: x.clone() for n, x in g.items()} if per_stream[s] is None
                         else {n: per_stream[s][n] + g[n] for n in g})
    ref = per_stream[0]
    for s in range(1, br.S):
        ref = {n: ref[n] + per_stream[s][n] for n in ref}
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(ref[k], got[k]), k
    # Oracle: the per-view upstream gradients with the oracle's flagged
    # (undecided) pixels zeroed, back-propagated by the GPU view by view and
    # by the FP64 oracle, each summed over the views; Gaussians flagged in
    # any view are left out of the comparison.
    gpu_sum, ora_sum, flagged = None, None, np.zeros(sc.P, bool)
    for cam, t, v, b in zip(cams, ts, views, br.bufs):
        H, W = cam.height, cam.width
        pix = O.all_pixels(W, H)
        ok = O.render(sc, cam, df, t=t)["flags"] == 0
        g_rgb = b["g_rgb"].cpu().numpy().reshape(3, H * W).T * ok[:, None]
        g_feat = b["g_feat"].cpu().numpy() * ok[:, None]
        G = O.backward(sc, cam, df, t, (0, 0, 0), pix, g_rgb, None, None, g_feat)
        r = Rasterizer(sc.P, sc.D, W, H, auto_grow=True)
        r.forward(scene, v.cam, deform, v.t)
        g = r.backward(scene, v.cam, deform, v.t, torch.tensor(g_rgb.T.reshape(3, H, W), dtype=torch.float32).cuda(),
                       None, None, torch.tensor(g_feat, dtype=torch.float32).cuda())
        g = {k: x.cpu().numpy().astype(np.float64) for k, x in g.items()}
        gpu_sum = g if gpu_sum is None else {k: gpu_sum[k] + g[k] for k in g}
        ora_sum = G if ora_sum is None else {k: ora_sum[k] + G[k] for k in G}
        flagged |= O.gaussians(sc, cam, df, t=t)["gflags"] != 0
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "feat"):
        e = rel_err(gpu_sum[k][~flagged], ora_sum[k][~flagged])
        assert e <= TOL_GRAD_REL, (k, e)


def test_autotuner_choice_is_result_neutral():
    # The images (hence the losses) do not depend on the tile shape; the
    # gradients are sums over tiles, so their rounding may.
    sc, df, cams, ts = _case(seed=1)
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=True)
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    tuned = BatchRenderer(scene, deform, views, Autotuner())
    plain = BatchRenderer(scene, deform, views, None)
    assert all(s in ((16, 16), (32, 8), (8, 32)) for s in tuned.tile_shapes)
    tuned.run()
    a = {k: v.clone() for k, v in tuned.grads.items()}
    la = tuned.losses.clone()
    plain.run()
    torch.cuda.synchronize()
    for k in a:
        assert rel_err(a[k].cpu().numpy(), plain.grads[k].cpu().numpy()) <= 1e-4, k
    assert torch.equal(la, plain.losses)


def test_streams_do_not_change_images_and_sum_within_rounding():
    sc, df, cams, ts = _case(seed=2)
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    one = BatchRenderer(scene, deform, views, None, streams=1)
    four = BatchRenderer(scene, deform, views, None, streams=4)
    one.capture()
    four.capture()
    one.replay()
    four.replay()
    torch.cuda.synchronize()
    assert torch.equal(one.losses, four.losses)
    for k in one.grads:
        assert rel_err(four.grads[k].cpu().numpy(), one.grads[k].cpu().numpy()) <= 1e-5, k
