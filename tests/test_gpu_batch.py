"""GPU checks of the batched multi-view form (fe_render_batch /
fe_render_batch_backward): views of mixed resolution and time, their
compositing as one persistent launch over (view, tile) work items, the
gradients summed over the views, the whole step captured in one CUDA graph.

* Images and summed gradients equal, bit for bit, the per-view renders with
  the same options, summed in view order.
* The summed gradients match the FP64 oracle's sum over the views, every
  pixel and every Gaussian compared (decisions as the GPU took them).
* The forward batch size and the autotuned tile shapes leave every image
  unchanged.
* A staging wait that gives up (the wait_polls test hook) is reported as
  FE_ERR_TIMEOUT, faults nothing, and the next call is clean."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2503_06161_gb300 import _lib, synth  # noqa: E402
from paper_2503_06161_gb300.batch import Autotuner, BatchRenderer, View  # noqa: E402
from paper_2503_06161_gb300.raster import DeformField, GaussianScene, Rasterizer, camera_struct  # noqa: E402

from gpu_helpers import (GRAD_KEYS, TOL_GRAD_REL, GpuRun, check_forward, forward_parity, rel_err,  # noqa: E402
                         _row_err)

TIMEOUT = 6


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


def _images(br):
    return [[x.clone() for x in b["out"]] for b in br.bufs]


TILES = [(16, 16), (32, 8), (8, 32), (16, 16)]


def _six_views(sc, df, cams, ts):
    # Two more views: helper streams then hold two views each.
    rng = np.random.default_rng(41)
    return cams + [synth.make_camera(96, 64, 80.0, rotation=synth.random_rotation(rng, 0.05)),
                   synth.make_camera(150, 100, 120.0, translation=[0.05, 0.0, 0.02])], ts + [0.5, 0.9]


@pytest.mark.parametrize("nviews", [4, 6])
def test_batch_equals_per_view_renders_bitwise(nviews):
    sc, df, cams, ts = _case()
    if nviews == 6:
        cams, ts = _six_views(sc, df, cams, ts)
    tiles = (TILES + TILES)[:nviews]
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, deform, views, None, fwd_batch=64, tiles=tiles)
    br.capture()
    br.replay()
    torch.cuda.synchronize()
    assert br.device_errors() == 0
    got = {k: v.clone() for k, v in br.grads.items()}
    imgs = _images(br)
    # Replaying again gives the same bits (view 0 overwrites the sums).
    br.replay()
    torch.cuda.synchronize()
    for k in got:
        assert torch.equal(got[k], br.grads[k]), k
    # The per-view calls with the same options; gradients summed in the
    # batch's fixed order: helper stream i adds views i, i + S, ... (S =
    # min(4, V)), then the stream sums in order.
    P, D = sc.P, sc.D
    S = min(4, nviews)
    parts = [{k: torch.empty_like(v) for k, v in got.items()} for _ in range(S)]
    for k, (v, b) in enumerate(zip(views, br.bufs)):
        r = Rasterizer(P, D, v.cam.width, v.cam.height, tile=tiles[k], max_dups=br.caps[k], auto_grow=False,
                       fwd_batch=64, accumulate=k >= S)
        out = r.forward(scene, v.cam, deform, v.t)
        for x, y in zip(out, imgs[k]):
            assert torch.equal(x, y), k
        r.backward(scene, v.cam, deform, v.t, b["g_rgb"], None, None, b["g_feat"], grads=parts[k % S])
    ref = {k: parts[0][k].clone() for k in got}
    for p_ in parts[1:]:
        for k in ref:
            ref[k] = ref[k] + p_[k]
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(ref[k], got[k]), k


def test_batch_d256_equals_per_view_renders_bitwise():
    # D = 256 runs as two channel-half passes, in the batch as two
    # persistent launches per direction.
    sc, df, cams, ts = _case(P=1500, D=256, seed=8)
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=True)
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, deform, views, None, fwd_batch=32, tiles=TILES)
    br.run()
    torch.cuda.synchronize()
    assert br.device_errors() == 0
    got = {k: v.clone() for k, v in br.grads.items()}
    ref = {k: torch.empty_like(v) for k, v in got.items()}
    for k, (v, b) in enumerate(zip(views, br.bufs)):
        r = Rasterizer(sc.P, sc.D, v.cam.width, v.cam.height, tile=TILES[k], max_dups=br.caps[k], auto_grow=False,
                       fwd_batch=32, accumulate=k > 0)
        out = r.forward(scene, v.cam, deform, v.t)
        for x, y in zip(out, b["out"]):
            assert torch.equal(x, y), k
        r.backward(scene, v.cam, deform, v.t, b["g_rgb"], None, None, b["g_feat"], grads=ref)
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(ref[k], got[k]), k


def test_batch_sum_matches_oracle_sum_over_views():
    # Every pixel of every view is compared (forward_parity), the oracle's
    # reverse of each view takes the decisions the GPU took, and a Gaussian
    # with a near-threshold gradient-only decision in a view is compared with
    # the sum in which that view's decision goes the way closest to the GPU.
    sc, df, cams, ts = _case(P=2000, seed=3)
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, deform, views, None, tiles=TILES)
    br.run()
    torch.cuda.synchronize()
    assert br.device_errors() == 0
    got = {k: br.grads[k].cpu().numpy().astype(np.float64) for k in GRAD_KEYS}
    base, alts = None, []
    for cam, t, v, b in zip(cams, ts, views, br.bufs):
        H, W = cam.height, cam.width
        HW = H * W
        run = GpuRun(None, None, None, None, b["out"][0].cpu().numpy().reshape(3, HW).T.copy(),
                     b["out"][1].cpu().numpy().reshape(HW), b["out"][2].cpu().numpy().reshape(HW),
                     b["out"][3].cpu().numpy())
        e, rep, flip = forward_parity(run, sc, cam, df, t=t)
        check_forward(e, rep, flagged_max=int(0.03 * HW) + 4)
        pix = O.all_pixels(W, H)
        G = dict(g_rgb=b["g_rgb"].cpu().numpy().reshape(3, HW).T, g_feat=b["g_feat"].cpu().numpy())
        r0 = O.backward(sc, cam, df, t, (0, 0, 0), pix, flip=flip, **G)
        base = r0 if base is None else {k: base[k] + r0[k] for k in GRAD_KEYS}
        gnd = O.gaussians(sc, cam, df, t=t)["gndec"]
        if (gnd > 0).any():
            r1 = O.backward(sc, cam, df, t, (0, 0, 0), pix, flip=flip, gflip=(gnd > 0).astype(np.uint64), **G)
            alts.append((gnd > 0, {k: r1[k] - r0[k] for k in GRAD_KEYS}))
    chosen = {k: base[k].copy() for k in GRAD_KEYS}
    for near, delta in alts:
        cand = {k: chosen[k] + delta[k] for k in GRAD_KEYS}
        s0 = np.max([_row_err(got[k], chosen[k]) for k in GRAD_KEYS], axis=0)
        s1 = np.max([_row_err(got[k], cand[k]) for k in GRAD_KEYS], axis=0)
        take = near & (s1 < s0)
        for k in GRAD_KEYS:
            chosen[k][take] = cand[k][take]
    errs = {k: rel_err(got[k], chosen[k]) for k in GRAD_KEYS}
    print("batch sum grad errors", errs, "views with near gradient decisions", len(alts))
    for k, e in errs.items():
        assert e <= TOL_GRAD_REL, (k, e)


def test_forward_batch_size_is_result_neutral():
    sc, df, cams, ts = _case(seed=1)
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=True)
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, deform, views, None, fwd_batch=32, tiles=TILES)
    results = []
    for B in (32, 64, 128):
        br.set_fwd_batch(B)
        br.run()
        torch.cuda.synchronize()
        assert br.device_errors() == 0
        results.append((_images(br), {k: v.clone() for k, v in br.grads.items()}))
    for imgs, grads in results[1:]:
        for a, b in zip(imgs, results[0][0]):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
        for k in grads:
            assert torch.equal(grads[k], results[0][1][k]), k


def test_autotuner_choice_is_result_neutral():
    # The images (hence the losses) do not depend on the tile shape or the
    # forward batch size; the gradients are sums over tiles, so their
    # rounding may depend on the tile shape.
    sc, df, cams, ts = _case(seed=1)
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=True)
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    tuner = Autotuner()
    tuned = BatchRenderer(scene, deform, views, tuner)
    plain = BatchRenderer(scene, deform, views, None)
    assert all(s in ((16, 16), (32, 8), (8, 32)) for s in tuned.tile_shapes)
    assert tuned.fwd_batch in (32, 64, 128)
    print("autotuner", tuned.tile_shapes, tuned.fwd_batch, tuner.timings)
    tuned.run()
    plain.run()
    torch.cuda.synchronize()
    for a, b in zip(_images(tuned), _images(plain)):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    assert torch.equal(tuned.losses, plain.losses)
    for k in tuned.grads:
        assert rel_err(tuned.grads[k].cpu().numpy(), plain.grads[k].cpu().numpy()) <= 1e-4, k


def test_batch_wait_that_gives_up_reports_timeout_and_recovers():
    sc, df, cams, ts = _case(P=1500, seed=4)
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, deform, views, None, tiles=TILES)
    br.run()
    torch.cuda.synchronize()
    good = _images(br)
    good_g = {k: v.clone() for k, v in br.grads.items()}
    br.set_wait_polls(-1)          # every staging wait gives up at once
    br.forward()
    rc, st = br.stats()
    assert rc == TIMEOUT and all(s["device_errors"] & 2 for s in st)
    br.backward()
    rc, st = br.stats()
    assert rc == TIMEOUT
    br.set_wait_polls(0)
    br.run()
    rc, st = br.stats()
    assert rc == 0 and all(s["device_errors"] == 0 for s in st)
    for a, b in zip(_images(br), good):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    for k in good_g:
        assert torch.equal(br.grads[k], good_g[k]), k


def test_single_view_wait_that_gives_up_reports_timeout_and_recovers():
    sc, df, cams, ts = _case(P=1500, seed=5)
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    cam = camera_struct(cams[0])
    good = Rasterizer(sc.P, sc.D, cam.width, cam.height, max_dups=64 * sc.P, auto_grow=False)
    ref = [x.clone() for x in good.forward(scene, cam, deform, 0.3)]
    g_rgb = torch.full((3, cam.height, cam.width), 1e-2, device="cuda")
    ref_g = {k: v.clone() for k, v in good.backward(scene, cam, deform, 0.3, g_rgb).items()}
    bad = Rasterizer(sc.P, sc.D, cam.width, cam.height, max_dups=64 * sc.P, auto_grow=False, wait_polls=-1,
                     workspace=good.workspace)
    bad.forward(scene, cam, deform, 0.3)
    st = bad.stats(raise_on_error=False)
    assert st["status"] == TIMEOUT and st["device_errors"] & 2
    bad.backward(scene, cam, deform, 0.3, g_rgb)
    assert bad.stats(raise_on_error=False)["status"] == TIMEOUT
    out = good.forward(scene, cam, deform, 0.3)
    g = good.backward(scene, cam, deform, 0.3, g_rgb)
    assert good.stats(raise_on_error=False)["status"] == 0
    for x, y in zip(out, ref):
        assert torch.equal(x, y)
    for k in ref_g:
        assert torch.equal(g[k], ref_g[k]), k


def test_render_makes_no_host_read_after_the_first_forward():
    # After the first forward has sized the list, forwards are capturable in
    # a CUDA graph: a host read (a stream synchronisation) inside the
    # capture would fail it.
    sc, df, cams, ts = _case(P=1500, seed=6)
    scene = GaussianScene.from_numpy(sc, "cuda")
    deform = DeformField.from_numpy(df, "cuda")
    cam = camera_struct(cams[0])
    rast = Rasterizer(sc.P, sc.D, cam.width, cam.height)
    out = rast.forward(scene, cam, deform, 0.2)
    ref = [x.clone() for x in out]
    for x in out:
        x.zero_()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            rast.forward(scene, cam, deform, 0.2, out=out)
    torch.cuda.current_stream().wait_stream(s)
    graph.replay()
    torch.cuda.synchronize()
    rast.check()
    for x, y in zip(out, ref):
        assert torch.equal(x, y)


def test_batch_rejects_bad_arguments():
    sc, df, cams, ts = _case(P=500, seed=2)
    scene = GaussianScene.from_numpy(sc, "cuda")
    views = _views(sc, cams, ts)
    br = BatchRenderer(scene, None, views, None, tiles=TILES)
    g = scene.struct()
    bad = _lib.make_batch([v.cam for v in views], [v.t for v in views],
                          [_lib.make_opts(max_dups=c, fwd_batch=48) for c in br.caps])
    with pytest.raises(_lib.FeError) as e:
        _lib.fe_render_batch(g, None, bad, br.workspace, [b["out"] for b in br.bufs])
    assert e.value.code == 4
    small = br.workspace[:1024]
    with pytest.raises(_lib.FeError) as e:
        _lib.fe_render_batch(g, None, br.batch, small, [b["out"] for b in br.bufs])
    assert e.value.code == 3


def test_ordered_sum_on_the_gpu_matches_the_host_sum_bitwise():
    # The exchange's fixed-order sum (fe_sum_f32, eight sources a call) gives
    # the bits of the host's left-to-right float32 sum.
    from paper_2503_06161_gb300 import dist as pdist
    rng = np.random.default_rng(1)
    host = [torch.tensor(rng.normal(size=100_003).astype(np.float32)) for _ in range(11)]
    out_h = torch.empty(100_003)
    pdist.ordered_sum(host, out_h)
    dev = [x.cuda() for x in host]
    out_d = torch.empty(100_003, device="cuda")
    pdist.ordered_sum(dev, out_d)
    torch.cuda.synchronize()
    assert torch.equal(out_d.cpu(), out_h)
