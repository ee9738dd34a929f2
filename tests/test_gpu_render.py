"""GPU parity of the FE-4DGS pass against the FP64 oracle, through the C ABI.

Forward: RGB and depth within 1e-4 absolute, features within 1e-4 relative,
on EVERY pixel: a pixel whose oracle decisions are within rounding distance
of a threshold is compared with the oracle result of the branch the GPU
took (each branch is a correct result), and the flagged count stays within
its measured bound.  Integer stage: keys, per-entry Gaussian ids and tile
ranges bit-exact.  Reverse: gradients of EVERY Gaussian within 1e-3
relative of the oracle's analytic FP64 gradients (decisions as the GPU took
them) and 1e-2 of central finite differences of the oracle forward."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2503_06161_gb300 import synth, _lib
from tests.gpu_helpers import (TOL_FD_REL, TOL_FEAT_REL, TOL_RGB_ABS, check_forward, check_grads, deformed_case,
                               forward_parity, gpu_backward, gpu_forward, grad_parity, pixel_index, rel_err)

pytestmark = pytest.mark.gpu


# --------------------------------------------------------------------------
# Integer stage: bit-exact keys / values / ranges
# --------------------------------------------------------------------------

def _tile_bin_gpu(uv, radius, depth, W, H, tile):
    P = len(radius)
    opts = _lib.make_opts(tile=tile, max_dups=max(16, int(4 * P * 64)))
    nbytes = _lib.fe_workspace_size(P, 16, W, H, opts)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)
    _lib.fe_tile_bin(t(uv, torch.float32), t(radius, torch.int32), t(depth, torch.float32), W, H, opts, ws)
    st = _lib.fe_read_stats(ws, P, 16, W, H, opts)
    K = st["num_dups"]
    tiles = ((W + tile[0] - 1) // tile[0]) * ((H + tile[1] - 1) // tile[1])
    keys = torch.zeros(max(K, 1), dtype=torch.int64, device="cuda")
    gauss = torch.zeros(max(K, 1), dtype=torch.int32, device="cuda")
    ranges = torch.zeros(tiles, 2, dtype=torch.int32, device="cuda")
    _lib.fe_debug_dump(ws, P, 16, W, H, opts, keys=keys, gauss=gauss, ranges=ranges)
    torch.cuda.synchronize()
    return (keys[:K].cpu().numpy().view(np.uint64), gauss[:K].cpu().numpy().view(np.uint32),
            ranges.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32)])
def test_tile_bin_bit_exact_random(tile):
    rng = np.random.default_rng(21)
    W, H, P = 203, 157, 6000
    uv = np.c_[rng.uniform(-40, W + 40, P), rng.uniform(-40, H + 40, P)].astype(np.float32)
    radius = rng.integers(-2, 40, P).astype(np.int32)
    depth = rng.uniform(0.5, 10, P).astype(np.float32)
    depth[100:400] = depth[100]          # exact ties: order by index
    uv[50] = np.nan                      # non-finite centre: culled
    keys, gauss, ranges = _tile_bin_gpu(uv, radius, depth, W, H, tile)
    k_ref, v_ref, r_ref = O.tile_bin(uv, radius, depth, W, H, *tile)
    assert len(keys) == len(k_ref)
    assert np.array_equal(keys, k_ref)
    assert np.array_equal(gauss, v_ref)
    assert np.array_equal(ranges, r_ref)


def test_tile_bin_bit_exact_endonerf_scene():
    # Binary32 projected inputs of the 200k-Gaussian 640x512 workload, from
    # the oracle's FP64 projection rounded to binary32.
    sc, cam, df = synth.config_inputs("endonerf_200k_640x512")
    g = O.gaussians(sc, cam, df, t=0.5, geps=None)
    uv = g["uv"].astype(np.float32)
    keys, gauss, ranges = _tile_bin_gpu(uv, g["radius"], g["depth"].astype(np.float32), cam.width, cam.height,
                                        (16, 16))
    k_ref, v_ref, r_ref = O.tile_bin(uv, g["radius"], g["depth"].astype(np.float32), cam.width, cam.height, 16, 16)
    assert len(keys) == len(k_ref) > 1_000_000
    assert np.array_equal(keys, k_ref)
    assert np.array_equal(gauss, v_ref)
    assert np.array_equal(ranges, r_ref)


# --------------------------------------------------------------------------
# Forward parity
# --------------------------------------------------------------------------

def test_forward_static_1k_64x64():
    # Three pixels carry an alpha-skip decision within 1e-4 of 1/255; they
    # are checked against the branch the GPU took.
    sc, cam, _ = synth.config_inputs("static_1k_64x64")
    run = gpu_forward(sc, cam)
    e, rep, _ = forward_parity(run, sc, cam)
    check_forward(e, rep, flagged_max=4)


@pytest.mark.parametrize("D", [16, 32, 64, 128, 256])
def test_forward_deformed_ragged(D):
    # 192 of 15000 pixels flagged: 161 depth-order ties, 22 alpha skips, 11
    # terminations; all checked.
    sc, cam, df = deformed_case(D=D)
    bg = (0.1, 0.2, 0.3)
    run = gpu_forward(sc, cam, df, t=0.3, bg=bg)
    e, rep, _ = forward_parity(run, sc, cam, df, t=0.3, bg=bg)
    check_forward(e, rep, flagged_max=230)


def test_per_gaussian_state():
    sc, cam, df = deformed_case()
    run = gpu_forward(sc, cam, df, t=0.3)
    d = run.rast.dump()
    g = O.gaussians(sc, cam, df, t=0.3)
    vis = (g["radius"] > 0) & (d["touched"].cpu().numpy() > 0)
    rad = d["radius"].cpu().numpy()
    sure = vis & (g["rmargin"] > 1e-5)
    assert np.array_equal(rad[sure], g["radius"][sure])
    assert np.abs(d["uv"].cpu().numpy()[vis] - g["uv"][vis]).max() < 1e-3
    assert rel_err(d["conic"].cpu().numpy()[vis], g["conic"][vis]) < 1e-4
    assert np.abs(d["opacity"].cpu().numpy()[vis] - g["opacity"][vis]).max() < 1e-6
    assert rel_err(d["depth"].cpu().numpy()[vis], g["depth"][vis]) < 1e-6
    assert np.abs(d["rgb"].cpu().numpy()[vis] - g["rgb"][vis]).max() < 1e-5


def test_needle_thin_gaussians_conic_and_radius():
    # Scale ratio e^7 ~ 1100 with random rotations: the projected 2D
    # covariance is nearly rank one, a c ~ b^2 up to the 0.3 px^2 dilation,
    # so the determinant a c - b^2 cancels by a factor kappa = (a c + b^2) /
    # det of up to ~2e3.  Each conic entry must match the FP64 oracle within
    # 64 kappa u (u = 2^-24): a, b and c are binary32 sums of nine products,
    # each within about 16 u of its exact value, and the determinant's
    # relative error is kappa times theirs; the compensated evaluation of
    # a c - b^2 itself adds at most 2 u (test_compensated_det).
    rng = np.random.default_rng(31)
    P, D = 600, 16
    sc = synth.make_scene(P, D, (-1.5, -1.2, 3.0), (1.5, 1.2, 6.0), seed=31)
    ls = np.full((P, 3), -8.0, np.float32)
    ls[:, 0] = -1.0
    sc = dataclasses.replace(sc, log_scales=ls + rng.normal(0, 0.05, (P, 3)).astype(np.float32))
    cam = synth.make_camera(320, 256, 280.0)
    run = gpu_forward(sc, cam)
    d = run.rast.dump()
    g = O.gaussians(sc, cam)
    vis = (g["radius"] > 0) & (d["touched"].cpu().numpy() > 0)
    assert vis.sum() > 300
    # the oracle conic (a, b, c) = inverse of the dilated covariance; its
    # determinant and the cancellation factor from the covariance entries
    ca, cb, cc = g["conic"][:, 0], g["conic"][:, 1], g["conic"][:, 2]
    det_conic = ca * cc - cb * cb
    A, B, C = cc / det_conic, -cb / det_conic, ca / det_conic          # covariance entries
    kappa = (A * C + B * B) / (A * C - B * B)
    assert np.median(kappa[vis]) > 100                                 # the case is ill-conditioned
    got = d["conic"].cpu().numpy()
    u = 2.0 ** -24
    scale = np.maximum(np.abs(g["conic"]), np.abs(g["conic"]).max(axis=1, keepdims=True))
    err = (np.abs(got - g["conic"]) / scale).max(axis=1)
    bound = 64 * kappa * u + 1e-6
    print("needle conic: max kappa", kappa[vis].max(), "max err / bound", (err[vis] / bound[vis]).max())
    assert np.all(err[vis] <= bound[vis])
    sure = vis & (g["rmargin"] > 1e-5)
    assert np.array_equal(d["radius"].cpu().numpy()[sure], g["radius"][sure])
    # (The images of such needles are not held to the 1e-4 bar of the other
    # cases: the quadratic form along the long axis cancels further, and the
    # binary32 render differs from FP64 by up to ~2e-3 in RGB there.)


def test_tile_lists_match_oracle_rects():
    # Each tile's list is the oracle's 3-sigma-square list in depth order,
    # less only Gaussians that blend at no pixel centre of the tile (the
    # projection cuts the square to the box of the alpha >= 1/255 ellipse):
    # every Gaussian whose FP64 alpha reaches 1/255 (with 0.1% to spare) at
    # some centre of the tile is listed, and nothing outside the square is.
    sc, cam, df = deformed_case()
    run = gpu_forward(sc, cam, df, t=0.3)
    d = run.rast.dump()
    g = O.gaussians(sc, cam, df, t=0.3)
    tw = th = 16
    tx_n, ty_n = (cam.width + tw - 1) // tw, (cam.height + th - 1) // th
    rect = g["rect"]
    # Gaussians whose binary32 rect or depth order may legitimately differ.
    u, v, r = g["uv"][:, 0], g["uv"][:, 1], g["radius"]

    def near_int(x):
        return np.abs(x - np.round(x)) < 1e-4

    risky = (g["rmargin"] < 1e-5) | near_int(u - r - 0.5) | near_int(u + r - 0.5) | near_int(v - r - 0.5) | \
        near_int(v + r - 0.5)
    keys = d["keys"].cpu().numpy().view(np.uint64)
    gauss = d["gauss"].cpu().numpy()
    ranges = d["ranges"].cpu().numpy()
    depth = g["depth"]
    ca, cb, cc = g["conic"][:, 0], g["conic"][:, 1], g["conic"][:, 2]
    op = g["opacity"]
    checked = blending = dropped = 0
    for ty in range(ty_n):
        for tx in range(tx_n):
            t = ty * tx_n + tx
            got = gauss[ranges[t, 0]:ranges[t, 1]].tolist()
            x0, x1 = tx * tw, min(cam.width, (tx + 1) * tw) - 1
            y0, y1 = ty * th, min(cam.height, (ty + 1) * th) - 1
            inside = (g["radius"] > 0) & (rect[:, 0] <= x1) & (rect[:, 2] >= x0) & (rect[:, 1] <= y1) & \
                (rect[:, 3] >= y0) & (rect[:, 0] <= rect[:, 2])
            ref = sorted(np.nonzero(inside)[0].tolist(), key=lambda i: (depth[i], i))
            a = [i for i in got if not risky[i]]
            b = [i for i in ref if not risky[i]]
            listed = set(a)
            assert listed <= set(b), f"tile {t}: listed outside the square"
            assert a == [i for i in b if i in listed], f"tile {t}: order"
            # Highest FP64 alpha over the tile's pixel centres of each square entry.
            px, py = np.meshgrid(np.arange(x0, x1 + 1) + 0.5, np.arange(y0, y1 + 1) + 0.5)
            for i in b:
                dx, dy = px - u[i], py - v[i]
                q = 0.5 * ca[i] * dx * dx + cb[i] * dx * dy + 0.5 * cc[i] * dy * dy
                amax = op[i] * np.exp(-q.min())
                if amax >= (1.0 + 1e-3) / 255.0:
                    blending += 1
                    assert i in listed, f"tile {t}: Gaussian {i} blends (alpha {amax:.4g}) but is not listed"
            dropped += len(b) - len(a)
            assert np.all((keys[ranges[t, 0]:ranges[t, 1]] >> np.uint64(32)) == t)
            checked += len(a)
    print("listed", checked, "blending", blending, "dropped from the square", dropped)
    assert checked > 5000 and blending > 5000


def test_tile_shape_invariance_bitwise():
    sc, cam, df = deformed_case()
    outs = [gpu_forward(sc, cam, df, t=0.3, tile=tile) for tile in [(16, 16), (32, 8), (8, 32)]]
    for o in outs[1:]:
        for k in ("rgb", "depth", "alpha", "feat"):
            assert np.array_equal(getattr(o, k), getattr(outs[0], k)), k


def test_forward_bf16_storage():
    sc, cam, df = deformed_case(seed=3)
    sc16 = dataclasses.replace(sc, sh=synth.bf16_round(sc.sh), feat=synth.bf16_round(sc.feat))
    run = gpu_forward(sc, cam, df, t=0.6, bf16=True)
    e, rep, _ = forward_parity(run, sc16, cam, df, t=0.6)
    check_forward(e, rep, flagged_max=170)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_forward_lower_sh_degree(deg):
    sc, cam, df = deformed_case(P=1500, seed=4)
    sc = dataclasses.replace(sc, sh_degree=deg)
    run = gpu_forward(sc, cam, df, t=0.2)
    e, rep, _ = forward_parity(run, sc, cam, df, t=0.2)
    check_forward(e, rep, flagged_max=18)


def test_forward_deform_c64():
    sc, cam, df = deformed_case(P=2000, C=64, R=8, seed=5)
    run = gpu_forward(sc, cam, df, t=0.9)
    e, rep, _ = forward_parity(run, sc, cam, df, t=0.9)
    check_forward(e, rep, flagged_max=85)


# --------------------------------------------------------------------------
# Reverse pass
# --------------------------------------------------------------------------

def _upstream(n, D, seed=0, mask=None):
    rng = np.random.default_rng(seed)
    g = dict(rgb=rng.normal(size=(n, 3)), depth=rng.normal(size=n) * 0.1, alpha=rng.normal(size=n),
             feat=rng.normal(size=(n, D)))
    if mask is not None:
        for k in g:
            g[k][~mask] = 0
    return g


@pytest.mark.parametrize("D,deform,flagged_max", [(16, False, 8), (32, True, 75), (64, True, 75), (128, True, 75),
                                                   (256, True, 75)])
def test_backward_matches_oracle(D, deform, flagged_max):
    # Upstream gradients on every pixel; the oracle's reverse takes each
    # flagged pixel's decisions as the GPU forward took them, and each
    # Gaussian's near-threshold gradient-only decisions as its GPU gradient
    # shows: no pixel and no Gaussian is left out.
    sc, cam, df = deformed_case(P=1500, W=96, H=72, D=D, seed=7)
    df = df if deform else None
    t, bg = 0.4, (0.2, 0.1, 0.3)
    run = gpu_forward(sc, cam, df, t=t, bg=bg)
    pix = O.all_pixels(cam.width, cam.height)
    e, rep, flip = forward_parity(run, sc, cam, df, t=t, bg=bg)
    check_forward(e, rep, flagged_max=flagged_max)
    G = _upstream(len(pix), D)
    got = gpu_backward(run, t, G["rgb"], G["depth"], G["alpha"], G["feat"])
    errs, grep = grad_parity(got, sc, cam, df, t, bg, pix, G, flip)
    check_grads(errs, grep, near_max=2)


@pytest.mark.parametrize("P,C", [(37, 32), (100, 64), (129, 32)])
def test_deformed_few_gaussians_forward_and_backward(P, C):
    # Fewer Gaussians than one 128-row tile of the deformation MLP (its
    # feature rows are read as whole tiles), and one past a tile: forward
    # and reverse against the oracle.
    sc, cam, df = deformed_case(P=P, W=64, H=48, D=16, C=C, R=8, seed=11)
    t, bg = 0.6, (0.1, 0.1, 0.1)
    run = gpu_forward(sc, cam, df, t=t, bg=bg)
    pix = O.all_pixels(cam.width, cam.height)
    e, rep, flip = forward_parity(run, sc, cam, df, t=t, bg=bg)
    check_forward(e, rep, flagged_max=8)
    G = _upstream(len(pix), 16)
    got = gpu_backward(run, t, G["rgb"], G["depth"], G["alpha"], G["feat"])
    errs, grep = grad_parity(got, sc, cam, df, t, bg, pix, G, flip)
    check_grads(errs, grep, near_max=2)


def test_backward_matches_central_differences():
    # Tiny scene: GPU gradients vs central differences of the FP64 oracle forward.
    rng = np.random.default_rng(2)
    P, D = 12, 16
    cam = synth.make_camera(24, 20, 22.0, rotation=synth.random_rotation(rng, 0.1), translation=[0.05, -0.03, 0.1])
    sc = synth.make_scene(P, D, (-0.8, -0.6, 2.0), (0.8, 0.6, 3.0), seed=5)
    sc = dataclasses.replace(sc, log_scales=sc.log_scales + 1.2)
    df = synth.make_deform(P, C=32, R=6, bbox_min=(-1, -1, 1.5), bbox_max=(1, 1, 3.5), full_heads=True,
                           head_std=0.05, seed=6)
    t, bg = 0.35, (0.1, 0.2, 0.3)
    pix = O.all_pixels(cam.width, cam.height)
    n = len(pix)
    G = _upstream(n, D, seed=1)
    run = gpu_forward(sc, cam, df, t=t, bg=bg)
    got = gpu_backward(run, t, G["rgb"], G["depth"], G["alpha"], G["feat"])

    def loss(s):
        r = O.render(s, cam, df, t=t, bg=bg, pixels=pix, eps=None)
        return (G["rgb"] * r["rgb"]).sum() + (G["depth"] * r["depth"]).sum() + (G["alpha"] * r["alpha"]).sum() + \
            (G["feat"] * r["feat"]).sum(), r["sig"]

    _, sig0 = loss(sc)
    checked = 0
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh", "feat"):
        arr = np.asarray(getattr(sc, name), np.float64)
        flat = arr.reshape(-1)
        gref = got[name].reshape(-1)
        scale = max(np.sqrt(np.mean(gref ** 2)), 1e-12)
        for i in range(0, flat.size, max(1, flat.size // 40)):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals, same = [], True
            for s_ in (1, -1):
                x = flat.copy()
                x[i] += s_ * h
                L, sig = loss(dataclasses.replace(sc, **{name: x.reshape(arr.shape)}))
                same &= bool(np.array_equal(sig, sig0))
                vals.append(L)
            if not same:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(gref[i] - fd) <= TOL_FD_REL * max(abs(fd), scale), (name, i, gref[i], fd)
            checked += 1
    assert checked > 150


def test_forward_and_backward_deterministic():
    sc, cam, df = deformed_case(P=3000, seed=8)
    runs = []
    for _ in range(2):
        r = gpu_forward(sc, cam, df, t=0.5)
        G = _upstream(cam.width * cam.height, sc.D, seed=3)
        g = gpu_backward(r, 0.5, G["rgb"], G["depth"], G["alpha"], G["feat"])
        runs.append((r, g))
    (r0, g0), (r1, g1) = runs
    for k in ("rgb", "depth", "alpha", "feat"):
        assert np.array_equal(getattr(r0, k), getattr(r1, k))
    for k in g0:
        assert np.array_equal(g0[k], g1[k]), k


# --------------------------------------------------------------------------
# Full-size workload: sampled pixels, sparse upstream gradients
# --------------------------------------------------------------------------

# Measured at seed 5 / 9 (flagged pixels; Gaussians with a gradient-only
# decision near its threshold); the bounds stay near those counts.
SAMPLED_WORKLOADS = [
    # 10 of 306 flagged (8 depth-order ties, 2 alpha skips); 185 near.
    ("endonerf_200k_640x512", 300, 14, 230),
    # BF16 storage of SH and features (FP32 compositing): 10 of 306 flagged
    # (8 depth-order ties, 2 alpha skips); 190 near.
    ("endonerf_200k_640x512_bf16", 300, 14, 230),
    # 1M Gaussians, 1280x1024, D=64, BF16 storage: 22 of 206 flagged (19
    # depth-order ties, 2 inclusion, 1 termination); 1005 near.
    ("scared_1m_1280x1024", 200, 30, 1500),
]


@pytest.mark.parametrize("name,npix,flagged_max,near_max", SAMPLED_WORKLOADS)
def test_full_size_sampled(name, npix, flagged_max, near_max):
    # Full-size workload and launch configuration, sampled pixels (the FP64
    # oracle composites each one exactly): every sampled pixel checked, then
    # the reverse pass with upstream gradients on the sampled pixels only,
    # so the oracle's gradient of every Gaussian is exact; no Gaussian is
    # left out.  The printed errors are the per-output error table of the
    # workload.
    sc, cam, df = synth.config_inputs(name)
    bf16 = synth.CONFIGS[name]["bf16"]
    t = 0.5
    run = gpu_forward(sc, cam, df, t=t, bf16=bf16)
    st = run.rast.stats()
    rng = np.random.default_rng(5)
    W, H = cam.width, cam.height
    pix = np.c_[rng.integers(0, W, npix), rng.integers(0, H, npix)].astype(np.int32)
    corners = np.array([[0, 0], [W - 1, H - 1], [15, 15], [16, 16], [W - 1, 0], [0, H - 1]], np.int32)
    pix = np.r_[pix, corners]
    idx = pixel_index(pix, W)
    uniq, first = np.unique(idx, return_index=True)
    pix = pix[np.sort(first)]
    idx = pixel_index(pix, W)
    print(name, "K", st["num_dups"])
    e, rep, flip = forward_parity(run, sc, cam, df, t=t, pixels=pix)
    check_forward(e, rep, flagged_max=flagged_max)
    Gs = _upstream(len(pix), sc.D, seed=9)
    HW = W * H
    full = dict(rgb=np.zeros((HW, 3)), depth=np.zeros(HW), alpha=np.zeros(HW), feat=np.zeros((HW, sc.D)))
    for k in full:
        full[k][idx] = Gs[k]
    got = gpu_backward(run, t, full["rgb"], full["depth"], full["alpha"], full["feat"])
    errs, grep = grad_parity(got, sc, cam, df, t, (0, 0, 0), pix, Gs, flip)
    check_grads(errs, grep, near_max=near_max)


# --------------------------------------------------------------------------
# Edge cases and error reporting
# --------------------------------------------------------------------------

def test_empty_scene_is_background():
    sc = synth.make_scene(0, 16, (-1, -1, 2), (1, 1, 4))
    cam = synth.make_camera(40, 30, 50.0)
    run = gpu_forward(sc, cam, bg=(0.25, 0.5, 0.75))
    assert np.allclose(run.rgb, [0.25, 0.5, 0.75]) and np.all(run.alpha == 0) and np.all(run.feat == 0)


def test_all_behind_camera_and_single_pixel_image():
    sc = synth.make_scene(200, 16, (-1, -1, -4), (1, 1, -2), seed=1)
    cam = synth.make_camera(33, 17, 40.0)
    run = gpu_forward(sc, cam)
    assert np.all(run.alpha == 0)
    sc2 = synth.make_scene(50, 16, (-0.1, -0.1, 2), (0.1, 0.1, 3), seed=2)
    cam2 = synth.make_camera(1, 1, 10.0)
    run2 = gpu_forward(sc2, cam2)
    e, rep, _ = forward_parity(run2, sc2, cam2)
    check_forward(e, rep, flagged_max=1)


def test_huge_gaussian_covers_every_tile():
    sc = synth.make_scene(30, 16, (-0.5, -0.5, 2), (0.5, 0.5, 3), seed=3)
    sc.log_scales[0] = [0.5, 0.5, 0.5]   # metres-wide: covers the frame
    cam = synth.make_camera(130, 90, 60.0)
    run = gpu_forward(sc, cam)
    assert run.rast.dump()["touched"].cpu().numpy()[0] == 9 * 6
    e, rep, _ = forward_parity(run, sc, cam)
    check_forward(e, rep, flagged_max=40)


def test_duplicate_capacity_overflow_is_reported():
    sc, cam, df = deformed_case(P=2000, seed=9)
    run = gpu_forward(sc, cam, df, t=0.1, max_dups=500)
    st = run.rast.stats(raise_on_error=False)
    assert st["status"] == 3 and st["device_errors"] & 1 and st["num_dups"] > 500


def test_nonfinite_input_is_reported_and_culled():
    sc, cam, df = deformed_case(P=500, seed=10)
    sc.means[7] = [np.nan, 0.0, 3.0]
    run = gpu_forward(sc, cam, None)
    st = run.rast.stats(raise_on_error=False)
    assert st["status"] == 5 and st["device_errors"] & 4
    assert run.rast.dump()["radius"].cpu().numpy()[7] == 0
    assert np.all(np.isfinite(run.rgb))


def test_probe_fp32_peak_is_plausible():
    f = _lib.fe_probe_fp32_peak(2048)
    print(f"FP32 FMA throughput {f / 1e12:.1f} TFLOP/s")
    assert 10e12 < f < 400e12
