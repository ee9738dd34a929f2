"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI and compare with the FP64 oracle."""
import dataclasses

import numpy as np
import torch

from oracle import oracle as O
from paper_2503_06161_gb300 import synth
from paper_2503_06161_gb300.raster import DeformField, GaussianScene, Rasterizer, camera_struct

# Bars (relative = |got - ref| / max(|ref|, rms(ref)) elementwise).
TOL_RGB_ABS = 1e-4
TOL_DEPTH_ABS = 1e-4
TOL_FEAT_REL = 1e-4
TOL_GRAD_REL = 1e-3
TOL_FD_REL = 1e-2


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    rms = np.sqrt(np.mean(ref ** 2))
    den = np.maximum(np.abs(ref), max(rms, 1e-30))
    return float(np.max(np.abs(got - ref) / den))


@dataclasses.dataclass
class GpuRun:
    rast: Rasterizer
    scene: GaussianScene
    cam: object
    deform: DeformField
    rgb: np.ndarray     # [H*W,3]
    depth: np.ndarray   # [H*W]
    alpha: np.ndarray
    feat: np.ndarray    # [H*W,D]


def gpu_forward(sc, cam, df=None, t=0.0, tile=(16, 16), bg=(0.0, 0.0, 0.0), bf16=False, max_dups=0):
    scene = GaussianScene.from_numpy(sc, "cuda", bf16=bf16)
    deform = DeformField.from_numpy(df, "cuda") if df is not None else None
    rast = Rasterizer(sc.P, sc.D, cam.width, cam.height, tile=tile, bg=bg, max_dups=max_dups,
                      auto_grow=(max_dups == 0))
    c = camera_struct(cam)
    rgb, depth, alpha, feat = rast.forward(scene, c, deform, t)
    torch.cuda.synchronize()
    HW = cam.width * cam.height
    return GpuRun(rast, scene, c, deform, rgb.cpu().numpy().reshape(3, HW).T.copy(),
                  depth.cpu().numpy().reshape(HW), alpha.cpu().numpy().reshape(HW), feat.cpu().numpy())


def gpu_backward(run: GpuRun, t, g_rgb=None, g_depth=None, g_alpha=None, g_feat=None):
    """Upstream gradients in oracle layout ([HW,3], [HW], [HW], [HW,D])."""
    H, W = run.rast.height, run.rast.width
    dev = "cuda"
    f = lambda a, shape: None if a is None else torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev).reshape(shape)
    gr = None if g_rgb is None else f(np.asarray(g_rgb).T, (3, H, W))
    g = run.rast.backward(run.scene, run.cam, run.deform, t, gr, f(g_depth, (H, W)), f(g_alpha, (H, W)),
                          f(g_feat, (H * W, run.rast.D)))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in g.items()}


def masked_forward_errors(run: GpuRun, ref, pix_index=None):
    """(errors dict, number of flagged pixels) comparing the GPU outputs at
    pix_index (default all) with the oracle, excluding flagged pixels."""
    idx = np.arange(run.rgb.shape[0]) if pix_index is None else np.asarray(pix_index)
    ok = (ref["flags"] & O.VALUE_FLAGS) == 0
    flagged = int((~ok).sum())
    g_rgb, g_d, g_a, g_f = run.rgb[idx][ok], run.depth[idx][ok], run.alpha[idx][ok], run.feat[idx][ok]
    e = dict(rgb=float(np.abs(g_rgb - ref["rgb"][ok]).max(initial=0)),
             depth=float(np.abs(g_d - ref["depth"][ok]).max(initial=0)),
             alpha=float(np.abs(g_a - ref["alpha"][ok]).max(initial=0)),
             feat=rel_err(g_f, ref["feat"][ok]))
    return e, flagged


FLAG_NAMES = {O.FLAG_INCL: "inclusion", O.FLAG_SKIP: "alpha_skip", O.FLAG_TERM: "termination",
              O.FLAG_DEPTH: "depth_order", O.FLAG_CLAMP: "alpha_clamp"}


def flag_breakdown(flags) -> dict:
    """Pixels per decision flag (a pixel may carry several)."""
    flags = np.asarray(flags)
    return {name: int(((flags & bit) != 0).sum()) for bit, name in FLAG_NAMES.items()}


def forward_parity(run: GpuRun, sc, cam, df=None, t=0.0, bg=(0.0, 0.0, 0.0), pixels=None):
    """Compares EVERY listed pixel (default all) with the oracle.

    A pixel whose FP64 decisions are all clear of their thresholds is
    compared with the FP64 result.  A flagged pixel (a decision within the
    binary32 error model of its threshold) is compared with the oracle result
    of each way of taking those decisions (``render_alternatives``) and the
    closest one is kept: both branches are correct results of the pass.
    Returns (errors over all pixels, report, flip) where flip [n] is the
    chosen decision mask per pixel (0 = the FP64 branch) for the reverse
    pass, and report holds the flagged count, the per-flag breakdown, the
    pixels whose GPU result took a non-FP64 branch and the number of pixels
    left unchecked (always 0)."""
    ref = O.render(sc, cam, df, t=t, bg=bg, pixels=pixels)
    n = ref["rgb"].shape[0]
    idx = np.arange(run.rgb.shape[0]) if pixels is None else pixel_index(pixels, cam.width)
    got = dict(rgb=run.rgb[idx], depth=run.depth[idx], alpha=run.alpha[idx], feat=run.feat[idx])
    want = {k: ref[k].copy() for k in ("rgb", "depth", "alpha", "feat")}
    frms = max(float(np.sqrt(np.mean(ref["feat"] ** 2))), 1e-30) if ref["feat"].size else 1.0
    flagged = (ref["flags"] & O.VALUE_FLAGS) != 0
    flip = np.zeros(n, np.uint64)
    nalts = np.ones(n, np.int32)
    if flagged.any():
        pix = O.all_pixels(cam.width, cam.height) if pixels is None else np.asarray(pixels)
        sel = np.nonzero(flagged)[0]
        alt = O.render_alternatives(sc, cam, df, t=t, bg=bg, pixels=pix[sel])
        for j, i in enumerate(sel):
            na = int(alt["nalts"][j])
            nalts[i] = na
            score = []
            for a in range(na):
                fden = np.maximum(np.abs(alt["feat"][j, a]), frms)
                score.append(max(np.abs(got["rgb"][i] - alt["rgb"][j, a]).max() / TOL_RGB_ABS,
                                 abs(got["depth"][i] - alt["depth"][j, a]) / TOL_DEPTH_ABS,
                                 abs(got["alpha"][i] - alt["alpha"][j, a]) / TOL_RGB_ABS,
                                 (np.abs(got["feat"][i] - alt["feat"][j, a]) / fden).max(initial=0) / TOL_FEAT_REL))
            a = int(np.argmin(score))
            for k in ("rgb", "depth", "alpha", "feat"):
                want[k][i] = alt[k][j, a]
            flip[i] = alt["flip"][j, a]
    e = dict(rgb=float(np.abs(got["rgb"] - want["rgb"]).max(initial=0)),
             depth=float(np.abs(got["depth"] - want["depth"]).max(initial=0)),
             alpha=float(np.abs(got["alpha"] - want["alpha"]).max(initial=0)),
             feat=float((np.abs(got["feat"] - want["feat"]) / np.maximum(np.abs(want["feat"]), frms)).max(initial=0)))
    report = dict(pixels=n, flagged=int(flagged.sum()), per_flag=flag_breakdown(ref["flags"]),
                  other_branch=int((flip != 0).sum()), max_alternatives=int(nalts.max(initial=1)), unchecked=0)
    return e, report, flip


def check_forward(e, report, flagged_max):
    """Asserts the forward bars and that the flagged count stays within its
    measured bound (a guard on the width of the decision margins)."""
    print("forward errors", e, "report", report)
    assert report["unchecked"] == 0
    assert report["flagged"] <= flagged_max, report
    assert e["rgb"] < TOL_RGB_ABS and e["depth"] < TOL_DEPTH_ABS and e["alpha"] < TOL_RGB_ABS, e
    assert e["feat"] < TOL_FEAT_REL, e


GRAD_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh", "feat")


def _row_err(got, ref):
    """Per-Gaussian worst relative error (rms floor over the whole array)."""
    got = np.asarray(got, np.float64).reshape(got.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    rms = max(float(np.sqrt(np.mean(ref ** 2))), 1e-30) if ref.size else 1.0
    return (np.abs(got - ref) / np.maximum(np.abs(ref), rms)).max(axis=1, initial=0)


def grad_parity(got, sc, cam, df, t, bg, pixels, G, flip=None, max_bits=3):
    """Compares the gradients of EVERY Gaussian with the oracle's gradients of
    the same upstream gradients G (per listed pixel), the pixels' decisions
    taken as the forward comparison found them (flip).  A Gaussian with a
    gradient-only decision within rounding of its threshold (rgb clamp, J
    clamp, ReLU, grid cell: gndec > 0) is compared with the oracle's
    gradients for each way of taking those decisions and the closest is
    kept.  Returns (errors per array, report)."""
    kw = dict(pixels=pixels, g_rgb=G["rgb"], g_depth=G["depth"], g_alpha=G["alpha"], g_feat=G["feat"], flip=flip)
    ref = O.backward(sc, cam, df, t, bg, **kw)
    gndec = O.gaussians(sc, cam, df, t=t)["gndec"]
    P = sc.P
    best = np.zeros(P, np.int64)
    chosen = {k: ref[k].copy() for k in GRAD_KEYS}
    if (gndec > 0).any():
        nb = min(int(gndec.max()), max_bits)
        score0 = np.max([_row_err(got[k], ref[k]) for k in GRAD_KEYS], axis=0)
        bscore = score0.copy()
        for mask in range(1, 1 << nb):
            need = mask.bit_length()
            gf = np.where(gndec >= need, mask, 0).astype(np.uint64)
            if not gf.any():
                continue
            alt = O.backward(sc, cam, df, t, bg, gflip=gf, **kw)
            sc_m = np.max([_row_err(got[k], alt[k]) for k in GRAD_KEYS], axis=0)
            better = (gf != 0) & (sc_m < bscore)
            bscore[better] = sc_m[better]
            best[better] = mask
            for k in GRAD_KEYS:
                chosen[k][better] = alt[k][better]
    errs = {k: rel_err(got[k], chosen[k]) for k in GRAD_KEYS}
    report = dict(gaussians=P, near_decisions=int((gndec > 0).sum()), other_branch=int((best != 0).sum()),
                  excluded=0)
    return errs, report


def check_grads(errs, report, tol=TOL_GRAD_REL, near_max=None):
    print("grad errors", errs, "report", report)
    assert report["excluded"] == 0
    if near_max is not None:
        assert report["near_decisions"] <= near_max, report
    for k, e in errs.items():
        assert e < tol, (k, e)


def pixel_index(pix, width):
    pix = np.asarray(pix)
    return pix[:, 1] * width + pix[:, 0]


def deformed_case(P=4000, W=150, H=100, D=32, f=120.0, seed=0, C=32, R=16, full_heads=True):
    """A deforming scene spanning several tiles with a ragged last row and
    column, a slightly rotated and translated camera, and a background."""
    rng = np.random.default_rng(seed + 100)
    sc = synth.make_scene(P, D, (-1.2, -0.8, 2.0), (1.2, 0.8, 4.5), seed=seed)
    cam = synth.make_camera(W, H, f, rotation=synth.random_rotation(rng, 0.05), translation=[0.02, -0.01, 0.05])
    df = synth.make_deform(P, C=C, R=R, bbox_min=(-1.5, -1.0, 1.5), bbox_max=(1.5, 1.0, 5.0), full_heads=full_heads,
                           head_std=0.02, seed=seed + 1)
    return sc, cam, df
