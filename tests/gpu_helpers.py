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
