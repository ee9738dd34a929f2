"""Seeded synthetic inputs for the FE-4DGS rasterization pass.

This module draws random scenes, cameras, deformation fields and loss
targets with numpy's PCG64 generator.  It holds none of the method's
arithmetic: nothing here projects, blends or differentiates.  Both the CUDA
path and the FP64 oracle consume the arrays it returns, so the two never
derive inputs from each other.

Scene shapes follow the paper's endoscopic workloads: 640x512 frames
(EndoNeRF / EndoVis18 downsampled, Sec. 4.2 "Datasets") and 1280x1024
frames (EndoVis18 native), with 1e5..1e6 Gaussians bracketing the 30k-90k
initial points of the hyperparameter table (Appendix E) after densification.
The real datasets are not available; these seeded scenes stand in for them.

Recipe (every array float32 unless stated):
  means          uniform in the box volume
  log_scales     N(-3, 0.5)
  quats (w,x,y,z) N(0, I4) normalised to unit length
  opacity_logits N(0, 1)
  sh [P,16,3]    N(0, 0.3) (all 48 coefficients drawn even when sh_degree<3)
  feat [P,D]     N(0, 1)
  deformation    6 channels-last planes [6,R,R,C] ~ N(1, 0.1); MLP C->64->64
                 weights N(0, sqrt(2/fan_in)), biases 0; head [11,64] weights
                 N(0, 0.01/8) with the d_mu rows (0..2) and the d_o row (10)
                 zero; noise xi [P,3] ~ N(0, 1) scaled by 0.01*t
  targets        rgb U(0,1) [3,H,W]; features N(0,1)
  density stats  views per Gaussian count ~ U{0..8} (int32); accum = the sum
                 of count Exp(2e-4) draws (NDC centre-gradient norms);
                 split normals [P,2,3] ~ N(0, 1)
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Scene", "Camera", "Deform", "make_scene", "make_camera", "make_deform",
    "make_targets", "bf16_round", "bf16_bits", "CONFIGS", "config_inputs",
]


@dataclasses.dataclass
class Scene:
    means: np.ndarray          # [P,3]
    log_scales: np.ndarray     # [P,3]
    quats: np.ndarray          # [P,4] (w,x,y,z)
    opacity_logits: np.ndarray  # [P]
    sh: np.ndarray             # [P,16,3]
    feat: np.ndarray           # [P,D]
    sh_degree: int = 3

    @property
    def P(self) -> int:
        return int(self.means.shape[0])

    @property
    def D(self) -> int:
        return int(self.feat.shape[1])


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray   # [4,4] row-major, float32
    campos: np.ndarray         # [3] camera centre in world space
    znear: float = 0.2


@dataclasses.dataclass
class Deform:
    planes: np.ndarray   # [6,R,R,C] channels-last; planes xy,xz,yz,xt,yt,zt
    w1: np.ndarray       # [64,C]
    b1: np.ndarray       # [64]
    w2: np.ndarray       # [64,64]
    b2: np.ndarray       # [64]
    wh: np.ndarray       # [11,64]  rows: d_mu(3) d_q(4) d_s(3) d_o(1)
    bh: np.ndarray       # [11]
    bbox_min: np.ndarray  # [3]
    bbox_max: np.ndarray  # [3]
    noise: np.ndarray | None  # [P,3] or None
    noise_scale: float = 0.01

    @property
    def C(self) -> int:
        return int(self.planes.shape[3])

    @property
    def R(self) -> int:
        return int(self.planes.shape[1])


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest, ties to even); return the
    16-bit patterns as uint16.  Inputs are finite."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 values exactly representable in bfloat16 (nearest-even)."""
    b = bf16_bits(x).astype(np.uint32) << 16
    return b.view(np.float32).reshape(np.shape(x))


def make_scene(P: int, D: int, lo, hi, seed: int = 0, sh_degree: int = 3,
               sh_std: float = 0.3, bf16_storage: bool = False) -> Scene:
    """Gaussians drawn uniformly inside the box [lo, hi] (3-vectors)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    means = (lo + (hi - lo) * rng.random((P, 3))).astype(np.float32)
    log_scales = rng.normal(-3.0, 0.5, (P, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, (P, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = q.astype(np.float32)
    logits = rng.normal(0.0, 1.0, P).astype(np.float32)
    sh = rng.normal(0.0, sh_std, (P, 16, 3)).astype(np.float32)
    feat = rng.normal(0.0, 1.0, (P, D)).astype(np.float32)
    if bf16_storage:
        sh = bf16_round(sh)
        feat = bf16_round(feat)
    return Scene(means, log_scales, quats, logits, sh, feat, sh_degree)


def make_camera(width: int, height: int, fx: float, fy: float | None = None,
                rotation: np.ndarray | None = None,
                translation: np.ndarray | None = None,
                znear: float = 0.2) -> Camera:
    """Pinhole camera with the principal point at the image centre.

    ``rotation``/``translation`` give the world->camera rigid transform
    (x_cam = R x_world + t); identity by default, as in the paper's
    single-viewpoint setup with all poses set to the identity (Appendix B).
    """
    fy = fx if fy is None else fy
    R = np.eye(3) if rotation is None else np.asarray(rotation, np.float64)
    t = np.zeros(3) if translation is None else np.asarray(translation, np.float64)
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = t
    campos = -R.T @ t
    return Camera(int(width), int(height), float(fx), float(fy),
                  width / 2.0, height / 2.0, V.astype(np.float32),
                  campos.astype(np.float32), float(znear))


def random_rotation(rng: np.random.Generator, angle: float) -> np.ndarray:
    """Rotation by ``angle`` radians about a random axis (Rodrigues)."""
    k = rng.normal(size=3)
    k /= np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def make_deform(P: int, C: int = 32, R: int = 64, seed: int = 1,
                bbox_min=(-2.0, -2.0, 3.0), bbox_max=(2.0, 2.0, 8.0),
                noise: bool = True, noise_scale: float = 0.01,
                full_heads: bool = False, head_std: float = 0.01 / 8.0) -> Deform:
    """Seeded HexPlane grid + MLP deformation field.

    With ``full_heads`` the d_mu and d_o head rows are drawn too (used by
    tests that exercise every branch); otherwise they are zero.
    """
    rng = np.random.default_rng(seed)
    H = 64
    planes = rng.normal(1.0, 0.1, (6, R, R, C)).astype(np.float32)
    w1 = rng.normal(0.0, np.sqrt(2.0 / C), (H, C)).astype(np.float32)
    w2 = rng.normal(0.0, np.sqrt(2.0 / H), (H, H)).astype(np.float32)
    wh = rng.normal(0.0, head_std, (11, H)).astype(np.float32)
    if not full_heads:
        wh[0:3] = 0.0
        wh[10] = 0.0
    b1 = np.zeros(H, np.float32)
    b2 = np.zeros(H, np.float32)
    bh = np.zeros(11, np.float32)
    if full_heads:
        b1 = rng.normal(0.0, 0.1, H).astype(np.float32)
        b2 = rng.normal(0.0, 0.1, H).astype(np.float32)
        bh = rng.normal(0.0, 0.01, 11).astype(np.float32)
    xi = rng.normal(0.0, 1.0, (P, 3)).astype(np.float32) if noise else None
    return Deform(planes, w1, b1, w2, b2, wh, bh,
                  np.asarray(bbox_min, np.float32), np.asarray(bbox_max, np.float32),
                  xi, float(noise_scale))


# Layer shapes of the full FST module in the flat parameter order of the
# library interface: F_out (L*32 -> 64, then 7 x 64 -> 64), per branch mu, R,
# S, o (64 -> 32, 32 -> 32, 32 -> d_g), F_feat (128 -> 64, 64 -> D).
def fst_layer_shapes(levels: int, D: int):
    out = [(64, levels * 32)] + [(64, 64)] * 7
    for d in (3, 4, 3, 1):
        out += [(32, 64), (32, 32), (d, 32)]
    return out + [(64, 128), (D, 64)]


def fst_plane_shapes(levels: int, rs: int, rt: int):
    out = []
    for lv in range(levels):
        res = (rs << lv, rs << lv, rs << lv, rt)
        for a, b in ((0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)):
            out.append((res[a], res[b], 32))
    return out


def make_fst(levels: int = 4, rs: int = 64, rt: int = 100, D: int = 32, seed: int = 5, plane_std: float = 0.1,
             head_std: float = 0.01, dz_std: float = 0.1, bias_std: float = 0.0):
    """Seeded parameters of the full FST deformation module as the two flat
    float32 arrays of the library interface: planes ~ N(1, plane_std);
    hidden layers N(0, sqrt(2 / fan_in)); branch heads N(0, head_std /
    sqrt(fan_in)) (small offsets); the dz layer N(0, dz_std / sqrt(fan_in));
    biases N(0, bias_std)."""
    rng = np.random.default_rng(seed)
    planes = np.concatenate([rng.normal(1.0, plane_std, s).astype(np.float32).ravel()
                             for s in fst_plane_shapes(levels, rs, rt)])
    parts = []
    shapes = fst_layer_shapes(levels, D)
    heads = {10, 13, 16, 19}
    for k, (o, i) in enumerate(shapes):
        std = np.sqrt(2.0 / i)
        if k in heads:
            std = head_std / np.sqrt(i)
        if k == len(shapes) - 1:
            std = dz_std / np.sqrt(i)
        parts.append(rng.normal(0.0, std, (o, i)).astype(np.float32).ravel())
        parts.append((rng.normal(0.0, bias_std, o) if bias_std > 0 else np.zeros(o)).astype(np.float32))
    return planes, np.concatenate(parts)


def make_targets(height: int, width: int, D: int, seed: int = 2, dec_channels: int = 0):
    """Random L1 targets: rgb U(0,1) [3,H,W]; features N(0,1) [H*W, D] (or
    [H*W, dec_channels] when a decoder output is the target)."""
    rng = np.random.default_rng(seed)
    rgb = rng.random((3, height, width)).astype(np.float32)
    Df = dec_channels if dec_channels else D
    feat = rng.normal(0.0, 1.0, (height * width, Df)).astype(np.float32)
    return rgb, feat


def make_depth_target(height: int, width: int, near: float, far: float, seed: int = 4):
    """Depth-map target (the stereo depth a training view supervises with):
    a smooth surface between near and far plus N(0, 1%) noise, [H,W]."""
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.linspace(0.0, 1.0, height), np.linspace(0.0, 1.0, width), indexing="ij")
    a = rng.uniform(0.0, 2.0 * np.pi, 3)
    s = 0.5 + 0.25 * np.sin(2.0 * np.pi * x + a[0]) * np.cos(np.pi * y + a[1]) + 0.2 * np.sin(3.0 * y + a[2])
    d = near + (far - near) * np.clip(s, 0.0, 1.0)
    d = d * (1.0 + 0.01 * rng.normal(size=d.shape))
    return d.astype(np.float32)


def make_density_stats(P: int, seed: int = 6, mean_grad: float = 2e-4, max_views: int = 8):
    """Statistics that adaptive density control reads after some iterations:
    (accum float32 [P], count int32 [P], normals float32 [P,2,3])."""
    rng = np.random.default_rng(seed)
    count = rng.integers(0, max_views + 1, P).astype(np.int32)
    accum = np.where(count > 0, rng.gamma(np.maximum(count, 1), mean_grad), 0.0).astype(np.float32)
    normals = rng.normal(0.0, 1.0, (P, 2, 3)).astype(np.float32)
    return accum, count, normals


def make_decoder(D: int, cout: int = 256, seed: int = 3, w_std: float = 0.05, b_std: float = 0.0):
    """1x1 decoder parameters: weight [cout, D] N(0, w_std) rounded to bf16
    values (float32 array), bias [cout] N(0, b_std)."""
    rng = np.random.default_rng(seed)
    w = bf16_round(rng.normal(0.0, w_std, (cout, D)).astype(np.float32))
    b = rng.normal(0.0, b_std, cout).astype(np.float32) if b_std > 0 else np.zeros(cout, np.float32)
    return w, b


# Workload presets.  Sizes and distributions are the ones stated for each
# workload; names describe what they are.
CONFIGS = {
    "static_1k_64x64": dict(P=1000, D=16, W=64, H=64, f=80.0, lo=(-1, -1, 2), hi=(1, 1, 4),
                            deform=False, bf16=False, seed=0),
    "endonerf_200k_640x512": dict(P=200_000, D=32, W=640, H=512, f=560.0, lo=(-2, -2, 3),
                                  hi=(2, 2, 8), deform=True, bf16=False, seed=0),
    "endonerf_200k_640x512_bf16": dict(P=200_000, D=32, W=640, H=512, f=560.0, lo=(-2, -2, 3),
                                       hi=(2, 2, 8), deform=True, bf16=True, seed=0,
                                       decoder=256),
    "batched_300k_16views": dict(P=300_000, D=32, W=640, H=512, f=560.0, lo=(-2, -2, 3),
                                 hi=(2, 2, 8), deform=True, bf16=True, seed=0, views=16),
    "scared_1m_1280x1024": dict(P=1_000_000, D=64, W=1280, H=1024, f=1000.0, lo=(-2, -2, 3),
                                hi=(2, 2, 8), deform=True, bf16=True, seed=0, decoder=256, train=True),
    # Training with the full FST module (4-level HexPlane 64^3 x 100, depth-8
    # MLP, branches, semantic updater; Sec. 3.2, Appendix A) and the TV term.
    "fst_200k_640x512_train": dict(P=200_000, D=32, W=640, H=512, f=560.0, lo=(-2, -2, 3), hi=(2, 2, 8),
                                   deform=False, bf16=True, seed=0, decoder=256, train=True,
                                   fst=dict(levels=4, rs=64, rt=100)),
}


def config_inputs(name: str, P: int | None = None, D: int | None = None):
    """(scene, camera, deform-or-None) for a named workload; ``P`` overrides
    the Gaussian count (same distributions) for scaled-down test cases, ``D``
    the feature width (feature-width sweeps)."""
    c = CONFIGS[name]
    n = c["P"] if P is None else P
    scene = make_scene(n, c["D"] if D is None else D, c["lo"], c["hi"], seed=c["seed"], bf16_storage=c["bf16"])
    cam = make_camera(c["W"], c["H"], c["f"])
    deform = make_deform(n, bbox_min=(-2, -2, 3), bbox_max=(2, 2, 8)) if c["deform"] else None
    return scene, cam, deform
