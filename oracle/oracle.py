"""Python wrapper of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The
product path never touches it, and it imports nothing from the product
package.

The C++ part (``fe_oracle.cpp``) holds the rasterizer definition; this file
adds marshalling plus two small numpy oracles:
  * ``decoder_forward`` / ``decoder_l1``: the pointwise-convolution semantic
    decoder (Sec. 3.3, "CNN-Based Semantic Decoder") and the per-pixel L1
    feature loss (Eq. 10 of Sec. 3.3), read as a 1x1 convolution with bias
    applied to the rendered feature map, loss = mean over pixels of the L1
    norm over channels.
  * ``adam_step``: the Adam update (Sec. 4.1 "Experimental Setup"; Kingma &
    Ba) with bias correction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Decision thresholds of the comparison protocol.  A pixel whose FP64
# decision lies closer than this to its threshold may legitimately take the
# other branch in binary32; such pixels are flagged, counted and masked.
# Order: inclusion (relative to |u|+|v|+r), radius ceil (relative), alpha
# skip (relative), termination (relative), depth tie (factor on the binary32
# depth error bounds), alpha clamp (relative).
DEFAULT_EPS = (1e-6, 5e-6, 1e-4, 1e-4, 2.0, 1e-4)
# Gradient-only decisions per Gaussian: rgb clamp |raw|, J clamp (relative),
# relu (relative to rms), grid cell (relative to R-1).
DEFAULT_GEPS = (1e-5, 1e-5, 1e-5, 1e-6)

FLAG_INCL, FLAG_SKIP, FLAG_TERM, FLAG_DEPTH, FLAG_CLAMP = 1, 2, 4, 8, 16
VALUE_FLAGS = FLAG_INCL | FLAG_SKIP | FLAG_TERM | FLAG_DEPTH


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB)
            _setup(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _Scene(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("D", ctypes.c_int), ("sh_degree", ctypes.c_int),
                ("means", _dp), ("log_scales", _dp), ("quats", _dp), ("logits", _dp),
                ("sh", _dp), ("feat", _dp)]


class _Deform(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("C", ctypes.c_int), ("R", ctypes.c_int),
                ("planes", _dp), ("w1", _dp), ("b1", _dp), ("w2", _dp), ("b2", _dp),
                ("wh", _dp), ("bh", _dp), ("bbox_min", ctypes.c_double * 3),
                ("bbox_max", ctypes.c_double * 3), ("noise", _dp), ("noise_scale", ctypes.c_double)]


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("view", ctypes.c_double * 16), ("campos", ctypes.c_double * 3),
                ("znear", ctypes.c_double)]


class _Gauss(ctypes.Structure):
    _fields_ = [("delta", _dp), ("uv", _dp), ("conic", _dp), ("opacity", _dp), ("depth", _dp),
                ("rgb", _dp), ("rgb_raw", _dp), ("radius", _ip), ("rect", _ip),
                ("rmargin", _dp), ("gflags", _ip), ("gndec", _ip)]


def _setup(L):
    L.or_preprocess.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Deform), ctypes.POINTER(_Camera),
                                ctypes.c_double, _dp, ctypes.POINTER(_Gauss)]
    L.or_render.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Deform), ctypes.POINTER(_Camera),
                            ctypes.c_double, _dp, ctypes.c_int, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _ip, _ip,
                            ctypes.POINTER(ctypes.c_uint64)]
    _u64p = ctypes.POINTER(ctypes.c_uint64)
    L.or_backward.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Deform), ctypes.POINTER(_Camera),
                              ctypes.c_double, _dp, ctypes.c_int, _ip, _dp, _dp, _dp, _dp,
                              _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _u64p, _dp, _u64p]
    L.or_render_alts.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Deform), ctypes.POINTER(_Camera),
                                 ctypes.c_double, _dp, ctypes.c_int, _ip, _dp, ctypes.c_int, ctypes.c_int,
                                 _dp, _dp, _dp, _dp, _u64p, _ip, _ip]
    L.or_tile_bin.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_float), _ip, ctypes.POINTER(ctypes.c_float),
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                              ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_longlong)]
    L.or_sh_eval.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.or_deform_eval.argtypes = [ctypes.POINTER(_Deform), ctypes.c_int, _dp, ctypes.c_double, _dp, _dp]
    for f in (L.or_preprocess, L.or_render, L.or_render_alts, L.or_backward, L.or_tile_bin, L.or_sh_eval,
              L.or_deform_eval):
        f.restype = ctypes.c_int
    L.or_num_threads.restype = ctypes.c_int


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


class _Keep:
    """Holds the fp64 copies alive while a C call runs."""

    def __init__(self):
        self.refs = []

    def d(self, a):
        if a is None:
            return None
        x = _d(a)
        self.refs.append(x)
        return x


def _marshal(scene, camera, deform, keep: _Keep):
    sc = _Scene()
    sc.P = scene.P
    sc.D = scene.D
    sc.sh_degree = scene.sh_degree
    sc.means = _ptr(keep.d(scene.means))
    sc.log_scales = _ptr(keep.d(scene.log_scales))
    sc.quats = _ptr(keep.d(scene.quats))
    sc.logits = _ptr(keep.d(scene.opacity_logits))
    sc.sh = _ptr(keep.d(np.asarray(scene.sh).reshape(scene.P, 48)))
    sc.feat = _ptr(keep.d(scene.feat))
    cam = _Camera()
    cam.width, cam.height = camera.width, camera.height
    cam.fx, cam.fy, cam.cx, cam.cy = camera.fx, camera.fy, camera.cx, camera.cy
    cam.view[:] = [float(v) for v in np.asarray(camera.world_to_cam, np.float64).reshape(16)]
    cam.campos[:] = [float(v) for v in np.asarray(camera.campos, np.float64).reshape(3)]
    cam.znear = camera.znear
    df = _Deform()
    df.enabled = 0
    if deform is not None:
        df.enabled = 1
        df.C, df.R = deform.C, deform.R
        df.planes = _ptr(keep.d(deform.planes))
        df.w1 = _ptr(keep.d(deform.w1))
        df.b1 = _ptr(keep.d(deform.b1))
        df.w2 = _ptr(keep.d(deform.w2))
        df.b2 = _ptr(keep.d(deform.b2))
        df.wh = _ptr(keep.d(deform.wh))
        df.bh = _ptr(keep.d(deform.bh))
        df.bbox_min[:] = [float(v) for v in deform.bbox_min]
        df.bbox_max[:] = [float(v) for v in deform.bbox_max]
        df.noise = _ptr(keep.d(deform.noise)) if deform.noise is not None else None
        df.noise_scale = deform.noise_scale
    return sc, cam, df


def gaussians(scene, camera, deform=None, t: float = 0.0, geps=DEFAULT_GEPS) -> dict:
    """Per-Gaussian FP64 state: delta[P,11], uv, conic, opacity, depth, rgb,
    rgb_raw, radius, rect, rmargin, gflags, gndec (number of near-threshold
    gradient-only decisions, the bits a backward gflip may set)."""
    L = lib()
    keep = _Keep()
    sc, cam, df = _marshal(scene, camera, deform, keep)
    P = scene.P
    out = {k: np.zeros(s) for k, s in dict(delta=(P, 11), uv=(P, 2), conic=(P, 3), opacity=P, depth=P,
                                            rgb=(P, 3), rgb_raw=(P, 3), rmargin=P).items()}
    out["radius"] = np.zeros(P, np.int32)
    out["rect"] = np.zeros((P, 4), np.int32)
    out["gflags"] = np.zeros(P, np.int32)
    out["gndec"] = np.zeros(P, np.int32)
    g = _Gauss()
    for k in ("delta", "uv", "conic", "opacity", "depth", "rgb", "rgb_raw", "rmargin"):
        setattr(g, k, _ptr(out[k]))
    for k in ("radius", "rect", "gflags", "gndec"):
        setattr(g, k, _ptr(out[k], _ip))
    ge = keep.d(np.asarray(geps)) if geps is not None else None
    rc = L.or_preprocess(ctypes.byref(sc), ctypes.byref(df), ctypes.byref(cam), float(t), _ptr(ge), ctypes.byref(g))
    if rc:
        raise RuntimeError(f"or_preprocess failed: {rc}")
    return out


def all_pixels(width: int, height: int) -> np.ndarray:
    ys, xs = np.mgrid[0:height, 0:width]
    return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)


def render(scene, camera, deform=None, t: float = 0.0, bg=(0.0, 0.0, 0.0), pixels=None, eps=DEFAULT_EPS) -> dict:
    """FP64 render of the listed pixels ((x,y) int pairs; default: all).
    Returns rgb [n,3], depth [n], alpha [n], feat [n,D], sumw, ncontrib,
    flags, sig."""
    L = lib()
    keep = _Keep()
    sc, cam, df = _marshal(scene, camera, deform, keep)
    pix = all_pixels(camera.width, camera.height) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    n = pix.shape[0]
    D = scene.D
    out = dict(rgb=np.zeros((n, 3)), depth=np.zeros(n), alpha=np.zeros(n), feat=np.zeros((n, D)),
               sumw=np.zeros(n), ncontrib=np.zeros(n, np.int32), flags=np.zeros(n, np.int32),
               sig=np.zeros(n, np.uint64))
    bgv = keep.d(np.asarray(bg))
    ep = keep.d(np.asarray(eps)) if eps is not None else None
    rc = L.or_render(ctypes.byref(sc), ctypes.byref(df), ctypes.byref(cam), float(t), _ptr(bgv), n,
                     _ptr(pix, _ip), _ptr(ep), _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["alpha"]),
                     _ptr(out["feat"]), _ptr(out["sumw"]), _ptr(out["ncontrib"], _ip), _ptr(out["flags"], _ip),
                     out["sig"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc:
        raise RuntimeError(f"or_render failed: {rc}")
    return out


def render_alternatives(scene, camera, deform=None, t: float = 0.0, bg=(0.0, 0.0, 0.0), pixels=None,
                        eps=DEFAULT_EPS, max_bits: int = 6, max_alts: int = 16) -> dict:
    """Every result a binary32 evaluation may legitimately give at the listed
    pixels: each combination of a pixel's near-threshold decisions (flags of
    ``render``) taken either way, at most 2**max_bits combinations, distinct
    results kept (the FP64 one first).  Returns rgb [n,A,3], depth [n,A],
    alpha [n,A], feat [n,A,D], flip [n,A] (uint64 decision mask for
    ``backward``), nalts [n], ndec [n]."""
    L = lib()
    keep = _Keep()
    sc, cam, df = _marshal(scene, camera, deform, keep)
    pix = all_pixels(camera.width, camera.height) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    n, A, D = pix.shape[0], int(max_alts), scene.D
    out = dict(rgb=np.zeros((n, A, 3)), depth=np.zeros((n, A)), alpha=np.zeros((n, A)), feat=np.zeros((n, A, D)),
               flip=np.zeros((n, A), np.uint64), nalts=np.zeros(n, np.int32), ndec=np.zeros(n, np.int32))
    bgv = keep.d(np.asarray(bg))
    ep = keep.d(np.asarray(eps))
    u64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    rc = L.or_render_alts(ctypes.byref(sc), ctypes.byref(df), ctypes.byref(cam), float(t), _ptr(bgv), n,
                          _ptr(pix, _ip), _ptr(ep), int(max_bits), A, _ptr(out["rgb"]), _ptr(out["depth"]),
                          _ptr(out["alpha"]), _ptr(out["feat"]), u64(out["flip"]), _ptr(out["nalts"], _ip),
                          _ptr(out["ndec"], _ip))
    if rc:
        raise RuntimeError(f"or_render_alts failed: {rc}")
    return out


def backward(scene, camera, deform=None, t: float = 0.0, bg=(0.0, 0.0, 0.0), pixels=None,
             g_rgb=None, g_depth=None, g_alpha=None, g_feat=None, want_uv: bool = False, flip=None,
             gflip=None, eps=DEFAULT_EPS, geps=DEFAULT_GEPS) -> dict:
    """FP64 gradients of sum(g . outputs) over the listed pixels w.r.t.
    means, log_scales, quats, opacity_logits, sh [P,16,3], feat [P,D]; with
    want_uv also "uv" [P,2], the gradient w.r.t. each projected centre
    (pixels).  flip [npix] (uint64, see ``render_alternatives``) takes a
    pixel's near-threshold decisions the other way; gflip [P] (uint64) takes
    a Gaussian's near-threshold gradient-only decisions (``gaussians``'
    gndec) the other way, bit k for the k-th."""
    L = lib()
    keep = _Keep()
    sc, cam, df = _marshal(scene, camera, deform, keep)
    pix = all_pixels(camera.width, camera.height) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    n = pix.shape[0]
    P, D = scene.P, scene.D
    gr = keep.d(np.zeros((n, 3)) if g_rgb is None else np.asarray(g_rgb).reshape(n, 3))
    gz = keep.d(np.zeros(n) if g_depth is None else np.asarray(g_depth).reshape(n))
    ga = keep.d(np.zeros(n) if g_alpha is None else np.asarray(g_alpha).reshape(n))
    gf = keep.d(np.zeros((n, D)) if g_feat is None else np.asarray(g_feat).reshape(n, D))
    out = dict(means=np.zeros((P, 3)), log_scales=np.zeros((P, 3)), quats=np.zeros((P, 4)),
               opacity_logits=np.zeros(P), sh=np.zeros((P, 16, 3)), feat=np.zeros((P, D)))
    bgv = keep.d(np.asarray(bg))
    if want_uv:
        out["uv"] = np.zeros((P, 2))
    u64 = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    fl = None if flip is None else np.ascontiguousarray(np.asarray(flip).reshape(n), np.uint64)
    gfl = None if gflip is None else np.ascontiguousarray(np.asarray(gflip).reshape(P), np.uint64)
    ep = keep.d(np.asarray(eps)) if fl is not None else None
    gep = keep.d(np.asarray(geps)) if gfl is not None else None
    rc = L.or_backward(ctypes.byref(sc), ctypes.byref(df), ctypes.byref(cam), float(t), _ptr(bgv), n,
                       _ptr(pix, _ip), _ptr(gr), _ptr(gz), _ptr(ga), _ptr(gf), _ptr(out["means"]),
                       _ptr(out["log_scales"]), _ptr(out["quats"]), _ptr(out["opacity_logits"]),
                       _ptr(out["sh"]), _ptr(out["feat"]), _ptr(out["uv"]) if want_uv else None,
                       _ptr(ep), u64(fl), _ptr(gep), u64(gfl))
    if rc:
        raise RuntimeError(f"or_backward failed: {rc}")
    return out


def tile_bin(uv, radius, depth, width: int, height: int, tile_w: int = 16, tile_h: int = 16):
    """Integer stage on binary32 inputs: (keys u64 [K], vals u32 [K],
    ranges u32 [tiles,2]) sorted by (tile, depth bits), ties by index."""
    L = lib()
    uv = np.ascontiguousarray(uv, np.float32)
    radius = np.ascontiguousarray(radius, np.int32)
    depth = np.ascontiguousarray(depth, np.float32)
    P = radius.shape[0]
    tiles = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    # Capacity bound: every tile of every rect.
    cap = 0
    K = ctypes.c_longlong(0)
    rc = L.or_tile_bin(P, uv.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _ptr(radius, _ip),
                       depth.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), width, height, tile_w, tile_h,
                       cap, None, None, None, ctypes.byref(K))
    cap = K.value
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    ranges = np.zeros((tiles, 2), np.uint32)
    rc = L.or_tile_bin(P, uv.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _ptr(radius, _ip),
                       depth.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), width, height, tile_w, tile_h,
                       cap, keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                       vals.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                       ranges.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), ctypes.byref(K))
    if rc:
        raise RuntimeError(f"or_tile_bin failed: {rc}")
    return keys[:cap], vals[:cap], ranges


def sh_eval(dirs):
    """Real SH basis (degree <= 3) at unit directions [n,3]: (Y [n,16], dY [n,16,3])."""
    d = _d(dirs).reshape(-1, 3)
    n = d.shape[0]
    Y = np.zeros((n, 16))
    dY = np.zeros((n, 16, 3))
    lib().or_sh_eval(n, _ptr(d), _ptr(Y), _ptr(dY))
    return Y, dY


def deform_eval(deform, mu, t: float):
    """HexPlane feature f [n,C] and head outputs delta [n,11] (no noise term)."""
    keep = _Keep()
    from types import SimpleNamespace
    dummy = SimpleNamespace(P=1, D=1, sh_degree=0, means=np.zeros((1, 3)), log_scales=np.zeros((1, 3)),
                            quats=np.zeros((1, 4)), opacity_logits=np.zeros(1), sh=np.zeros((1, 16, 3)),
                            feat=np.zeros((1, 1)))
    cam = SimpleNamespace(width=1, height=1, fx=1.0, fy=1.0, cx=0.0, cy=0.0, world_to_cam=np.eye(4),
                          campos=np.zeros(3), znear=0.2)
    _, _, df = _marshal(dummy, cam, deform, keep)
    m = keep.d(np.asarray(mu).reshape(-1, 3))
    n = m.shape[0]
    f = np.zeros((n, deform.C))
    delta = np.zeros((n, 11))
    rc = lib().or_deform_eval(ctypes.byref(df), n, _ptr(m), float(t), _ptr(f), _ptr(delta))
    if rc:
        raise RuntimeError("or_deform_eval failed")
    return f, delta


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# numpy FP64 oracles for the decoder, L1 losses and Adam.
# ---------------------------------------------------------------------------

def decoder_forward(feat_map, weight, bias):
    """Pointwise (1x1) convolution D -> Cout over a channels-last map:
    out[p, o] = sum_d feat[p, d] * weight[o, d] + bias[o]."""
    return np.asarray(feat_map, np.float64) @ np.asarray(weight, np.float64).T + np.asarray(bias, np.float64)


def l1_loss_and_grad(pred, target):
    """Per-pixel L1 (Eq. 10 of Sec. 3.3): mean over pixels (rows) of the L1
    norm over channels.  Returns (loss, dloss/dpred).  The sub-gradient at
    pred == target is taken as 0."""
    pred = np.asarray(pred, np.float64)
    diff = pred - np.asarray(target, np.float64)
    n = pred.shape[0]
    return float(np.abs(diff).sum() / n), np.sign(diff) / n


def decoder_backward(feat_map, weight, dout):
    """Gradients of the 1x1 convolution: (dfeat [HW,D], dweight [Cout,D],
    dbias [Cout])."""
    f = np.asarray(feat_map, np.float64)
    w = np.asarray(weight, np.float64)
    g = np.asarray(dout, np.float64)
    return g @ w, g.T @ f, g.sum(0)


def adam_step(param, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-15):
    """One Adam update with bias correction; returns (param, m, v)."""
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
