"""ctypes binding of ``libfe4dgs.so`` (the C ABI in ``include/fe4dgs.h``).

Argument marshalling only: every function here has the name of its C entry
point, turns torch tensors into raw device pointers and the current CUDA
stream into a ``cudaStream_t`` handle, and raises on a non-zero status.
There is no fallback: if the library is missing the import fails.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfe4dgs.so")

c_int, c_float, c_void_p, c_int64 = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_int64

FE_OK = 0
STATUS = {0: "FE_OK", 1: "FE_ERR_INVALID_ARG", 2: "FE_ERR_CUDA", 3: "FE_ERR_WORKSPACE", 4: "FE_ERR_UNSUPPORTED",
          5: "FE_ERR_NONFINITE", 6: "FE_ERR_TIMEOUT", 7: "FE_ERR_STATE"}


class FeError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn} returned {STATUS.get(code, code)}: {status_string(code)}")


class fe_camera(ctypes.Structure):
    _fields_ = [("width", c_int), ("height", c_int), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("world_to_cam", c_float * 16), ("campos", c_float * 3), ("znear", c_float)]


class fe_gaussians(ctypes.Structure):
    _fields_ = [("P", c_int), ("D", c_int), ("sh_degree", c_int), ("sh_bf16", c_int), ("feat_bf16", c_int),
                ("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("sh", c_void_p), ("feat", c_void_p)]


class fe_deform(ctypes.Structure):
    _fields_ = [("C", c_int), ("R", c_int), ("planes", c_void_p), ("w1", c_void_p), ("b1", c_void_p),
                ("w2", c_void_p), ("b2", c_void_p), ("wh", c_void_p), ("bh", c_void_p),
                ("bbox_min", c_float * 3), ("bbox_max", c_float * 3), ("noise", c_void_p),
                ("noise_scale", c_float)]


class fe_opts(ctypes.Structure):
    _fields_ = [("tile_w", c_int), ("tile_h", c_int), ("bg", c_float * 3), ("max_dups", c_int64),
                ("forward_only", c_int), ("accumulate_grads", c_int), ("events", ctypes.POINTER(c_void_p)),
                ("fwd_batch", c_int), ("wait_polls", c_int)]


class fe_batch(ctypes.Structure):
    _fields_ = [("V", c_int), ("cams", ctypes.POINTER(fe_camera)), ("t", ctypes.POINTER(c_float)),
                ("opts", ctypes.POINTER(fe_opts))]


FE_MAX_VIEWS = 32


class fe_outputs(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("alpha", c_void_p), ("feat", c_void_p),
                ("feat_bf16", c_void_p)]


class fe_output_grads(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("alpha", c_void_p), ("feat", c_void_p)]


class fe_grads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("sh", c_void_p), ("feat", c_void_p)]


class fe_stats(ctypes.Structure):
    _fields_ = [("num_dups", c_int64), ("capacity", c_int64), ("num_visible", c_int64),
                ("device_errors", ctypes.c_uint32), ("has_forward", ctypes.c_int32)]


class fe_decoder_args(ctypes.Structure):
    _fields_ = [("HW", c_int64), ("D", c_int), ("feat", c_void_p), ("weight", c_void_p), ("bias", c_void_p)]


class fe_adam_group(ctypes.Structure):
    _fields_ = [("param", c_void_p), ("grad", c_void_p), ("m", c_void_p), ("v", c_void_p),
                ("param_bf16", c_void_p), ("n", c_int64), ("lr", c_float)]


class fe_fst(ctypes.Structure):
    _fields_ = [("levels", c_int), ("rs", c_int), ("rt", c_int), ("D", c_int), ("planes", c_void_p),
                ("mlp", c_void_p), ("bbox_min", c_float * 3), ("bbox_max", c_float * 3), ("exact_planes", c_int)]


class fe_attr(ctypes.Structure):
    _fields_ = [("src", c_void_p), ("dst", c_void_p), ("width", c_int), ("elem_bytes", c_int), ("role", c_int)]


class fe_densify_args(ctypes.Structure):
    _fields_ = [("P", c_int), ("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p),
                ("opacity_logits", c_void_p), ("accum", c_void_p), ("count", c_void_p), ("normals", c_void_p),
                ("grad_thresh", c_float), ("dense_scale", c_float), ("min_opacity", c_float),
                ("attrs", c_void_p), ("nattrs", c_int), ("capacity", c_int64)]


FE_ATTR_COPY, FE_ATTR_MEANS, FE_ATTR_LOG_SCALES, FE_ATTR_STATE = 0, 1, 2, 3

_P = ctypes.POINTER
_SIGNATURES = {
    "fe_workspace_size": [c_int, c_int, c_int, c_int, _P(fe_opts), _P(ctypes.c_size_t)],
    "fe_render_forward": [_P(fe_gaussians), _P(fe_deform), _P(fe_camera), c_float, _P(fe_opts), c_void_p,
                          ctypes.c_size_t, _P(fe_outputs), c_void_p],
    "fe_render_backward": [_P(fe_gaussians), _P(fe_deform), _P(fe_camera), c_float, _P(fe_opts), c_void_p,
                           ctypes.c_size_t, _P(fe_output_grads), _P(fe_grads), c_void_p],
    "fe_tile_bin": [c_int, c_void_p, c_void_p, c_void_p, c_int, c_int, _P(fe_opts), c_void_p, ctypes.c_size_t,
                    c_void_p],
    "fe_read_stats": [c_void_p, ctypes.c_size_t, c_int, c_int, c_int, c_int, _P(fe_opts), _P(fe_stats), c_void_p],
    "fe_debug_dump": [c_void_p, ctypes.c_size_t, c_int, c_int, c_int, c_int, _P(fe_opts)] + [c_void_p] * 12
                     + [c_void_p],
    "fe_probe_fp32_peak": [c_int, _P(ctypes.c_double), c_void_p],
    "fe_l1_loss_grad": [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_void_p],
    "fe_l1_loss_grad_noalloc": [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p, c_void_p],
    "fe_count_pairs": [_P(fe_gaussians), _P(fe_camera), _P(fe_opts), c_void_p, ctypes.c_size_t, c_void_p,
                       c_void_p],
    "fe_decode_forward": [_P(fe_decoder_args), c_void_p, c_void_p, ctypes.c_size_t, c_void_p],
    "fe_decode_l1": [_P(fe_decoder_args), c_void_p, c_int, c_float, c_void_p, c_void_p, c_void_p, c_void_p,
                     c_void_p, ctypes.c_size_t, c_void_p],
    "fe_decoder_read_errors": [c_void_p, _P(ctypes.c_uint32), c_void_p],
    "fe_adam_step": [_P(fe_adam_group), c_int, c_int, c_float, c_float, c_float, c_void_p],
    "fe_sum_f32": [c_void_p, _P(c_void_p), c_int, c_int64, c_void_p],
    "fe_fst_workspace_size": [c_int, c_int, c_int, c_int, c_int, c_int, _P(ctypes.c_size_t)],
    "fe_fst_forward": [_P(fe_fst), c_int] + [c_void_p] * 5 + [c_int, c_float] + [c_void_p] * 6
                      + [ctypes.c_size_t, c_int, c_void_p],
    "fe_fst_backward": [_P(fe_fst), c_int, c_void_p, c_float] + [c_void_p] * 9 + [ctypes.c_size_t, c_void_p],
    "fe_fst_tv": [_P(fe_fst), c_float, c_void_p, c_void_p, c_void_p, c_void_p],
    "fe_screen_grad_stats": [c_void_p, ctypes.c_size_t, c_int, c_int, c_int, c_int, _P(fe_opts), c_void_p,
                             c_void_p, c_void_p],
    "fe_densify": [_P(fe_densify_args), c_void_p, c_void_p, ctypes.c_size_t, c_void_p],
    "fe_reset_opacity": [c_void_p, c_int64, c_float, c_void_p],
    "fe_batch_workspace_size": [c_int, c_int, _P(fe_batch), _P(ctypes.c_size_t)],
    "fe_render_batch": [_P(fe_gaussians), _P(fe_deform), _P(fe_batch), c_void_p, ctypes.c_size_t, _P(fe_outputs),
                        c_void_p],
    "fe_render_batch_backward": [_P(fe_gaussians), _P(fe_deform), _P(fe_batch), c_void_p, ctypes.c_size_t,
                                 _P(fe_output_grads), _P(fe_grads), c_void_p],
    "fe_batch_read_stats": [c_void_p, ctypes.c_size_t, c_int, c_int, _P(fe_batch), _P(fe_stats), c_void_p],
}

_lib = None


def load():
    """Load the in-tree shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2503_06161_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = c_int
        for name in ("fe_fst_plane_floats", "fe_fst_mlp_floats"):
            getattr(L, name).restype = c_int64
        L.fe_fst_plane_floats.argtypes = [c_int, c_int, c_int]
        L.fe_fst_mlp_floats.argtypes = [c_int, c_int]
        L.fe_densify_workspace_size.argtypes = [c_int]
        L.fe_densify_workspace_size.restype = ctypes.c_size_t
        L.fe_decoder_workspace_size.argtypes = [c_int64, c_int]
        L.fe_decoder_workspace_size.restype = ctypes.c_size_t
        L.fe_status_string.argtypes = [c_int]
        L.fe_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return load().fe_status_string(int(code)).decode()


def _check(fn: str, rc: int):
    if rc != FE_OK:
        raise FeError(fn, rc)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_opts(tile=(16, 16), bg=(0.0, 0.0, 0.0), max_dups=0, forward_only=False, accumulate=False, fwd_batch=0,
              wait_polls=0) -> fe_opts:
    o = fe_opts()
    o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
    o.bg[:] = [float(x) for x in bg]
    o.max_dups = int(max_dups)
    o.forward_only = 1 if forward_only else 0
    o.accumulate_grads = 1 if accumulate else 0
    o.fwd_batch = int(fwd_batch)
    o.wait_polls = int(wait_polls)
    return o


def make_batch(cams, ts, opts) -> fe_batch:
    """fe_batch over host arrays of cameras (fe_camera), times and fe_opts
    (kept alive by the returned object)."""
    V = len(cams)
    if not (len(ts) == V and len(opts) == V):
        raise ValueError("one camera, time and options struct per view")
    b = fe_batch()
    b._cams = (fe_camera * V)(*cams)
    b._t = (c_float * V)(*[float(t) for t in ts])
    b._opts = (fe_opts * V)(*opts)
    b.V = V
    b.cams = ctypes.cast(b._cams, ctypes.POINTER(fe_camera))
    b.t = ctypes.cast(b._t, ctypes.POINTER(c_float))
    b.opts = ctypes.cast(b._opts, ctypes.POINTER(fe_opts))
    return b


def make_camera(width, height, fx, fy, cx, cy, world_to_cam, campos, znear=0.2) -> fe_camera:
    c = fe_camera()
    c.width, c.height = int(width), int(height)
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    c.world_to_cam[:] = [float(v) for v in list(world_to_cam)]
    c.campos[:] = [float(v) for v in list(campos)]
    c.znear = float(znear)
    return c


def make_gaussians(means, log_scales, quats, opacity_logits, sh, feat, sh_degree=3) -> fe_gaussians:
    import torch
    g = fe_gaussians()
    g.P = int(means.shape[0])
    g.D = int(feat.shape[1])
    g.sh_degree = int(sh_degree)
    g.sh_bf16 = int(sh.dtype == torch.bfloat16)
    g.feat_bf16 = int(feat.dtype == torch.bfloat16)
    g.means, g.log_scales, g.quats = _ptr(means), _ptr(log_scales), _ptr(quats)
    g.opacity_logits, g.sh, g.feat = _ptr(opacity_logits), _ptr(sh), _ptr(feat)
    return g


def make_deform(planes, w1, b1, w2, b2, wh, bh, bbox_min, bbox_max, noise=None, noise_scale=0.01) -> fe_deform:
    d = fe_deform()
    d.C = int(planes.shape[3])
    d.R = int(planes.shape[1])
    d.planes, d.w1, d.b1, d.w2, d.b2, d.wh, d.bh = (_ptr(x) for x in (planes, w1, b1, w2, b2, wh, bh))
    d.bbox_min[:] = [float(v) for v in bbox_min]
    d.bbox_max[:] = [float(v) for v in bbox_max]
    d.noise = _ptr(noise)
    d.noise_scale = float(noise_scale)
    return d


def fe_workspace_size(P: int, D: int, width: int, height: int, opts: fe_opts) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_workspace_size", load().fe_workspace_size(P, D, width, height, ctypes.byref(opts), ctypes.byref(n)))
    return int(n.value)


def fe_render_forward(g: fe_gaussians, deform, cam: fe_camera, t: float, opts: fe_opts, workspace, rgb, depth,
                      alpha, feat, stream=None, feat_bf16=None):
    out = fe_outputs(_ptr(rgb), _ptr(depth), _ptr(alpha), _ptr(feat), _ptr(feat_bf16))
    rc = load().fe_render_forward(ctypes.byref(g), ctypes.byref(deform) if deform is not None else None,
                                  ctypes.byref(cam), float(t), ctypes.byref(opts), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), ctypes.byref(out), _stream(stream))
    _check("fe_render_forward", rc)


def fe_render_backward(g: fe_gaussians, deform, cam: fe_camera, t: float, opts: fe_opts, workspace, g_rgb, g_depth,
                       g_alpha, g_feat, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_feat, stream=None):
    go = fe_output_grads(_ptr(g_rgb), _ptr(g_depth), _ptr(g_alpha), _ptr(g_feat))
    gr = fe_grads(_ptr(d_means), _ptr(d_log_scales), _ptr(d_quats), _ptr(d_opacity_logits), _ptr(d_sh),
                  _ptr(d_feat))
    rc = load().fe_render_backward(ctypes.byref(g), ctypes.byref(deform) if deform is not None else None,
                                   ctypes.byref(cam), float(t), ctypes.byref(opts), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), ctypes.byref(go), ctypes.byref(gr),
                                   _stream(stream))
    _check("fe_render_backward", rc)


def fe_batch_workspace_size(P: int, D: int, batch: fe_batch) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_batch_workspace_size", load().fe_batch_workspace_size(int(P), int(D), ctypes.byref(batch),
                                                                      ctypes.byref(n)))
    return int(n.value)


def fe_render_batch(g: fe_gaussians, deform, batch: fe_batch, workspace, outs, stream=None):
    """outs: per view (rgb, depth, alpha, feat[, feat_bf16]) device tensors."""
    arr = (fe_outputs * batch.V)()
    for k, o in enumerate(outs):
        arr[k] = fe_outputs(_ptr(o[0]), _ptr(o[1]), _ptr(o[2]), _ptr(o[3]), _ptr(o[4]) if len(o) > 4 else None)
    rc = load().fe_render_batch(ctypes.byref(g), ctypes.byref(deform) if deform is not None else None,
                                ctypes.byref(batch), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                arr, _stream(stream))
    _check("fe_render_batch", rc)


def fe_render_batch_backward(g: fe_gaussians, deform, batch: fe_batch, workspace, grad_outs, grads: dict,
                             stream=None):
    """grad_outs: per view (g_rgb, g_depth, g_alpha, g_feat), any None;
    grads: dict of the summed gradient tensors (means, log_scales, quats,
    opacity_logits, sh, feat)."""
    arr = (fe_output_grads * batch.V)()
    for k, o in enumerate(grad_outs):
        arr[k] = fe_output_grads(*[_ptr(x) for x in o])
    gr = fe_grads(*[_ptr(grads[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "feat")])
    rc = load().fe_render_batch_backward(ctypes.byref(g), ctypes.byref(deform) if deform is not None else None,
                                         ctypes.byref(batch), _ptr(workspace),
                                         workspace.numel() * workspace.element_size(), arr, ctypes.byref(gr),
                                         _stream(stream))
    _check("fe_render_batch_backward", rc)


def fe_batch_read_stats(workspace, P: int, D: int, batch: fe_batch, stream=None, raise_on_error: bool = True):
    """(status, per-view stats dicts); synchronous."""
    arr = (fe_stats * batch.V)()
    rc = load().fe_batch_read_stats(_ptr(workspace), workspace.numel() * workspace.element_size(), int(P), int(D),
                                    ctypes.byref(batch), arr, _stream(stream))
    if raise_on_error:
        _check("fe_batch_read_stats", rc)
    return rc, [dict(num_dups=s.num_dups, capacity=s.capacity, num_visible=s.num_visible,
                     device_errors=s.device_errors, has_forward=s.has_forward) for s in arr]


def fe_tile_bin(uv, radius, depth, width: int, height: int, opts: fe_opts, workspace, stream=None):
    P = int(radius.shape[0])
    rc = load().fe_tile_bin(P, _ptr(uv), _ptr(radius), _ptr(depth), int(width), int(height), ctypes.byref(opts),
                            _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    _check("fe_tile_bin", rc)


def fe_read_stats(workspace, P: int, D: int, width: int, height: int, opts: fe_opts, stream=None,
                  raise_on_error: bool = True) -> dict:
    s = fe_stats()
    rc = load().fe_read_stats(_ptr(workspace), workspace.numel() * workspace.element_size(), P, D, width, height,
                              ctypes.byref(opts), ctypes.byref(s), _stream(stream))
    if raise_on_error:
        _check("fe_read_stats", rc)
    return dict(status=rc, num_dups=s.num_dups, capacity=s.capacity, num_visible=s.num_visible,
                device_errors=s.device_errors, has_forward=s.has_forward)


def fe_debug_dump(workspace, P: int, D: int, width: int, height: int, opts: fe_opts, keys=None, gauss=None,
                  ranges=None, n_contrib=None, t_final=None, uv=None, conic=None, opacity=None, depth=None,
                  rgb=None, radius=None, touched=None, stream=None):
    rc = load().fe_debug_dump(_ptr(workspace), workspace.numel() * workspace.element_size(), P, D, width, height,
                              ctypes.byref(opts), _ptr(keys), _ptr(gauss), _ptr(ranges), _ptr(n_contrib),
                              _ptr(t_final), _ptr(uv), _ptr(conic), _ptr(opacity), _ptr(depth), _ptr(rgb),
                              _ptr(radius), _ptr(touched), _stream(stream))
    _check("fe_debug_dump", rc)


def set_events(opts: fe_opts, events):
    """Attach 8 stage-boundary events (torch.cuda.Event, recorded once so
    their handles exist) to opts; None detaches.  Keeps the array alive."""
    if events is None:
        opts.events = None
        opts._event_array = None
        return
    arr = (c_void_p * 8)(*[c_void_p(e.cuda_event) if e is not None else None for e in events])
    opts._event_array = arr
    opts.events = ctypes.cast(arr, ctypes.POINTER(c_void_p))


def fe_l1_loss_grad(pred, target, rows: int, grad, loss, scratch, stream=None):
    rc = load().fe_l1_loss_grad(_ptr(pred), _ptr(target), int(pred.numel()), int(rows), _ptr(grad), _ptr(loss),
                                _ptr(scratch), _stream(stream))
    _check("fe_l1_loss_grad", rc)


def fe_l1_loss_grad_noalloc(pred, target, rows: int, grad, loss, stream=None):
    """fe_l1_loss_grad without caller scratch (see the header for its limits)."""
    rc = load().fe_l1_loss_grad_noalloc(_ptr(pred), _ptr(target), int(pred.numel()), int(rows), _ptr(grad),
                                        _ptr(loss), _stream(stream))
    _check("fe_l1_loss_grad_noalloc", rc)


def fe_count_pairs(g: fe_gaussians, cam: fe_camera, opts: fe_opts, workspace, counts, stream=None):
    rc = load().fe_count_pairs(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _ptr(counts), _stream(stream))
    _check("fe_count_pairs", rc)


def fe_probe_fp32_peak(iters: int = 4096, stream=None) -> float:
    f = ctypes.c_double(0.0)
    _check("fe_probe_fp32_peak", load().fe_probe_fp32_peak(int(iters), ctypes.byref(f), _stream(stream)))
    return float(f.value)


def make_decoder_args(feat, weight, bias, HW=None) -> fe_decoder_args:
    """feat [HW, D] and weight [256, D] bf16 tensors, bias [256] float32."""
    a = fe_decoder_args()
    a.HW = int(feat.shape[0] if HW is None else HW)
    a.D = int(weight.shape[1])
    a.feat = feat.data_ptr() if feat is not None and feat.numel() else None
    a.weight = weight.data_ptr()
    a.bias = bias.data_ptr()
    return a


def fe_decoder_workspace_size(HW: int, D: int) -> int:
    return int(load().fe_decoder_workspace_size(int(HW), int(D)))


def fe_decode_forward(args: fe_decoder_args, out, workspace, stream=None):
    rc = load().fe_decode_forward(ctypes.byref(args), _ptr(out), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream))
    _check("fe_decode_forward", rc)


def fe_decode_l1(args: fe_decoder_args, target, scale: float, loss, d_feat, d_weight, d_bias, workspace,
                 stream=None):
    import torch
    rc = load().fe_decode_l1(ctypes.byref(args), _ptr(target), int(target.dtype == torch.bfloat16), float(scale),
                             _ptr(loss), _ptr(d_feat), _ptr(d_weight), _ptr(d_bias), _ptr(workspace),
                             workspace.numel() * workspace.element_size(), _stream(stream))
    _check("fe_decode_l1", rc)


def fe_decoder_read_errors(workspace, stream=None) -> int:
    e = ctypes.c_uint32(0)
    _check("fe_decoder_read_errors", load().fe_decoder_read_errors(_ptr(workspace), ctypes.byref(e),
                                                                    _stream(stream)))
    return int(e.value)


def fe_adam_step(groups, step: int, beta1: float, beta2: float, eps: float, stream=None):
    """groups: list of dicts with param, grad, m, v (float32 tensors), lr, and
    optionally param_bf16 (bf16 tensor)."""
    arr = (fe_adam_group * len(groups))()
    for k, g in enumerate(groups):
        arr[k].param = g["param"].data_ptr()
        arr[k].grad = g["grad"].data_ptr()
        arr[k].m = g["m"].data_ptr()
        arr[k].v = g["v"].data_ptr()
        pb = g.get("param_bf16")
        arr[k].param_bf16 = pb.data_ptr() if pb is not None else None
        arr[k].n = int(g["param"].numel())
        arr[k].lr = float(g["lr"])
    _check("fe_adam_step", load().fe_adam_step(arr, len(groups), int(step), float(beta1), float(beta2), float(eps),
                                               _stream(stream)))


def fe_sum_f32(dst, srcs, stream=None):
    """dst = srcs[0] + srcs[1] + ... (float32 tensors of equal size), summed
    left to right."""
    arr = (c_void_p * len(srcs))(*[c_void_p(x.data_ptr()) for x in srcs])
    _check("fe_sum_f32", load().fe_sum_f32(_ptr(dst), arr, len(srcs), int(dst.numel()), _stream(stream)))


# --- full FST deformation module ---------------------------------------------
def make_fst(levels: int, rs: int, rt: int, D: int, planes, mlp, bbox_min, bbox_max, exact_planes=False) -> fe_fst:
    f = fe_fst()
    f.levels, f.rs, f.rt, f.D = int(levels), int(rs), int(rt), int(D)
    f.exact_planes = 1 if exact_planes else 0
    f.planes = _ptr(planes)
    f.mlp = _ptr(mlp)
    for a in range(3):
        f.bbox_min[a] = float(bbox_min[a])
        f.bbox_max[a] = float(bbox_max[a])
    return f


def fe_fst_plane_floats(levels: int, rs: int, rt: int) -> int:
    return int(load().fe_fst_plane_floats(levels, rs, rt))


def fe_fst_mlp_floats(levels: int, D: int) -> int:
    return int(load().fe_fst_mlp_floats(levels, D))


def fe_fst_workspace_size(P: int, levels: int, rs: int, rt: int, D: int, with_backward) -> int:
    """with_backward: 0 / False (forward only), 1 / True, or 2 (with the exact
    plane-gradient accumulators)."""
    n = ctypes.c_size_t(0)
    _check("fe_fst_workspace_size", load().fe_fst_workspace_size(P, levels, rs, rt, D, int(with_backward),
                                                                  ctypes.byref(n)))
    return int(n.value)


def fe_fst_forward(fst: fe_fst, P: int, means, quats, log_scales, logits, feat, t: float, means_t, quats_t,
                   log_scales_t, logits_t, feat_t, workspace, with_backward: bool, stream=None):
    import torch
    rc = load().fe_fst_forward(ctypes.byref(fst), int(P), _ptr(means), _ptr(quats), _ptr(log_scales), _ptr(logits),
                               _ptr(feat), int(feat.dtype == torch.bfloat16), float(t), _ptr(means_t),
                               _ptr(quats_t), _ptr(log_scales_t), _ptr(logits_t), _ptr(feat_t), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), int(with_backward), _stream(stream))
    _check("fe_fst_forward", rc)


def fe_fst_backward(fst: fe_fst, P: int, means, t: float, d_means_t, d_quats_t, d_log_scales_t, d_logits_t,
                    d_feat_t, d_means, d_planes, d_mlp, workspace, stream=None):
    rc = load().fe_fst_backward(ctypes.byref(fst), int(P), _ptr(means), float(t), _ptr(d_means_t), _ptr(d_quats_t),
                                _ptr(d_log_scales_t), _ptr(d_logits_t), _ptr(d_feat_t), _ptr(d_means),
                                _ptr(d_planes), _ptr(d_mlp), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream))
    _check("fe_fst_backward", rc)


def fe_fst_tv(fst: fe_fst, weight: float, loss, d_planes, scratch, stream=None):
    rc = load().fe_fst_tv(ctypes.byref(fst), float(weight), _ptr(loss), _ptr(d_planes), _ptr(scratch),
                          _stream(stream))
    _check("fe_fst_tv", rc)


# --- adaptive density control --------------------------------------------------
def fe_screen_grad_stats(workspace, P: int, D: int, width: int, height: int, opts: fe_opts, accum, count,
                         stream=None):
    rc = load().fe_screen_grad_stats(_ptr(workspace), workspace.numel() * workspace.element_size(), int(P), int(D),
                                     int(width), int(height), ctypes.byref(opts), _ptr(accum), _ptr(count),
                                     _stream(stream))
    _check("fe_screen_grad_stats", rc)


def fe_densify_workspace_size(P: int) -> int:
    return int(load().fe_densify_workspace_size(int(P)))


def fe_densify(P: int, means, log_scales, quats, opacity_logits, accum, count, normals, grad_thresh: float,
               dense_scale: float, min_opacity: float, attrs, capacity: int, new_P, workspace, stream=None):
    """attrs: list of (src, dst, role) with src [P, ...] and dst [capacity, ...]
    tensors of float32 (any role) or bf16 (FE_ATTR_COPY / FE_ATTR_STATE)."""
    import torch
    arr = (fe_attr * len(attrs))()
    for k, (src, dst, role) in enumerate(attrs):
        arr[k].src = src.data_ptr()
        arr[k].dst = dst.data_ptr()
        arr[k].width = math.prod(src.shape[1:])
        arr[k].elem_bytes = 2 if src.dtype == torch.bfloat16 else 4
        arr[k].role = int(role)
    a = fe_densify_args()
    a.P = int(P)
    a.means, a.log_scales, a.quats = _ptr(means), _ptr(log_scales), _ptr(quats)
    a.opacity_logits, a.accum, a.count, a.normals = _ptr(opacity_logits), _ptr(accum), _ptr(count), _ptr(normals)
    a.grad_thresh, a.dense_scale, a.min_opacity = float(grad_thresh), float(dense_scale), float(min_opacity)
    a.attrs = ctypes.cast(arr, c_void_p)
    a.nattrs = len(attrs)
    a.capacity = int(capacity)
    rc = load().fe_densify(ctypes.byref(a), _ptr(new_P), _ptr(workspace), workspace.numel() * workspace.element_size(),
                           _stream(stream))
    _check("fe_densify", rc)


def fe_reset_opacity(logits, max_opacity: float, stream=None):
    _check("fe_reset_opacity", load().fe_reset_opacity(_ptr(logits), int(logits.numel()), float(max_opacity),
                                                       _stream(stream)))
