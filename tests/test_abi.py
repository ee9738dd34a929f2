"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every entry point that include/fe4dgs.h declares, its structs match the
ctypes mirrors byte for byte, and host-side argument checks return the
documented status codes (no CUDA call is made by these)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2503_06161_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fe4dgs.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "fe_render_forward" in names and "fe_render_backward" in names
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fe_[a-z0-9_]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_layouts_match_header(tmp_path):
    structs = ["fe_camera", "fe_gaussians", "fe_deform", "fe_opts", "fe_outputs", "fe_output_grads", "fe_grads",
               "fe_stats", "fe_fst", "fe_attr", "fe_densify_args", "fe_batch"]
    c = "#include <stdio.h>\n#include <stddef.h>\n#include \"fe4dgs.h\"\nint main(void){\n"
    for s in structs:
        c += f'printf("{s} %zu\\n", sizeof({s}));\n'
    c += 'printf("fe_opts.max_dups %zu\\n", offsetof(fe_opts, max_dups));\n'
    c += 'printf("fe_deform.bbox_min %zu\\n", offsetof(fe_deform, bbox_min));\n'
    c += 'printf("fe_opts.fwd_batch %zu\\n", offsetof(fe_opts, fwd_batch));\n'
    c += 'printf("fe_opts.wait_polls %zu\\n", offsetof(fe_opts, wait_polls));\n'
    c += 'printf("FE_MAX_VIEWS %d\\n", FE_MAX_VIEWS);\n'
    for f in ("normals", "grad_thresh", "attrs", "capacity"):
        c += f'printf("fe_densify_args.{f} %zu\\n", offsetof(fe_densify_args, {f}));\n'
    c += "return 0;}\n"
    (tmp_path / "t.c").write_text(c)
    exe = tmp_path / "t"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(tmp_path / "t.c"), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for s in structs:
        assert int(got[s]) == ctypes.sizeof(getattr(_lib, s)), s
    assert int(got["fe_opts.max_dups"]) == _lib.fe_opts.max_dups.offset
    assert int(got["fe_deform.bbox_min"]) == _lib.fe_deform.bbox_min.offset
    assert int(got["fe_opts.fwd_batch"]) == _lib.fe_opts.fwd_batch.offset
    assert int(got["fe_opts.wait_polls"]) == _lib.fe_opts.wait_polls.offset
    assert int(got["FE_MAX_VIEWS"]) == _lib.FE_MAX_VIEWS
    for f in ("normals", "grad_thresh", "attrs", "capacity"):
        assert int(got[f"fe_densify_args.{f}"]) == getattr(_lib.fe_densify_args, f).offset, f


def test_host_side_status_codes(lib):
    o = _lib.make_opts()
    n = ctypes.c_size_t(0)
    assert lib.fe_workspace_size(1000, 16, 64, 64, ctypes.byref(o), ctypes.byref(n)) == 0 and n.value > 0
    assert lib.fe_workspace_size(1000, 24, 64, 64, ctypes.byref(o), ctypes.byref(n)) == 4   # D not compiled in
    bad = _lib.make_opts(tile=(12, 12))
    assert lib.fe_workspace_size(1000, 16, 64, 64, ctypes.byref(bad), ctypes.byref(n)) == 4
    assert lib.fe_workspace_size(-1, 16, 64, 64, ctypes.byref(o), ctypes.byref(n)) == 1
    assert lib.fe_workspace_size(10, 16, 0, 64, ctypes.byref(o), ctypes.byref(n)) == 1
    huge = _lib.make_opts(max_dups=1 << 31)
    assert lib.fe_workspace_size(10, 16, 64, 64, ctypes.byref(huge), ctypes.byref(n)) == 1
    assert lib.fe_render_forward(None, None, None, 0.0, None, None, 0, None, None) == 1
    assert lib.fe_render_backward(None, None, None, 0.0, None, None, 0, None, None, None) == 1
    assert _lib.status_string(3).startswith("workspace")


def test_workspace_grows_with_capacity_and_backward(lib):
    a = _lib.fe_workspace_size(5000, 32, 320, 256, _lib.make_opts(max_dups=100000))
    b = _lib.fe_workspace_size(5000, 32, 320, 256, _lib.make_opts(max_dups=200000))
    c = _lib.fe_workspace_size(5000, 32, 320, 256, _lib.make_opts(max_dups=200000, forward_only=True))
    assert b > a > c


def test_decoder_host_side_status_codes(lib):
    # Argument checks of the decoder entry points return before any CUDA call.
    assert lib.fe_decoder_workspace_size(1000, 256) == 0         # D not supported by the decoder
    assert lib.fe_decoder_workspace_size(1000, 16) == lib.fe_decoder_workspace_size(1000, 32)   # runs as 32
    assert lib.fe_decoder_workspace_size(-1, 32) == 0
    a = _lib.fe_decoder_args()
    a.HW, a.D, a.feat, a.weight, a.bias = 1000, 256, 16, 16, 16
    args = [None, 0, 1.0, None, None, None, None, None, 0, None]
    assert lib.fe_decode_l1(ctypes.byref(a), *args) == 4         # FE_ERR_UNSUPPORTED
    assert lib.fe_decode_forward(ctypes.byref(a), None, None, 0, None) == 4
    a.D = 32
    a.weight = 8                                                   # not 16-byte aligned
    assert lib.fe_decode_l1(ctypes.byref(a), *args) == 1
    a.weight, a.HW = 16, -5
    assert lib.fe_decode_forward(ctypes.byref(a), None, None, 0, None) == 1
    assert lib.fe_decode_l1(None, *args) == 1
    assert lib.fe_decoder_read_errors(None, None, None) == 1


def test_adam_host_side_status_codes(lib):
    g = (_lib.fe_adam_group * 1)()
    g[0].param = g[0].grad = g[0].m = g[0].v = 16
    g[0].n = 8
    g[0].lr = 1.0
    assert lib.fe_adam_step(None, 1, 1, 0.9, 0.999, 1e-15, None) == 1
    assert lib.fe_adam_step(g, 0, 1, 0.9, 0.999, 1e-15, None) == 1       # no groups
    assert lib.fe_adam_step(g, 9, 1, 0.9, 0.999, 1e-15, None) == 1       # more than 8
    assert lib.fe_adam_step(g, 1, 0, 0.9, 0.999, 1e-15, None) == 1       # step counts from 1
    assert lib.fe_adam_step(g, 1, 1, 1.0, 0.999, 1e-15, None) == 1       # beta1 must be < 1
    g[0].m = 20                                                           # misaligned moment
    assert lib.fe_adam_step(g, 1, 1, 0.9, 0.999, 1e-15, None) == 1
    g[0].n = 0                                                            # empty group: nothing to do
    assert lib.fe_adam_step(g, 1, 1, 0.9, 0.999, 1e-15, None) == 0


def test_sum_host_side_status_codes(lib):
    srcs = (ctypes.c_void_p * 2)(16, 32)
    assert lib.fe_sum_f32(None, srcs, 2, 8, None) == 1
    assert lib.fe_sum_f32(16, None, 2, 8, None) == 1
    assert lib.fe_sum_f32(16, srcs, 0, 8, None) == 1          # no sources
    assert lib.fe_sum_f32(16, srcs, 9, 8, None) == 1          # more than 8
    assert lib.fe_sum_f32(8, srcs, 2, 8, None) == 1           # misaligned destination
    assert lib.fe_sum_f32(16, srcs, 2, 0, None) == 0          # nothing to add


def test_fst_sizes_and_host_side_status_codes(lib):
    import numpy as np
    from paper_2503_06161_gb300 import synth
    for levels, rs, rt, D in [(1, 4, 4, 16), (4, 64, 100, 32), (3, 6, 7, 128)]:
        want_p = sum(a * b * c for a, b, c in synth.fst_plane_shapes(levels, rs, rt))
        want_m = sum(o * i + o for o, i in synth.fst_layer_shapes(levels, D))
        assert lib.fe_fst_plane_floats(levels, rs, rt) == want_p
        assert lib.fe_fst_mlp_floats(levels, D) == want_m
    assert lib.fe_fst_plane_floats(0, 4, 4) == 0 and lib.fe_fst_plane_floats(5, 4, 4) == 0
    assert lib.fe_fst_plane_floats(2, 1, 4) == 0 and lib.fe_fst_mlp_floats(2, 24) == 0
    n = ctypes.c_size_t(0)
    assert lib.fe_fst_workspace_size(1000, 4, 8, 6, 32, 0, ctypes.byref(n)) == 0
    fwd_only = n.value
    assert lib.fe_fst_workspace_size(1000, 4, 8, 6, 32, 1, ctypes.byref(n)) == 0
    assert n.value > fwd_only + 1000 * 4 * 900      # the activations kept for the reverse pass
    with_bwd = n.value
    assert lib.fe_fst_workspace_size(1000, 4, 8, 6, 32, 2, ctypes.byref(n)) == 0
    assert n.value >= with_bwd + 16 * lib.fe_fst_plane_floats(4, 8, 6)      # exact plane accumulators
    assert lib.fe_fst_workspace_size(1000, 4, 8, 6, 32, 3, ctypes.byref(n)) == 1
    assert lib.fe_fst_workspace_size(1000, 4, 8, 6, 24, 1, ctypes.byref(n)) == 4   # D not compiled in
    assert lib.fe_fst_workspace_size(-1, 4, 8, 6, 32, 1, ctypes.byref(n)) == 1
    assert lib.fe_fst_workspace_size(1000, 4, 1, 6, 32, 1, ctypes.byref(n)) == 1    # rs < 2
    f = _lib.fe_fst()
    f.levels, f.rs, f.rt, f.D = 2, 8, 6, 32
    for a in range(3):
        f.bbox_max[a] = 1.0
    ws = ctypes.c_void_p(256)
    args = [None] * 5
    assert lib.fe_fst_forward(None, 1, *args, 0, 0.5, *args, ws, 1 << 30, 1, None) == 1
    assert lib.fe_fst_forward(ctypes.byref(f), 1, *args, 0, 0.5, *args, ws, 16, 1, None) == 3   # workspace
    assert lib.fe_fst_forward(ctypes.byref(f), 1, *args, 0, 0.5, *args, ws, 1 << 30, 1, None) == 1  # NULLs
    f.D = 24
    assert lib.fe_fst_forward(ctypes.byref(f), 1, *args, 0, 0.5, *args, ws, 1 << 30, 1, None) == 4
    f.bbox_max[1] = 1.0
    f.D, f.planes = 32, 1 << 20
    n_pl = lib.fe_fst_plane_floats(2, 8, 6)
    for d in (1 << 20, (1 << 20) + 4 * (n_pl - 1), (1 << 20) - 4 * (n_pl - 1)):   # d_planes overlapping the planes
        assert lib.fe_fst_tv(ctypes.byref(f), 0.03, ws, ctypes.c_void_p(d), ws, None) == 1
    assert lib.fe_fst_tv(ctypes.byref(f), 0.03, None, ctypes.c_void_p(1 << 24), ws, None) == 1      # NULL loss
    f.bbox_max[1] = -1.0                                                 # empty box
    assert lib.fe_fst_forward(ctypes.byref(f), 1, *args, 0, 0.5, *args, ws, 1 << 30, 1, None) == 1


def test_density_host_side_status_codes(lib):
    """Every case is refused on the host, before any CUDA call."""
    buf = ctypes.create_string_buffer(1 << 16)
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    ws, n_ws = ctypes.c_void_p(base), 4096
    assert lib.fe_densify_workspace_size(1000) >= 1000 and lib.fe_densify_workspace_size(-1) == 0
    attrs = (_lib.fe_attr * 2)()
    attrs[0].src, attrs[0].dst, attrs[0].width, attrs[0].elem_bytes, attrs[0].role = base, base + 64, 3, 4, 1
    attrs[1].src, attrs[1].dst, attrs[1].width, attrs[1].elem_bytes, attrs[1].role = base, base + 128, 4, 4, 3
    a = _lib.fe_densify_args()
    a.P = 10
    for f in ("means", "log_scales", "quats", "opacity_logits", "accum", "count", "normals"):
        setattr(a, f, base)
    a.grad_thresh, a.dense_scale, a.min_opacity = 2e-4, 0.05, 0.005
    a.attrs, a.nattrs, a.capacity = ctypes.cast(attrs, ctypes.c_void_p), 2, 20
    new_p = ctypes.c_void_p(base + 512)
    assert lib.fe_densify(None, new_p, ws, n_ws, None) == 1
    assert lib.fe_densify(ctypes.byref(a), None, ws, n_ws, None) == 1
    a.capacity = 19                                                            # < 2 P
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    a.capacity = 20
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, 16, None) == 3           # workspace
    assert lib.fe_densify(ctypes.byref(a), new_p, ctypes.c_void_p(base + 8), n_ws, None) == 1   # unaligned
    a.nattrs = 0
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    a.nattrs = 33
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    a.nattrs = 2
    attrs[0].width = 4                                                         # means must be [P][3]
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    attrs[0].width, attrs[0].elem_bytes = 3, 2                                 # and float32
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    attrs[0].elem_bytes, attrs[0].dst = 4, base                                # dst aliases src
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    attrs[0].dst, attrs[1].role = base + 64, 4                                 # unknown role
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    attrs[1].role, a.quats = 3, base + 2                                       # unaligned floats
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    a.quats, a.normals = base, None
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    a.normals, a.dense_scale = base, float("nan")
    assert lib.fe_densify(ctypes.byref(a), new_p, ws, n_ws, None) == 1
    for m in (0.0, 1.0, -0.5, float("nan")):
        assert lib.fe_reset_opacity(ctypes.c_void_p(base), 10, m, None) == 1
    assert lib.fe_reset_opacity(None, 10, 0.01, None) == 1
    assert lib.fe_reset_opacity(None, 0, 0.01, None) == 0                     # nothing to do
    assert lib.fe_reset_opacity(ctypes.c_void_p(base), -1, 0.01, None) == 1
    opts = _lib.make_opts()
    assert lib.fe_screen_grad_stats(None, 1 << 30, 10, 32, 64, 64, ctypes.byref(opts), base, base, None) == 1
    assert lib.fe_screen_grad_stats(ws, 1 << 30, 10, 32, 64, 64, ctypes.byref(opts), None, base, None) == 1
    assert lib.fe_screen_grad_stats(ws, 16, 10, 32, 64, 64, ctypes.byref(opts), base, base, None) == 3
    assert lib.fe_screen_grad_stats(ws, 1 << 30, 10, 24, 64, 64, ctypes.byref(opts), base, base, None) == 4
    fwd = _lib.make_opts(forward_only=True)
    assert lib.fe_screen_grad_stats(ws, 1 << 30, 10, 32, 64, 64, ctypes.byref(fwd), base, base, None) == 1


def test_batch_host_side_checks(lib):
    cam = _lib.make_camera(64, 48, 50.0, 50.0, 32.0, 24.0, [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1],
                           [0, 0, 0])
    small = _lib.make_camera(20, 12, 20.0, 20.0, 10.0, 6.0, [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1],
                             [0, 0, 0])
    n = ctypes.c_size_t(0)
    b = _lib.make_batch([cam, small], [0.0, 0.5], [_lib.make_opts(), _lib.make_opts(tile=(32, 8))])
    assert lib.fe_batch_workspace_size(1000, 32, ctypes.byref(b), ctypes.byref(n)) == 0
    # A 256-byte header, each view's single-view workspace (256-aligned),
    # then one gradient set per helper stream (two views: two streams).
    one = _lib.fe_workspace_size(1000, 32, 64, 48, _lib.make_opts())
    two = _lib.fe_workspace_size(1000, 32, 20, 12, _lib.make_opts(tile=(32, 8)))
    a256 = lambda x: (x + 255) // 256 * 256
    gset = sum(a256(4 * 1000 * w) for w in (3, 3, 4, 1, 48, 32))
    assert n.value == 256 + one + two + 2 * gset
    fwd_only = _lib.make_batch([cam, small], [0.0, 0.5], [_lib.make_opts(forward_only=True), _lib.make_opts()])
    assert lib.fe_batch_workspace_size(1000, 32, ctypes.byref(fwd_only), ctypes.byref(n)) == 0
    assert n.value == 256 + _lib.fe_workspace_size(1000, 32, 64, 48, _lib.make_opts(forward_only=True)) + \
        _lib.fe_workspace_size(1000, 32, 20, 12, _lib.make_opts(forward_only=True))
    assert lib.fe_batch_workspace_size(1000, 24, ctypes.byref(b), ctypes.byref(n)) == 4      # D
    b0 = _lib.make_batch([], [], [])
    assert lib.fe_batch_workspace_size(1000, 32, ctypes.byref(b0), ctypes.byref(n)) == 1     # no views
    many = _lib.make_batch([cam] * 33, [0.0] * 33, [_lib.make_opts()] * 33)
    assert lib.fe_batch_workspace_size(1000, 32, ctypes.byref(many), ctypes.byref(n)) == 1   # > FE_MAX_VIEWS
    bad_tile = _lib.make_batch([cam], [0.0], [_lib.make_opts(tile=(12, 12))])
    assert lib.fe_batch_workspace_size(1000, 32, ctypes.byref(bad_tile), ctypes.byref(n)) == 4
    assert lib.fe_render_batch(None, None, ctypes.byref(b), None, 0, None, None) == 1
    assert lib.fe_render_batch_backward(None, None, ctypes.byref(b), None, 0, None, None, None) == 1
    assert lib.fe_batch_read_stats(None, 0, 1000, 32, ctypes.byref(b), None, None) == 1


def test_injected_workspace_failures_return_a_status(lib):
    # A caller whose allocation failed passes NULL, or a buffer one byte too
    # small: every render entry point returns a status before any CUDA call
    # (the pointers below are never dereferenced).
    P, D, W, H = 100, 32, 64, 48
    o = _lib.make_opts()
    need = _lib.fe_workspace_size(P, D, W, H, o)
    cam = _lib.make_camera(W, H, 50.0, 50.0, 32.0, 24.0, [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1], [0, 0, 0])
    g = _lib.fe_gaussians()
    g.P, g.D, g.sh_degree = P, D, 3
    g.means = g.log_scales = g.quats = g.opacity_logits = g.sh = g.feat = 1 << 20
    out = _lib.fe_outputs(1 << 21, 1 << 21, 1 << 21, 1 << 21, None)
    go = _lib.fe_output_grads(None, None, None, None)
    gr = _lib.fe_grads(*([1 << 22] * 6))
    ws = ctypes.c_void_p(1 << 24)                                   # 256-byte aligned
    stats = _lib.fe_stats()
    for bytes_, want in ((need - 1, 3), (0, 3)):
        assert lib.fe_render_forward(ctypes.byref(g), None, ctypes.byref(cam), 0.0, ctypes.byref(o), ws, bytes_,
                                     ctypes.byref(out), None) == want
        assert lib.fe_render_backward(ctypes.byref(g), None, ctypes.byref(cam), 0.0, ctypes.byref(o), ws, bytes_,
                                      ctypes.byref(go), ctypes.byref(gr), None) == want
        assert lib.fe_read_stats(ws, bytes_, P, D, W, H, ctypes.byref(o), ctypes.byref(stats), None) == want
        assert lib.fe_count_pairs(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(o), ws, bytes_, ws, None) == want
    assert lib.fe_render_forward(ctypes.byref(g), None, ctypes.byref(cam), 0.0, ctypes.byref(o), None, need,
                                 ctypes.byref(out), None) == 1
    assert lib.fe_render_backward(ctypes.byref(g), None, ctypes.byref(cam), 0.0, ctypes.byref(o), None, need,
                                  ctypes.byref(go), ctypes.byref(gr), None) == 1
    assert lib.fe_render_forward(ctypes.byref(g), None, ctypes.byref(cam), 0.0, ctypes.byref(o),
                                 ctypes.c_void_p((1 << 24) + 16), need, ctypes.byref(out), None) == 1  # misaligned
    b = _lib.make_batch([cam, cam], [0.0, 1.0], [o, o])
    nb = _lib.fe_batch_workspace_size(P, D, b)
    outs = (_lib.fe_outputs * 2)(out, out)
    gos = (_lib.fe_output_grads * 2)(go, go)
    assert lib.fe_render_batch(ctypes.byref(g), None, ctypes.byref(b), ws, nb - 1, outs, None) == 3
    assert lib.fe_render_batch(ctypes.byref(g), None, ctypes.byref(b), None, nb, outs, None) == 1
    assert lib.fe_render_batch_backward(ctypes.byref(g), None, ctypes.byref(b), ws, nb - 1, gos, ctypes.byref(gr),
                                        None) == 3
    sts = (_lib.fe_stats * 2)()
    assert lib.fe_batch_read_stats(ws, nb - 1, P, D, ctypes.byref(b), sts, None) == 3
    # The Python layer refuses a shared workspace that is too small.
    import torch
    from paper_2503_06161_gb300.raster import Rasterizer
    with pytest.raises(ValueError):
        Rasterizer(P, D, W, H, device="cpu", workspace=torch.empty(need - 1, dtype=torch.uint8))
