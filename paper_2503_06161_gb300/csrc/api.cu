// C-ABI entry points declared in include/fe4dgs.h: argument checks,
// workspace layout and the launch sequence of each call.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

using namespace fe;

namespace {

constexpr int64_t kMaxCap = (1ll << 30) - 1;  // look-back words carry 30-bit counts

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fe_status resolve_opts(const fe_opts* o, int P, int& tw, int& th, int64_t& cap, bool& with_bwd, float bg[3]) {
  tw = o ? o->tile_w : 16;
  th = o ? o->tile_h : 16;
  if (tw == 0 && th == 0) tw = th = 16;
  if (tw * th != kThreads || (tw != 8 && tw != 16 && tw != 32) || (th != 8 && th != 16 && th != 32))
    return FE_ERR_UNSUPPORTED;
  cap = (o && o->max_dups > 0) ? o->max_dups : (int64_t)16 * (P > 0 ? P : 0) + 4096;
  if (cap > kMaxCap) return FE_ERR_INVALID_ARG;
  with_bwd = !(o && o->forward_only);
  for (int i = 0; i < 3; ++i) bg[i] = o ? o->bg[i] : 0.0f;
  return FE_OK;
}

bool d_supported(int D) { return D == 16 || D == 32 || D == 64 || D == 128; }

fe_status layout_for(int P, int D, int W, int H, const fe_opts* opts, Layout& L, float bg[3]) {
  if (P < 0 || W <= 0 || H <= 0) return FE_ERR_INVALID_ARG;
  if (!d_supported(D)) return FE_ERR_UNSUPPORTED;
  int tw, th;
  int64_t cap;
  bool wb;
  fe_status s = resolve_opts(opts, P, tw, th, cap, wb, bg);
  if (s != FE_OK) return s;
  const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
  if ((int64_t)tiles_x * tiles_y > kMaxTiles) return FE_ERR_UNSUPPORTED;
  L = make_layout(P, D, W, H, tw, th, cap, wb);
  return FE_OK;
}

fe_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FE_OK : FE_ERR_CUDA; }

// Profiling hook: record opts->events[i] (if any) on the stream.
cudaError_t mark(const fe_opts* o, int i, cudaStream_t st) {
  if (!o || !o->events || !o->events[i]) return cudaSuccess;
  return cudaEventRecord(static_cast<cudaEvent_t>(o->events[i]), st);
}

#define FE_TRY_CUDA(x)                      \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return FE_ERR_CUDA; \
  } while (0)

fe_status fill_gauss_args(const fe_gaussians* g, const fe_deform* df, const fe_camera* cam, float t, const Layout& L,
                          void* ws, GaussArgs& a) {
  if (!g || !cam) return FE_ERR_INVALID_ARG;
  if (g->P > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh || !g->feat))
    return FE_ERR_INVALID_ARG;
  if (g->sh_degree < 0 || g->sh_degree > 3) return FE_ERR_UNSUPPORTED;
  if (!aligned16(g->quats) || !aligned16(g->sh) || !aligned16(g->feat)) return FE_ERR_INVALID_ARG;
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !(cam->znear > 0.f)) return FE_ERR_INVALID_ARG;
  a = GaussArgs{};
  a.P = g->P;
  a.sh_degree = g->sh_degree;
  a.sh_bf16 = g->sh_bf16 ? 1 : 0;
  a.means = g->means;
  a.log_scales = g->log_scales;
  a.quats = g->quats;
  a.logits = g->opacity_logits;
  a.sh = g->sh;
  a.has_deform = df ? 1 : 0;
  if (df) {
    if (df->C != 32 && df->C != 64) return FE_ERR_UNSUPPORTED;
    if (df->R < 2 || !df->planes || !df->w1 || !df->b1 || !df->w2 || !df->b2 || !df->wh || !df->bh)
      return FE_ERR_INVALID_ARG;
    if (!aligned16(df->planes)) return FE_ERR_INVALID_ARG;
    a.C = df->C;
    a.R = df->R;
    a.planes = df->planes;
    a.w1 = df->w1; a.b1 = df->b1; a.w2 = df->w2; a.b2 = df->b2; a.wh = df->wh; a.bh = df->bh;
    for (int i = 0; i < 3; ++i) {
      if (!(df->bbox_max[i] > df->bbox_min[i])) return FE_ERR_INVALID_ARG;
      a.bmin[i] = df->bbox_min[i];
      a.bscale[i] = 2.0f / (df->bbox_max[i] - df->bbox_min[i]);
    }
    a.noise = df->noise;
    a.noise_scale = df->noise_scale;
  }
  a.t = t;
  a.W = L.W; a.H = L.H; a.tw = L.tw; a.th = L.th;
  a.fx = cam->fx; a.fy = cam->fy; a.cx = cam->cx; a.cy = cam->cy; a.znear = cam->znear;
  a.limx = 1.3f * 0.5f * (float)cam->width / cam->fx;
  a.limy = 1.3f * 0.5f * (float)cam->height / cam->fy;
  for (int i = 0; i < 12; ++i) a.V[i] = cam->world_to_cam[i];
  for (int i = 0; i < 3; ++i) a.campos[i] = cam->campos[i];
  Header* hdr = at<Header>(ws, L.hdr);
  a.rec = at<float4>(ws, L.rec);
  a.rect = at<ushort4>(ws, L.rect);
  a.touched = at<uint32_t>(ws, L.touched);
  a.dkey = at<uint32_t>(ws, L.dkey[0]);
  a.err = &hdr->err;
  a.num_visible = &hdr->num_visible;
  if (L.with_backward) a.dstate = at<float>(ws, L.dstate);
  return FE_OK;
}

BinArgs bin_args(const Layout& L, void* ws) {
  BinArgs b{};
  b.P = L.P;
  b.ntiles = L.ntiles;
  b.tiles_x = L.tiles_x;
  b.pblocks = L.pblocks;
  b.bblocks = L.bblocks;
  b.cap = L.cap;
  b.rect = at<ushort4>(ws, L.rect);
  b.touched = at<uint32_t>(ws, L.touched);
  for (int i = 0; i < 2; ++i) {
    b.dkey[i] = at<uint32_t>(ws, L.dkey[i]);
    b.dval[i] = at<uint32_t>(ws, L.dval[i]);
  }
  b.offs = at<uint32_t>(ws, L.offs);
  b.offs_by_gid = at<uint32_t>(ws, L.offs_by_gid);
  b.sorted = at<uint2>(ws, L.sorted);
  b.table = at<uint32_t>(ws, L.table);
  b.status = at<uint32_t>(ws, L.status);
  b.hist = at<uint32_t>(ws, L.hist);
  b.ranges = at<uint2>(ws, L.ranges);
  b.hdr = at<Header>(ws, L.hdr);
  return b;
}

// Clears the per-call state: header, histograms, look-back words, ranges.
fe_status clear_state(const Layout& L, void* ws, cudaStream_t st) {
  FE_TRY_CUDA(cudaMemsetAsync(at<char>(ws, L.hdr), 0, sizeof(Header), st));
  FE_TRY_CUDA(cudaMemsetAsync(at<char>(ws, L.hist), 0, (4 + 3) * 256 * 4, st));
  FE_TRY_CUDA(cudaMemsetAsync(at<char>(ws, L.status), 0, L.status_words * 4, st));
  FE_TRY_CUDA(cudaMemsetAsync(at<char>(ws, L.ranges), 0, (size_t)L.ntiles * 8, st));
  return FE_OK;
}

CompositeArgs composite_args(const Layout& L, void* ws, int feat_bf16, const void* feat, const float bg[3]) {
  CompositeArgs c{};
  c.W = L.W; c.H = L.H; c.tw = L.tw; c.th = L.th; c.tiles_x = L.tiles_x; c.D = L.D;
  c.feat_bf16 = feat_bf16;
  for (int i = 0; i < 3; ++i) c.bg[i] = bg[i];
  c.ranges = at<uint2>(ws, L.ranges);
  c.sorted = at<uint2>(ws, L.sorted);
  c.rec = at<float4>(ws, L.rec);
  c.feat = feat;
  c.t_final = at<float>(ws, L.tfinal);
  c.n_contrib = at<uint32_t>(ws, L.ncontrib);
  c.ntiles = L.ntiles;
  c.cap = L.cap;
  c.err = &at<Header>(ws, L.hdr)->err;
  if (L.with_backward) {
    c.partials = at<float>(ws, L.partials);
    c.pflags = at<uint32_t>(ws, L.pflags);
    c.cmask = at<uint32_t>(ws, L.cmask);
  }
  return c;
}

}  // namespace

extern "C" {

const char* fe_status_string(fe_status s) {
  switch (s) {
    case FE_OK: return "ok";
    case FE_ERR_INVALID_ARG: return "invalid argument";
    case FE_ERR_CUDA: return "CUDA runtime error";
    case FE_ERR_WORKSPACE: return "workspace too small or duplicate capacity exceeded";
    case FE_ERR_UNSUPPORTED: return "unsupported configuration (D, channels, SH degree or tile shape)";
    case FE_ERR_NONFINITE: return "non-finite Gaussian parameter";
    case FE_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case FE_ERR_STATE: return "backward without a matching forward";
  }
  return "unknown status";
}

fe_status fe_workspace_size(int P, int D, int width, int height, const fe_opts* opts, size_t* bytes) {
  if (!bytes) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(P, D, width, height, opts, L, bg);
  if (s != FE_OK) return s;
  *bytes = L.total;
  return FE_OK;
}

fe_status fe_render_forward(const fe_gaussians* g, const fe_deform* deform, const fe_camera* cam, float t,
                            const fe_opts* opts, void* workspace, size_t workspace_bytes, const fe_outputs* out,
                            void* stream) {
  if (!g || !cam || !out || !workspace) return FE_ERR_INVALID_ARG;
  if (!out->rgb || !out->depth || !out->alpha || !out->feat || !aligned16(out->feat)) return FE_ERR_INVALID_ARG;
  if (out->feat_bf16 && !aligned16(out->feat_bf16)) return FE_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(g->P, g->D, cam->width, cam->height, opts, L, bg);
  if (s != FE_OK) return s;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GaussArgs ga;
  if ((s = fill_gauss_args(g, deform, cam, t, L, workspace, ga)) != FE_OK) return s;
  if ((s = clear_state(L, workspace, st)) != FE_OK) return s;
  FE_TRY_CUDA(mark(opts, 0, st));
  FE_TRY_CUDA(launch_gauss_fwd(ga, st));
  FE_TRY_CUDA(mark(opts, 1, st));
  BinArgs b = bin_args(L, workspace);
  FE_TRY_CUDA(launch_binning(b, st));
  FE_TRY_CUDA(mark(opts, 2, st));
  CompositeArgs c = composite_args(L, workspace, g->feat_bf16, g->feat, bg);
  c.out_rgb = out->rgb;
  c.out_depth = out->depth;
  c.out_alpha = out->alpha;
  c.out_feat = out->feat;
  c.out_feat_bf16 = static_cast<uint16_t*>(out->feat_bf16);
  FE_TRY_CUDA(launch_composite_fwd(c, st));
  FE_TRY_CUDA(mark(opts, 3, st));
  return FE_OK;
}

fe_status fe_render_backward(const fe_gaussians* g, const fe_deform* deform, const fe_camera* cam, float t,
                             const fe_opts* opts, void* workspace, size_t workspace_bytes,
                             const fe_output_grads* grad_out, const fe_grads* grads, void* stream) {
  if (!g || !cam || !grad_out || !grads || !workspace) return FE_ERR_INVALID_ARG;
  if (g->P > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh ||
                   !grads->feat))
    return FE_ERR_INVALID_ARG;
  if (!aligned16(grads->quats) || !aligned16(grads->sh) || !aligned16(grads->feat)) return FE_ERR_INVALID_ARG;
  if (grad_out->feat && !aligned16(grad_out->feat)) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(g->P, g->D, cam->width, cam->height, opts, L, bg);
  if (s != FE_OK) return s;
  if (!L.with_backward) return FE_ERR_INVALID_ARG;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GaussArgs ga;
  if ((s = fill_gauss_args(g, deform, cam, t, L, workspace, ga)) != FE_OK) return s;
  FE_TRY_CUDA(cudaMemsetAsync(at<char>(workspace, L.pflags), 0, ((size_t)L.cap + 31) / 32 * 4, st));
  FE_TRY_CUDA(mark(opts, 4, st));
  CompositeArgs c = composite_args(L, workspace, g->feat_bf16, g->feat, bg);
  c.g_rgb = grad_out->rgb;
  c.g_depth = grad_out->depth;
  c.g_alpha = grad_out->alpha;
  c.g_feat = grad_out->feat;
  FE_TRY_CUDA(launch_composite_bwd(c, st));
  FE_TRY_CUDA(mark(opts, 5, st));
  GaussBwdArgs gb{};
  gb.D = L.D;
  gb.cap = L.cap;
  gb.touched = at<uint32_t>(workspace, L.touched);
  gb.offs_by_gid = at<uint32_t>(workspace, L.offs_by_gid);
  gb.partials = at<float>(workspace, L.partials);
  gb.pflags = at<uint32_t>(workspace, L.pflags);
  gb.d_means = grads->means;
  gb.d_log_scales = grads->log_scales;
  gb.d_quats = grads->quats;
  gb.d_logits = grads->opacity_logits;
  gb.d_sh = grads->sh;
  gb.d_feat = grads->feat;
  gb.ddstate = at<float>(workspace, L.ddstate);
  gb.psum = at<float>(workspace, L.psum);
  gb.accumulate = opts && opts->accumulate_grads ? 1 : 0;
  FE_TRY_CUDA(launch_gauss_bwd(ga, gb, st, opts && opts->events ? static_cast<cudaEvent_t>(opts->events[6]) : nullptr));
  FE_TRY_CUDA(mark(opts, 7, st));
  return FE_OK;
}

fe_status fe_tile_bin(int P, const float* uv, const int* radius, const float* depth, int width, int height,
                      const fe_opts* opts, void* workspace, size_t workspace_bytes, void* stream) {
  if (P < 0 || !workspace || (P > 0 && (!uv || !radius || !depth))) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(P, 16, width, height, opts, L, bg);
  if (s != FE_OK) return s;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = clear_state(L, workspace, st)) != FE_OK) return s;
  Header* hdr = at<Header>(workspace, L.hdr);
  FE_TRY_CUDA(launch_bin_prep(P, uv, radius, depth, width, height, L.tw, L.th, at<ushort4>(workspace, L.rect),
                              at<uint32_t>(workspace, L.touched), at<uint32_t>(workspace, L.dkey[0]),
                              &hdr->num_visible, st));
  // The dump reconstructs keys from the record's depth slot: store depths there.
  if (P > 0) {
    FE_TRY_CUDA(cudaMemsetAsync(at<char>(workspace, L.rec), 0, (size_t)P * kRec * 4, st));
    FE_TRY_CUDA(cudaMemcpy2DAsync(at<char>(workspace, L.rec) + 6 * 4, kRec * 4, depth, 4, 4, P,
                                  cudaMemcpyDeviceToDevice, st));
  }
  BinArgs b = bin_args(L, workspace);
  FE_TRY_CUDA(launch_binning(b, st));
  return FE_OK;
}

fe_status fe_read_stats(const void* workspace, size_t workspace_bytes, int P, int D, int width, int height,
                        const fe_opts* opts, fe_stats* stats, void* stream) {
  if (!workspace || !stats) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(P, D, width, height, opts, L, bg);
  if (s != FE_OK) return s;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  FE_TRY_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  Header h;
  FE_TRY_CUDA(cudaMemcpy(&h, at<char>(const_cast<void*>(workspace), L.hdr), sizeof(Header), cudaMemcpyDeviceToHost));
  stats->num_dups = h.num_dups;
  stats->capacity = L.cap;
  stats->num_visible = h.num_visible;
  stats->device_errors = h.err;
  stats->has_forward = (int32_t)h.has_forward;
  if (h.err & kErrTimeout) return FE_ERR_TIMEOUT;
  if (h.err & kErrOverflow) return FE_ERR_WORKSPACE;
  if (h.err & kErrNonFinite) return FE_ERR_NONFINITE;
  return FE_OK;
}

fe_status fe_screen_grad_stats(const void* workspace, size_t workspace_bytes, int P, int D, int width, int height,
                               const fe_opts* opts, float* accum, int32_t* count, void* stream) {
  if (!workspace || (P > 0 && (!accum || !count))) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(P, D, width, height, opts, L, bg);
  if (s != FE_OK) return s;
  if (!L.with_backward) return FE_ERR_INVALID_ARG;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  void* ws = const_cast<void*>(workspace);
  // psum[g][0..1] hold dL/du and dL/dv of the last fe_render_backward.
  return cuda_status(launch_screen_stats(at<uint32_t>(ws, L.touched), at<float>(ws, L.psum), P, width, height, accum,
                                         count, static_cast<cudaStream_t>(stream)));
}

fe_status fe_debug_dump(const void* workspace, size_t workspace_bytes, int P, int D, int width, int height,
                        const fe_opts* opts, uint64_t* keys, uint32_t* gauss, uint32_t* ranges, uint32_t* n_contrib,
                        float* t_final, float* uv, float* conic, float* opacity, float* depth, float* rgb,
                        int32_t* radius, uint32_t* touched, void* stream) {
  if (!workspace) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(P, D, width, height, opts, L, bg);
  if (s != FE_OK) return s;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  void* ws = const_cast<void*>(workspace);
  DumpArgs d{};
  d.cap = L.cap;
  d.P = P;
  d.ntiles = L.ntiles;
  d.HW = width * height;
  d.hdr = at<Header>(ws, L.hdr);
  d.sorted = at<uint2>(ws, L.sorted);
  d.ranges = at<uint2>(ws, L.ranges);
  d.ncontrib = at<uint32_t>(ws, L.ncontrib);
  d.tfinal = at<float>(ws, L.tfinal);
  d.rec = at<float4>(ws, L.rec);
  d.touched = at<uint32_t>(ws, L.touched);
  d.keys = keys; d.gauss = gauss; d.ranges_out = ranges; d.ncontrib_out = n_contrib; d.tfinal_out = t_final;
  d.uv = uv; d.conic = conic; d.opacity = opacity; d.depth = depth; d.rgb = rgb; d.radius = radius;
  d.touched_out = touched;
  return cuda_status(launch_dump(d, static_cast<cudaStream_t>(stream)));
}

fe_status fe_l1_loss_grad(const float* pred, const float* target, int64_t n, int64_t rows, float* grad, float* loss,
                          float* scratch, void* stream) {
  if (n < 0 || rows <= 0 || (n > 0 && (!pred || !target || !grad)) || !loss || !scratch) return FE_ERR_INVALID_ARG;
  return cuda_status(launch_l1(pred, target, n, rows, grad, loss, scratch, static_cast<cudaStream_t>(stream)));
}

fe_status fe_count_pairs(const fe_gaussians* g, const fe_camera* cam, const fe_opts* opts, void* workspace,
                         size_t workspace_bytes, uint64_t* counts, void* stream) {
  if (!g || !cam || !workspace || !counts) return FE_ERR_INVALID_ARG;
  Layout L;
  float bg[3];
  fe_status s = layout_for(g->P, g->D, cam->width, cam->height, opts, L, bg);
  if (s != FE_OK) return s;
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FE_TRY_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(uint64_t), st));
  CompositeArgs c = composite_args(L, workspace, g->feat_bf16, g->feat, bg);
  c.counts = counts;
  return cuda_status(launch_composite_fwd(c, st));
}

fe_status fe_probe_fp32_peak(int iters, double* flops, void* stream) {
  if (iters <= 0 || !flops) return FE_ERR_INVALID_ARG;
  return cuda_status(probe_fp32(iters, flops, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
