// C-ABI entry points declared in include/fe4dgs.h: argument checks,
// workspace layout and the launch sequence of each call.
#include <algorithm>
#include <cmath>
#include <memory>
#include <mutex>
#include <new>

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

bool d_supported(int D) { return D == 16 || D == 32 || D == 64 || D == 128 || D == 256; }

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
  a.dstate = at<float>(ws, L.dstate);
  a.fsplit = at<uint16_t>(ws, L.fsplit);
  return FE_OK;
}

GaussBwdArgs gauss_bwd_args(const Layout& L, void* ws, const fe_grads* grads, int accumulate) {
  GaussBwdArgs gb{};
  gb.D = L.D;
  gb.cap = L.cap;
  gb.touched = at<uint32_t>(ws, L.touched);
  gb.offs_by_gid = at<uint32_t>(ws, L.offs_by_gid);
  gb.order = at<uint32_t>(ws, L.dval[0]);
  gb.offs = at<uint32_t>(ws, L.offs);
  gb.partials = at<float>(ws, L.partials);
  gb.pflags = at<uint32_t>(ws, L.pflags);
  gb.d_means = grads->means;
  gb.d_log_scales = grads->log_scales;
  gb.d_quats = grads->quats;
  gb.d_logits = grads->opacity_logits;
  gb.d_sh = grads->sh;
  gb.d_feat = grads->feat;
  gb.ddstate = at<float>(ws, L.ddstate);
  gb.psum = at<float>(ws, L.psum);
  gb.accumulate = accumulate;
  return gb;
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

// Staging-wait bound of the compositing kernels (fe_opts.wait_polls).
int wait_polls(const fe_opts* o) {
  if (!o || o->wait_polls == 0) return kWaitPolls;
  return o->wait_polls < 0 ? 0 : o->wait_polls;
}

CompositeArgs composite_args(const Layout& L, void* ws, int feat_bf16, const void* feat, const float bg[3],
                             const fe_opts* o) {
  CompositeArgs c{};
  c.polls = wait_polls(o);
  c.feat_row_bytes = (uint32_t)L.D * (feat_bf16 ? 2u : 4u);
  c.out_ld = L.D;
  c.prow = partial_stride(L.D);
  c.pcol0 = 0;
  c.pscal = L.D;
  c.aux = 1;
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

// ---------------------------------------------------------------------------
// Batched views: a 256-byte batch header (the two work-item counters of the
// persistent compositing launches), then one single-view workspace per view.
// ---------------------------------------------------------------------------
static_assert(FE_MAX_VIEWS == kMaxViews, "view limit of the ABI and the kernels");

// Per-view per-Gaussian stages (deformation, projection, binning; their
// reverse) run on up to this many helper streams forked from the caller's
// stream, views dealt round-robin; the reverse's gradient sums of each
// helper stream go to a buffer of its own in the workspace.
constexpr int kBatchStreams = 4;
constexpr int kGradArrays = 6;  // means, log_scales, quats, opacity logits, sh, feat

struct BatchLayout {
  int V, S;
  Layout L[kMaxViews];
  size_t off[kMaxViews];
  float bg[kMaxViews][3];
  size_t gset[kBatchStreams];   // offsets of the per-stream gradient sets (S > 1, with backward)
  size_t garr[kGradArrays];     // offsets of the arrays within a set
  int64_t gn[kGradArrays];      // floats per array
  size_t total;
};

fe_status batch_layout(int P, int D, const fe_batch* b, BatchLayout& B) {
  if (!b || b->V < 1 || b->V > kMaxViews || !b->cams || !b->t || !b->opts) return FE_ERR_INVALID_ARG;
  B.V = b->V;
  B.S = b->V < kBatchStreams ? b->V : kBatchStreams;
  size_t off = 256;
  for (int v = 0; v < b->V; ++v) {
    fe_opts o = b->opts[v];
    o.forward_only = b->opts[0].forward_only;
    const fe_status s = layout_for(P, D, b->cams[v].width, b->cams[v].height, &o, B.L[v], B.bg[v]);
    if (s != FE_OK) return s;
    B.off[v] = off;
    off = align_up(off + B.L[v].total, 256);
  }
  const int64_t Pn = P > 0 ? P : 0;
  const int64_t widths[kGradArrays] = {3, 3, 4, 1, 48, D};
  size_t set_bytes = 0;
  for (int k = 0; k < kGradArrays; ++k) {
    B.gn[k] = Pn * widths[k];
    B.garr[k] = set_bytes;
    set_bytes = align_up(set_bytes + (size_t)B.gn[k] * 4, 256);
  }
  if (B.S > 1 && B.L[0].with_backward)
    for (int i = 0; i < B.S; ++i) {
      B.gset[i] = off;
      off += set_bytes;
    }
  B.total = off;
  return FE_OK;
}

// Helper streams and events of the batched calls, one set per device,
// created on first use.  Calls that use a set hold its lock while they
// enqueue, so concurrent callers cannot interleave their fork / join.
struct StreamPool {
  bool ready = false;
  cudaStream_t s[kBatchStreams];
  cudaEvent_t fork, join[kBatchStreams];
  std::mutex mu;
};
constexpr int kPoolDevices = 64;
StreamPool g_pools[kPoolDevices];
std::mutex g_pools_mu;

cudaError_t stream_pool(StreamPool*& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pools_mu);
  StreamPool& p = g_pools[dev];
  if (!p.ready) {
    int made = 0, ev = 0;
    for (; made < kBatchStreams; ++made)
      if ((e = cudaStreamCreateWithFlags(&p.s[made], cudaStreamNonBlocking)) != cudaSuccess) break;
    if (e == cudaSuccess && (e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming)) == cudaSuccess) {
      ev = 1;
      for (int i = 0; i < kBatchStreams && e == cudaSuccess; ++i)
        if ((e = cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming)) == cudaSuccess) ++ev;
    }
    if (e != cudaSuccess) {
      for (int i = 0; i < made; ++i) cudaStreamDestroy(p.s[i]);
      if (ev > 0) cudaEventDestroy(p.fork);
      for (int i = 0; i + 1 < ev; ++i) cudaEventDestroy(p.join[i]);
      return e;
    }
    p.ready = true;
  }
  out = &p;
  return cudaSuccess;
}

// The helper streams wait for everything enqueued on `st` so far.
cudaError_t fork_streams(StreamPool& p, int S, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(p.fork, st);
  for (int i = 0; i < S && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(p.s[i], p.fork, 0);
  return e;
}

// `st` waits for everything enqueued on the helper streams so far.
cudaError_t join_streams(StreamPool& p, int S, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = cudaEventRecord(p.join[i], p.s[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p.join[i], 0);
  }
  return e;
}

// Work-item order of the persistent launches: views by decreasing pixel
// count (the largest views' tiles are taken first), ties in view order.
void batch_order(const BatchLayout& B, int order[kMaxViews]) {
  for (int v = 0; v < B.V; ++v) order[v] = v;
  std::stable_sort(order, order + B.V, [&](int a, int c) {
    return (int64_t)B.L[a].W * B.L[a].H > (int64_t)B.L[c].W * B.L[c].H;
  });
}

void batch_items(const BatchLayout& B, const CompositeArgs* per_view, void* ws, int queue_slot, BatchCompositeArgs& ba) {
  int order[kMaxViews];
  batch_order(B, order);
  ba.V = B.V;
  int n = 0;
  for (int i = 0; i < B.V; ++i) {
    ba.view[i] = per_view[order[i]];
    ba.item_start[i] = n;
    n += B.L[order[i]].ntiles;
  }
  ba.item_start[B.V] = n;
  ba.nitems = n;
  ba.queue = static_cast<uint32_t*>(ws) + queue_slot;
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
  if (opts && !fwd_batch_supported(opts->fwd_batch)) return FE_ERR_UNSUPPORTED;
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
  CompositeArgs c = composite_args(L, workspace, g->feat_bf16, g->feat, bg, opts);
  c.out_rgb = out->rgb;
  c.out_depth = out->depth;
  c.out_alpha = out->alpha;
  c.out_feat = out->feat;
  c.out_feat_bf16 = static_cast<uint16_t*>(out->feat_bf16);
  FE_TRY_CUDA(launch_composite_fwd(c, opts ? opts->fwd_batch : 0, st));
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
  CompositeArgs c = composite_args(L, workspace, g->feat_bf16, g->feat, bg, opts);
  c.g_rgb = grad_out->rgb;
  c.g_depth = grad_out->depth;
  c.g_alpha = grad_out->alpha;
  c.g_feat = grad_out->feat;
  FE_TRY_CUDA(launch_composite_bwd(c, st));
  FE_TRY_CUDA(mark(opts, 5, st));
  const GaussBwdArgs gb = gauss_bwd_args(L, workspace, grads, opts && opts->accumulate_grads ? 1 : 0);
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
  return cuda_status(launch_screen_stats(at<float4>(ws, L.rec), at<float>(ws, L.psum), P, width, height, accum,
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
  CompositeArgs c = composite_args(L, workspace, g->feat_bf16, g->feat, bg, opts);
  c.counts = counts;
  return cuda_status(launch_composite_fwd(c, 0, st));
}

fe_status fe_batch_workspace_size(int P, int D, const fe_batch* b, size_t* bytes) {
  if (!bytes) return FE_ERR_INVALID_ARG;
  std::unique_ptr<BatchLayout> BL(new (std::nothrow) BatchLayout);  // large: kept off the stack
  if (!BL) return FE_ERR_WORKSPACE;
  const fe_status s = batch_layout(P, D, b, *BL);
  if (s == FE_OK) *bytes = BL->total;
  return s;
}

fe_status fe_render_batch(const fe_gaussians* g, const fe_deform* deform, const fe_batch* b, void* workspace,
                          size_t workspace_bytes, const fe_outputs* out, void* stream) {
  if (!g || !b || !out || !workspace) return FE_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return FE_ERR_INVALID_ARG;
  std::unique_ptr<BatchLayout> BL(new (std::nothrow) BatchLayout);
  if (!BL) return FE_ERR_WORKSPACE;
  fe_status s = batch_layout(g->P, g->D, b, *BL);
  if (s != FE_OK) return s;
  if (workspace_bytes < BL->total) return FE_ERR_WORKSPACE;
  const fe_opts* o0 = &b->opts[0];
  if (!fwd_batch_supported(o0->fwd_batch)) return FE_ERR_UNSUPPORTED;
  for (int v = 0; v < b->V; ++v) {
    const fe_outputs& ov = out[v];
    if (!ov.rgb || !ov.depth || !ov.alpha || !ov.feat || !aligned16(ov.feat)) return FE_ERR_INVALID_ARG;
    if (ov.feat_bf16 && !aligned16(ov.feat_bf16)) return FE_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::unique_ptr<BatchCompositeArgs> ba(new (std::nothrow) BatchCompositeArgs());
  std::unique_ptr<CompositeArgs[]> cv(new (std::nothrow) CompositeArgs[kMaxViews]);
  if (!ba || !cv) return FE_ERR_WORKSPACE;
  const int S = BL->S;
  StreamPool* pool = nullptr;
  if (S > 1) FE_TRY_CUDA(stream_pool(pool));
  std::unique_lock<std::mutex> lk;
  if (pool) lk = std::unique_lock<std::mutex>(pool->mu);
  FE_TRY_CUDA(cudaMemsetAsync(workspace, 0, 256, st));
  FE_TRY_CUDA(mark(o0, 0, st));
  if (pool) FE_TRY_CUDA(fork_streams(*pool, S, st));
  for (int v = 0; v < b->V; ++v) {
    const Layout& L = BL->L[v];
    void* ws = static_cast<char*>(workspace) + BL->off[v];
    cudaStream_t vs = pool ? pool->s[v % S] : st;
    GaussArgs ga;
    if ((s = fill_gauss_args(g, deform, &b->cams[v], b->t[v], L, ws, ga)) != FE_OK) return s;
    if ((s = clear_state(L, ws, vs)) != FE_OK) return s;
    FE_TRY_CUDA(launch_gauss_fwd(ga, vs));
    BinArgs bn = bin_args(L, ws);
    FE_TRY_CUDA(launch_binning(bn, vs));
    CompositeArgs c = composite_args(L, ws, g->feat_bf16, g->feat, BL->bg[v], o0);
    c.out_rgb = out[v].rgb;
    c.out_depth = out[v].depth;
    c.out_alpha = out[v].alpha;
    c.out_feat = out[v].feat;
    c.out_feat_bf16 = static_cast<uint16_t*>(out[v].feat_bf16);
    cv[v] = c;
  }
  if (pool) FE_TRY_CUDA(join_streams(*pool, S, st));
  batch_items(*BL, cv.get(), workspace, 0, *ba);
  FE_TRY_CUDA(mark(o0, 1, st));
  FE_TRY_CUDA(launch_composite_fwd_batch(*ba, g->D, g->feat_bf16, o0->fwd_batch, st));
  FE_TRY_CUDA(mark(o0, 2, st));
  return FE_OK;
}

fe_status fe_render_batch_backward(const fe_gaussians* g, const fe_deform* deform, const fe_batch* b,
                                   void* workspace, size_t workspace_bytes, const fe_output_grads* grad_out,
                                   const fe_grads* grads, void* stream) {
  if (!g || !b || !grad_out || !grads || !workspace) return FE_ERR_INVALID_ARG;
  if (g->P > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh ||
                   !grads->feat))
    return FE_ERR_INVALID_ARG;
  if (!aligned16(grads->quats) || !aligned16(grads->sh) || !aligned16(grads->feat)) return FE_ERR_INVALID_ARG;
  std::unique_ptr<BatchLayout> BL(new (std::nothrow) BatchLayout);
  if (!BL) return FE_ERR_WORKSPACE;
  fe_status s = batch_layout(g->P, g->D, b, *BL);
  if (s != FE_OK) return s;
  if (!BL->L[0].with_backward) return FE_ERR_INVALID_ARG;
  if (workspace_bytes < BL->total) return FE_ERR_WORKSPACE;
  for (int v = 0; v < b->V; ++v)
    if (grad_out[v].feat && !aligned16(grad_out[v].feat)) return FE_ERR_INVALID_ARG;
  const fe_opts* o0 = &b->opts[0];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::unique_ptr<BatchCompositeArgs> ba(new (std::nothrow) BatchCompositeArgs());
  std::unique_ptr<CompositeArgs[]> cv(new (std::nothrow) CompositeArgs[kMaxViews]);
  if (!ba || !cv) return FE_ERR_WORKSPACE;
  FE_TRY_CUDA(cudaMemsetAsync(static_cast<uint32_t*>(workspace) + 1, 0, 4, st));      // reverse counters
  FE_TRY_CUDA(cudaMemsetAsync(static_cast<uint32_t*>(workspace) + 3, 0, 4, st));      // (second channel half)
  for (int v = 0; v < b->V; ++v) {
    const Layout& L = BL->L[v];
    void* ws = static_cast<char*>(workspace) + BL->off[v];
    FE_TRY_CUDA(cudaMemsetAsync(at<char>(ws, L.pflags), 0, ((size_t)L.cap + 31) / 32 * 4, st));
    CompositeArgs c = composite_args(L, ws, g->feat_bf16, g->feat, BL->bg[v], o0);
    c.g_rgb = grad_out[v].rgb;
    c.g_depth = grad_out[v].depth;
    c.g_alpha = grad_out[v].alpha;
    c.g_feat = grad_out[v].feat;
    cv[v] = c;
  }
  batch_items(*BL, cv.get(), workspace, 1, *ba);
  FE_TRY_CUDA(mark(o0, 4, st));
  FE_TRY_CUDA(launch_composite_bwd_batch(*ba, g->D, g->feat_bf16, st));
  FE_TRY_CUDA(mark(o0, 5, st));
  // Per-Gaussian reverse of each view.  One stream: summed into grads in
  // view order.  S helper streams: stream i sums views i, i + S, ... in
  // order into its own gradient set, then the sets are added in stream
  // order (after grads itself when accumulating).
  const int S = BL->S;
  StreamPool* pool = nullptr;
  if (S > 1) FE_TRY_CUDA(stream_pool(pool));
  std::unique_lock<std::mutex> lk;
  if (pool) {
    lk = std::unique_lock<std::mutex>(pool->mu);
    FE_TRY_CUDA(fork_streams(*pool, S, st));
  }
  float* dst[kGradArrays] = {grads->means, grads->log_scales, grads->quats, grads->opacity_logits, grads->sh,
                             grads->feat};
  for (int v = 0; v < b->V; ++v) {
    const Layout& L = BL->L[v];
    void* ws = static_cast<char*>(workspace) + BL->off[v];
    GaussArgs ga;
    if ((s = fill_gauss_args(g, deform, &b->cams[v], b->t[v], L, ws, ga)) != FE_OK) return s;
    if (!pool) {
      const GaussBwdArgs gb = gauss_bwd_args(L, ws, grads, (v > 0 || o0->accumulate_grads) ? 1 : 0);
      FE_TRY_CUDA(launch_gauss_bwd(ga, gb, st, nullptr));
      continue;
    }
    char* set = static_cast<char*>(workspace) + BL->gset[v % S];
    fe_grads gs;
    gs.means = reinterpret_cast<float*>(set + BL->garr[0]);
    gs.log_scales = reinterpret_cast<float*>(set + BL->garr[1]);
    gs.quats = reinterpret_cast<float*>(set + BL->garr[2]);
    gs.opacity_logits = reinterpret_cast<float*>(set + BL->garr[3]);
    gs.sh = reinterpret_cast<float*>(set + BL->garr[4]);
    gs.feat = reinterpret_cast<float*>(set + BL->garr[5]);
    const GaussBwdArgs gb = gauss_bwd_args(L, ws, &gs, v >= S ? 1 : 0);
    FE_TRY_CUDA(launch_gauss_bwd(ga, gb, pool->s[v % S], nullptr));
  }
  if (pool) {
    FE_TRY_CUDA(join_streams(*pool, S, st));
    for (int k = 0; k < kGradArrays; ++k) {
      const float* src[kBatchStreams + 1];
      int n = 0;
      if (o0->accumulate_grads) src[n++] = dst[k];
      for (int i = 0; i < S; ++i) src[n++] = reinterpret_cast<const float*>(
          static_cast<const char*>(workspace) + BL->gset[i] + BL->garr[k]);
      FE_TRY_CUDA(launch_sum_f32(dst[k], src, n, BL->gn[k], st));
    }
  }
  FE_TRY_CUDA(mark(o0, 7, st));
  return FE_OK;
}

fe_status fe_batch_read_stats(const void* workspace, size_t workspace_bytes, int P, int D, const fe_batch* b,
                              fe_stats* stats, void* stream) {
  if (!workspace || !stats) return FE_ERR_INVALID_ARG;
  std::unique_ptr<BatchLayout> BL(new (std::nothrow) BatchLayout);
  if (!BL) return FE_ERR_WORKSPACE;
  fe_status s = batch_layout(P, D, b, *BL);
  if (s != FE_OK) return s;
  if (workspace_bytes < BL->total) return FE_ERR_WORKSPACE;
  fe_status first = FE_OK;
  for (int v = 0; v < b->V; ++v) {
    fe_opts o = b->opts[v];
    o.forward_only = b->opts[0].forward_only;
    const void* ws = static_cast<const char*>(workspace) + BL->off[v];
    s = fe_read_stats(ws, BL->L[v].total, P, D, b->cams[v].width, b->cams[v].height, &o, &stats[v], stream);
    if (s != FE_OK && first == FE_OK) first = s;
  }
  return first;
}

fe_status fe_probe_fp32_peak(int iters, double* flops, void* stream) {
  if (iters <= 0 || !flops) return FE_ERR_INVALID_ARG;
  return cuda_status(probe_fp32(iters, flops, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
