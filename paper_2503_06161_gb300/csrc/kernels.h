// Internal launcher interface between the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fe {

constexpr int kDStride = 16;  // floats per Gaussian of reverse-pass state: offsets[11], pad, unit masks[4]

struct GaussArgs {
  int P, sh_degree, sh_bf16;
  const float *means, *log_scales, *quats, *logits;
  const void* sh;
  // deformation
  int has_deform, C, R;
  const float *planes, *w1, *b1, *w2, *b2, *wh, *bh;
  float bmin[3], bscale[3];  // coordinate = (mu - bmin) * bscale - 1
  const float* noise;
  float noise_scale, t;
  // camera
  int W, H, tw, th;
  float fx, fy, cx, cy, znear, limx, limy;
  float V[12];
  float campos[3];
  // [P][kDStride] deformation offsets and MLP unit masks (written by the
  // MLP kernel, read by the projection and the reverse pass)
  float* dstate;
  // three [P][C] BF16 arrays: the HexPlane features split hi + mid + lo
  uint16_t* fsplit;
  // outputs
  float4* rec;
  ushort4* rect;
  uint32_t *touched, *dkey;
  uint32_t *err, *num_visible;
};

struct GaussBwdArgs {
  int D;
  int64_t cap;
  const uint32_t *touched, *offs_by_gid;
  const uint32_t* order;  // [P] Gaussian ids in depth order (the emission order of their entries)
  const uint32_t* offs;   // [P + 1] first emission index of each depth rank
  const float* partials;
  const uint32_t* pflags;  // bit e set: partial row e was written
  float *d_means, *d_log_scales, *d_quats, *d_logits, *d_sh, *d_feat;
  float* ddstate;  // [P][12] dL/d delta, [11] = active flag
  float* psum;     // [P][12] sums of the partial rows' scalars
  int accumulate;  // 1: add to the gradient buffers
};

cudaError_t launch_gauss_fwd(const GaussArgs& a, cudaStream_t st);
// Deformation MLP on the tensor cores: a.fsplit -> a.dstate (deform_mlp.cu).
cudaError_t launch_deform_mlp(const GaussArgs& a, cudaStream_t st);
cudaError_t launch_gauss_bwd(const GaussArgs& a, const GaussBwdArgs& b, cudaStream_t st, cudaEvent_t mid);
// Reverse of the deformation MLP on the tensor cores: b.ddstate -> df [P][C]
// (deform_mlp.cu).
cudaError_t launch_deform_mlp_bwd(const GaussArgs& a, const GaussBwdArgs& b, float* df, cudaStream_t st);

// Integer stage: binning of projected Gaussians into tile lists.
struct BinArgs {
  int P, ntiles, tiles_x, pblocks, bblocks;
  int64_t cap;
  const ushort4* rect;
  const uint32_t* touched;
  uint32_t *dkey[2], *dval[2];  // depth-sort ping-pong (final: index 0)
  uint32_t *offs, *offs_by_gid;
  uint2* sorted;                 // [cap] (emission index, Gaussian) per list position
  uint32_t* table;              // [ntiles][bblocks] counts, then segment starts
  uint32_t* status;             // decoupled look-back words
  uint32_t* hist;               // depth digit histograms [4][256]
  uint2* ranges;
  void* hdr;                    // fe::Header*
};

// Rect / touched / depth key from given (u, v, r, depth) (fe_tile_bin).
cudaError_t launch_bin_prep(int P, const float* uv, const int* radius, const float* depth, int W, int H, int tw,
                            int th, ushort4* rect, uint32_t* touched, uint32_t* dkey, uint32_t* num_visible,
                            cudaStream_t st);
cudaError_t launch_binning(BinArgs& b, cudaStream_t st);

struct CompositeArgs {
  int W, H, tw, th, tiles_x, D, feat_bf16;
  float bg[3];
  const uint2* ranges;
  const uint2* sorted;  // (emission index, Gaussian) per list position
  const float4* rec;
  const void* feat;
  float *out_rgb, *out_depth, *out_alpha, *out_feat;
  uint16_t* out_feat_bf16;  // optional bf16 copy of out_feat
  float* t_final;
  uint32_t* n_contrib;
  // backward
  const float *g_rgb, *g_depth, *g_alpha, *g_feat;
  float* partials;
  uint32_t* pflags;
  int ntiles;
  int64_t cap;       // list capacity: emission indices at or past it are skipped
  uint64_t* counts;  // non-NULL: counting variant of the forward (no outputs)
  uint32_t* err;     // header error bits (staging timeouts)
  uint32_t* cmask;   // NULL, or per (tile, 32-entry group, warp) masks of blended entries
  int polls;         // bound of each staging wait (polls); 0: give up at once
  // Channel split (D = 256 runs as two passes over 128-channel halves; a
  // single pass has feat_row_bytes = D x element size, out_ld = D,
  // prow = D + 12, pcol0 = 0, pscal = D, aux = 1):
  uint32_t feat_row_bytes;  // bytes between consecutive Gaussians' rows of `feat` (pointer at this pass's channels)
  int out_ld;               // floats between pixels of out_feat / out_feat_bf16 / g_feat (pointers at this pass's channels)
  int prow, pcol0, pscal;   // partial row stride (floats), column of this pass's first channel, of the scalars
  int aux;                  // 1: this pass writes colour, depth, alpha, T_final, n_contrib, the blend masks and
                            // (reverse) the scalar columns; 0: (reverse) adds its geometric terms to them
};

// Forward compositing; fwd_batch = Gaussians per staged batch (32, 64 or
// 128; 0 = the default for D).
cudaError_t launch_composite_fwd(const CompositeArgs& a, int fwd_batch, cudaStream_t st);
cudaError_t launch_composite_bwd(const CompositeArgs& a, cudaStream_t st);

// Views of one batched launch (kernel parameter space holds them all).
constexpr int kMaxViews = 32;

// A batch of views composited by one persistent launch: (view, tile) work
// items numbered view after view (view v owns items [item_start[v],
// item_start[v+1])), taken by the blocks from the device counter `queue`
// (zeroed before the launch).
struct BatchCompositeArgs {
  int V, nitems;
  int item_start[kMaxViews + 1];
  CompositeArgs view[kMaxViews];
  uint32_t* queue;
};

cudaError_t launch_composite_fwd_batch(const BatchCompositeArgs& b, int D, int feat_bf16, int fwd_batch,
                                       cudaStream_t st);
cudaError_t launch_composite_bwd_batch(const BatchCompositeArgs& b, int D, int feat_bf16, cudaStream_t st);
bool fwd_batch_supported(int fwd_batch);

struct DumpArgs {
  int64_t cap;
  int P, ntiles, HW;
  const void* hdr;
  const uint2* sorted;  // (emission index, Gaussian) per list position
  const uint2* ranges;
  const uint32_t* ncontrib;
  const float* tfinal;
  const float4* rec;
  const uint32_t* touched;
  uint64_t* keys;
  uint32_t *gauss, *ranges_out, *ncontrib_out, *touched_out;
  float *tfinal_out, *uv, *conic, *opacity, *depth, *rgb;
  int32_t* radius;
};
cudaError_t launch_dump(const DumpArgs& d, cudaStream_t st);

// Screen-space gradient statistics of adaptive density control (density.cu).
cudaError_t launch_screen_stats(const float4* rec, const float* psum, int P, int W, int H, float* accum,
                                int32_t* count, cudaStream_t st);

cudaError_t probe_fp32(int iters, double* flops, cudaStream_t st);
// dst = ((srcs[0] + srcs[1]) + ...) elementwise (1..8 sources, any alignment;
// dst may alias srcs[0]).
cudaError_t launch_sum_f32(float* dst, const float* const* srcs, int nsrc, int64_t n, cudaStream_t st);
cudaError_t launch_l1(const float* pred, const float* target, int64_t n, int64_t rows, float* grad, float* loss,
                      float* scratch, cudaStream_t st);
void l1_grad_launch(const float* pred, const float* target, int64_t n, float inv_rows, float* grad, float* partial,
                    int blocks, cudaStream_t st);
void l1_finish_launch(const float* partial, int nparts, float inv_rows, float* loss, cudaStream_t st);

}  // namespace fe
