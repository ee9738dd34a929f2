// Full FST deformation module (Sec. 3.2, Eq. 4-6; Appendix A): the
// multi-resolution HexPlane encoding of (mu, t), the decoder MLP F_out
// (width 64, depth 8), the four branches (mu, R, S, o) with their feature
// extractors and heads, and the semantic updater F_feat giving dz; forward
// and reverse, including the gradients of the planes and of every weight.
//
// Forward: one thread per Gaussian for the MLP chain (activations in
// registers, weights from a 16-byte-aligned transposed copy, packed FP32
// FMA over output pairs); the HexPlane is sampled lane-cooperatively (the
// warp takes its 32 Gaussians one at a time, lane = channel, so each corner
// fetch is one coalesced 128-byte line of the channels-last planes).
//
// Reverse (persistent blocks of 128 Gaussians): each thread back-propagates
// its Gaussian through the layers (weights from an aligned row-major copy),
// and every layer's weight gradient sum_g delta_g x_g^T over the block's
// Gaussians is a block-level product from shared memory, added into the
// block's own partial (reduced over blocks in a fixed order afterwards:
// reproducible).  Plane gradients are scattered with coalesced float
// atomics (the only order-dependent sum of this file).
#include <cstdint>

#include "common.cuh"

namespace fe {

namespace {

constexpr int kFW = 64, kFHalf = 32, kFDepth = 8, kFC = 32, kFMaxL = 4;
constexpr int kFLayers = kFDepth + 12 + 2;
constexpr int kFThreads = 128;
constexpr int kFRow = 68;  // shared-memory row stride (floats) of the block products
constexpr int kLZ1 = kFDepth + 12, kLZ2 = kFDepth + 13;

__host__ __device__ constexpr int branch_e1(int g) { return kFDepth + 3 * g; }
// Offset sizes of the branches mu, R, S, o (Eq. 4).
__host__ __device__ constexpr int branch_out(int g) { return g == 1 ? 4 : (g == 3 ? 1 : 3); }
// Coordinate pairs of the planes xy, xz, yz, xt, yt, zt.
__host__ __device__ constexpr int pair_a(int k) { return k == 2 || k == 4 ? 1 : (k == 5 ? 2 : 0); }
__host__ __device__ constexpr int pair_b(int k) { return k == 0 ? 1 : (k == 1 || k == 2 ? 2 : 3); }

struct FstGeom {
  int levels, rs, rt, D, P;
  int nslots, sf, sz, se1, shg, sv;  // activation slots ([slot][P] float32)
  int nout[kFLayers], nin[kFLayers];
  int64_t pw[kFLayers], pb[kFLayers];  // offsets in the caller's packed array
  int64_t aw[kFLayers], ab[kFLayers];  // offsets in the aligned copies
  int64_t mlp_packed, mlp_aligned;
  int64_t poff[kFMaxL * 6];
  int pra[kFMaxL * 6], prb[kFMaxL * 6];
  float lo[3], scale[3];  // coordinate = (mu - lo) * scale - 1, scale = 2 / (hi - lo)
};

bool make_geom(const fe_fst* f, int P, FstGeom& g) {
  if (!f || f->levels < 1 || f->levels > kFMaxL || f->rs < 2 || f->rt < 2 || P < 0) return false;
  if (!(f->D == 16 || f->D == 32 || f->D == 64 || f->D == 128)) return false;
  if (((int64_t)f->rs << (f->levels - 1)) > (1 << 20) || f->rt > (1 << 20)) return false;
  g = FstGeom{};
  g.levels = f->levels;
  g.rs = f->rs;
  g.rt = f->rt;
  g.D = f->D;
  g.P = P;
  int l = 0;
  auto add = [&](int o, int i) { g.nout[l] = o; g.nin[l] = i; ++l; };
  add(kFW, f->levels * kFC);
  for (int j = 1; j < kFDepth; ++j) add(kFW, kFW);
  for (int b = 0; b < 4; ++b) {
    add(kFHalf, kFW);
    add(kFHalf, kFHalf);
    add(branch_out(b), kFHalf);
  }
  add(kFW, 4 * kFHalf);
  add(f->D, kFW);
  int64_t p = 0, a = 0;
  for (int k = 0; k < kFLayers; ++k) {
    const int64_t nw = (int64_t)g.nout[k] * g.nin[k];
    g.pw[k] = p;
    g.pb[k] = p + nw;
    p += nw + g.nout[k];
    g.aw[k] = a;
    a += (nw + 3) / 4 * 4;
    g.ab[k] = a;
    a += (g.nout[k] + 3) / 4 * 4;
  }
  g.mlp_packed = p;
  g.mlp_aligned = a;
  int64_t off = 0;
  for (int lv = 0; lv < f->levels; ++lv) {
    const int res[4] = {f->rs << lv, f->rs << lv, f->rs << lv, f->rt};
    for (int k = 0; k < 6; ++k) {
      g.poff[lv * 6 + k] = off;
      g.pra[lv * 6 + k] = res[pair_a(k)];
      g.prb[lv * 6 + k] = res[pair_b(k)];
      off += (int64_t)res[pair_a(k)] * res[pair_b(k)] * kFC;
    }
  }
  for (int k = 0; k < f->levels * 6; ++k)
    if ((int64_t)g.pra[k] * g.prb[k] * kFC > (int64_t)0x7FFFFFFF) return false;  // 32-bit plane indexing
  g.sf = 0;
  g.sz = f->levels * kFC;
  g.se1 = g.sz + kFDepth * kFW;
  g.shg = g.se1 + 4 * kFHalf;
  g.sv = g.shg + 4 * kFHalf;
  g.nslots = g.sv + kFW;
  for (int a3 = 0; a3 < 3; ++a3) {
    const float ext = f->bbox_max[a3] - f->bbox_min[a3];
    if (!(ext > 0.0f)) return false;
    g.lo[a3] = f->bbox_min[a3];
    g.scale[a3] = 2.0f / ext;
  }
  return true;
}

__host__ __device__ int64_t plane_floats(const FstGeom& g) {
  const int last = g.levels * 6 - 1;
  return g.poff[last] + (int64_t)g.pra[last] * g.prb[last] * kFC;
}

// Workspace: header | transposed weights (aligned) | row-major weights
// (aligned) | activations [nslots][P] | per-block partials of the weight
// gradients [nblk][mlp_aligned].
constexpr size_t kWsHeader = 256;
int bwd_blocks(int P) {
  const int chunks = (P + kFThreads - 1) / kFThreads;
  return chunks < 2 * 152 ? chunks : 2 * 152;
}
size_t al256(size_t x) { return (x + 255) / 256 * 256; }
// Row stride of the forward's per-thread shared-memory row: the level
// features, later relu(h).
__host__ __device__ constexpr int fwd_row(int levels) { return (levels * kFC > 2 * kFW ? levels * kFC : 2 * kFW) + 4; }
struct WsLayout {
  size_t wt, wn, act, dv, part, total;
};
WsLayout ws_layout(const FstGeom& g, int with_backward) {
  WsLayout w{};
  w.wt = kWsHeader;
  w.wn = w.wt + al256((size_t)g.mlp_aligned * 4);
  w.act = w.wn + al256((size_t)g.mlp_aligned * 4);
  w.dv = w.act + (with_backward ? al256((size_t)g.nslots * g.P * 4) : 0);
  w.part = w.dv + (with_backward ? al256((size_t)kFW * g.P * 4) : 0);
  w.total = w.part + (with_backward ? al256((size_t)bwd_blocks(g.P) * g.mlp_aligned * 4) : 0);
  return w;
}

// ---------------------------------------------------------------------------
// Weight copies: transposed [in][out] and row-major [out][in], each layer at
// a 16-byte-aligned offset (biases copied beside both).
// ---------------------------------------------------------------------------
__global__ void fst_pack_kernel(const FstGeom g, const float* __restrict__ mlp, float* __restrict__ wt,
                                float* __restrict__ wn) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.mlp_packed;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < kFLayers && e >= g.pw[k + 1]) ++k;
    const float v = mlp[e];
    if (e < g.pb[k]) {
      const int64_t r = e - g.pw[k];
      const int o = (int)(r / g.nin[k]), i = (int)(r % g.nin[k]);
      wt[g.aw[k] + (int64_t)i * g.nout[k] + o] = v;
      wn[g.aw[k] + r] = v;
    } else {
      wt[g.ab[k] + (e - g.pb[k])] = v;
      wn[g.ab[k] + (e - g.pb[k])] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Grid positions of one Gaussian: per level and axis, the cell index (bit 30
// set when the coordinate was clamped) and the fraction within the cell.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void grid_axes(const FstGeom& g, const float* mu, float t, int* ci, float* cf) {
  float c[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = (mu[a] - g.lo[a]) * g.scale[a] - 1.0f;
  c[3] = 2.0f * t - 1.0f;
  for (int lv = 0; lv < g.levels; ++lv) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int R = a < 3 ? (g.rs << lv) : g.rt;
      float x = (c[a] + 1.0f) * 0.5f * (float)(R - 1);
      int cl = 0;
      if (!(x >= 0.0f)) { x = 0.0f; cl = 1; }  // also catches NaN
      if (x > (float)(R - 1)) { x = (float)(R - 1); cl = 1; }
      int i = (int)floorf(x);
      if (i > R - 2) i = R - 2;
      ci[lv * 4 + a] = i | (cl << 30);
      cf[lv * 4 + a] = x - (float)i;
    }
  }
}

// ---------------------------------------------------------------------------
// Dense layer pieces: accumulators in registers, the layer input in the
// thread's own shared-memory row.  y (pairs) += W x, with W^T rows of `ld`
// floats (16-byte aligned) starting at wt.
// ---------------------------------------------------------------------------
template <int NIN, int NOUT>
__device__ __forceinline__ void dense_t(const float* __restrict__ wt, int ld, const float* x, float2* y,
                                        int nin = NIN) {
#pragma unroll 2
  for (int i = 0; i < nin; ++i) {
    const float2 xi = make_float2(x[i], x[i]);
    const float4* w4 = reinterpret_cast<const float4*>(wt + (size_t)i * ld);
#pragma unroll
    for (int q = 0; q < NOUT / 4; ++q) {
      const float4 w = __ldg(w4 + q);
      y[2 * q] = __ffma2_rn(make_float2(w.x, w.y), xi, y[2 * q]);
      y[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), xi, y[2 * q + 1]);
    }
  }
}

template <int N>
__device__ __forceinline__ void load_bias(const float* __restrict__ b, float2* y) {
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(b) + q);
    y[2 * q] = make_float2(v.x, v.y);
    y[2 * q + 1] = make_float2(v.z, v.w);
  }
}

template <int N>
__device__ __forceinline__ void put_relu(float* row, const float2* y) {
#pragma unroll
  for (int q = 0; q < N / 4; ++q)
    reinterpret_cast<float4*>(row)[q] = make_float4(fmaxf(y[2 * q].x, 0.0f), fmaxf(y[2 * q].y, 0.0f),
                                                    fmaxf(y[2 * q + 1].x, 0.0f), fmaxf(y[2 * q + 1].y, 0.0f));
}

template <int N>
__device__ __forceinline__ void relu_of(const float2* y, float* x) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    x[2 * q] = fmaxf(y[q].x, 0.0f);
    x[2 * q + 1] = fmaxf(y[q].y, 0.0f);
  }
}

// d x (pairs) += W^T delta with W row-major rows of `ld` floats at wn
// (rows 16-byte aligned), columns [0, NIN).
template <int NOUT, int NIN>
__device__ __forceinline__ void dense_back(const float* __restrict__ wn, int ld, const float* delta, float2* dx) {
#pragma unroll 2
  for (int o = 0; o < NOUT; ++o) {
    const float2 d = make_float2(delta[o], delta[o]);
    const float4* w4 = reinterpret_cast<const float4*>(wn + (size_t)o * ld);
#pragma unroll
    for (int q = 0; q < NIN / 4; ++q) {
      const float4 w = __ldg(w4 + q);
      dx[2 * q] = __ffma2_rn(make_float2(w.x, w.y), d, dx[2 * q]);
      dx[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), d, dx[2 * q + 1]);
    }
  }
}

template <int N>
__device__ __forceinline__ void zero2(float2* y) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) y[q] = make_float2(0.0f, 0.0f);
}

// Activation slot store / load ([slot][P], coalesced over the block).
template <int N>
__device__ __forceinline__ void store_slots(float* act, int P, int slot, int p, const float2* y) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    act[(size_t)(slot + 2 * q) * P + p] = y[q].x;
    act[(size_t)(slot + 2 * q + 1) * P + p] = y[q].y;
  }
}
template <int N>
__device__ __forceinline__ void load_slots(const float* act, int P, int slot, int p, bool valid, float* x) {
#pragma unroll
  for (int q = 0; q < N; ++q) x[q] = valid ? __ldg(act + (size_t)(slot + q) * P + p) : 0.0f;
}

struct FwdArgs {
  FstGeom g;
  const float *planes, *wt;
  const float *means, *quats, *log_scales, *logits;
  const void* feat;
  int feat_bf16;
  float t;
  float *means_t, *quats_t, *log_scales_t, *logits_t;
  void* feat_t;
  float* act;  // NULL: forward only
};

__device__ __forceinline__ float load_feat(const void* f, int bf16, size_t i) {
  if (bf16) {
    const uint16_t b = reinterpret_cast<const uint16_t*>(f)[i];
    return __uint_as_float((uint32_t)b << 16);
  }
  return reinterpret_cast<const float*>(f)[i];
}
__device__ __forceinline__ void store_feat(void* f, int bf16, size_t i, float v) {
  if (bf16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    reinterpret_cast<uint16_t*>(f)[i] = *reinterpret_cast<const uint16_t*>(&h);
  } else {
    reinterpret_cast<float*>(f)[i] = v;
  }
}

// Lane-cooperative HexPlane sample of level lv for the Gaussian whose grid
// axes are (ci, cf): returns channel `lane` of the level's feature.
__device__ __forceinline__ float level_feature(const FstGeom& g, const float* __restrict__ planes, int lv,
                                               const int* ci, const float* cf, int lane) {
  float f = 1.0f;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int a = pair_a(k), b = pair_b(k);
    const int ia = ci[lv * 4 + a] & 0x3FFFFFFF, ib = ci[lv * 4 + b] & 0x3FFFFFFF;
    const float fa = cf[lv * 4 + a], fb = cf[lv * 4 + b];
    const int rb = g.prb[lv * 6 + k];
    const float* base = planes + g.poff[lv * 6 + k] + ((size_t)ia * rb + ib) * kFC + lane;
    const float p00 = __ldg(base), p01 = __ldg(base + kFC);
    const float p10 = __ldg(base + (size_t)rb * kFC), p11 = __ldg(base + (size_t)rb * kFC + kFC);
    const float s = (1.0f - fa) * ((1.0f - fb) * p00 + fb * p01) + fa * ((1.0f - fb) * p10 + fb * p11);
    f *= s;
  }
  return f;
}

template <int D>
__global__ void __launch_bounds__(kFThreads, 2) fst_fwd_kernel(const FwdArgs a) {
  __shared__ int s_ci[kFThreads][kFMaxL * 4];
  __shared__ float s_cf[kFThreads][kFMaxL * 4];
  extern __shared__ __align__(16) float s_f[];  // [128][FS]: HexPlane features, then relu(h)
  const FstGeom& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = blockIdx.x * kFThreads + tid;
  const bool valid = p < g.P;
  const int FS = fwd_row(g.levels);
  float mu[3] = {0.0f, 0.0f, 0.0f};
  if (valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k) mu[k] = a.means[(size_t)p * 3 + k];
  }
  grid_axes(g, mu, a.t, s_ci[tid], s_cf[tid]);
  __syncwarp();
  // HexPlane features of the warp's Gaussians, lane = channel.
  const int gbase = blockIdx.x * kFThreads + warp * 32;
  for (int j = 0; j < 32 && gbase + j < g.P; ++j) {
    const int r = warp * 32 + j;
    for (int lv = 0; lv < g.levels; ++lv)
      s_f[r * FS + lv * kFC + lane] = level_feature(g, a.planes, lv, s_ci[r], s_cf[r], lane);
  }
  __syncwarp();
  if (!valid) return;  // no block-wide barrier follows
  float* frow = s_f + tid * FS;
  float* act = a.act;
  const int P = g.P;
  // F_out: z0 = W0 f + b0, then z_j = W_j relu(z_{j-1}) + b_j.
  float2 h[kFW / 2];
  load_bias<kFW>(a.wt + g.ab[0], h);
  if (act) {
    for (int c = 0; c < g.levels * kFC; ++c) act[(size_t)(g.sf + c) * P + p] = frow[c];
  }
  dense_t<kFMaxL * kFC, kFW>(a.wt + g.aw[0], kFW, frow, h, g.levels * kFC);
  if (act) store_slots<kFW>(act, P, g.sz, p, h);
  for (int j = 1; j < kFDepth; ++j) {
    put_relu<kFW>(frow, h);
    load_bias<kFW>(a.wt + g.ab[j], h);
    dense_t<kFW, kFW>(a.wt + g.aw[j], kFW, frow, h);
    if (act) store_slots<kFW>(act, P, g.sz + j * kFW, p, h);
  }
  // relu(h) stays in row[0, 64) while the branches run; row[64, 96) holds
  // relu(e1), row[96, 128) relu(h_g).
  put_relu<kFW>(frow, h);
  // Branches and the semantic updater's first layer (accumulated per branch).
  float2 v[kFW / 2];
  load_bias<kFW>(a.wt + g.ab[kLZ1], v);
  float out[11];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int l1 = branch_e1(b);
    {
      float2 e1[kFHalf / 2];
      load_bias<kFHalf>(a.wt + g.ab[l1], e1);
      dense_t<kFW, kFHalf>(a.wt + g.aw[l1], kFHalf, frow, e1);
      if (act) store_slots<kFHalf>(act, P, g.se1 + b * kFHalf, p, e1);
      put_relu<kFHalf>(frow + kFW, e1);
    }
    {
      float2 hg[kFHalf / 2];
      load_bias<kFHalf>(a.wt + g.ab[l1 + 1], hg);
      dense_t<kFHalf, kFHalf>(a.wt + g.aw[l1 + 1], kFHalf, frow + kFW, hg);
      if (act) store_slots<kFHalf>(act, P, g.shg + b * kFHalf, p, hg);
      put_relu<kFHalf>(frow + kFW + kFHalf, hg);
    }
    const float* hgr = frow + kFW + kFHalf;
    constexpr int dgs[4] = {3, 4, 3, 1}, oos[4] = {0, 3, 7, 10};
    const int dg = dgs[b], oo = oos[b];
    const float* wt_h = a.wt + g.aw[l1 + 2];  // [32][dg]
    const float* bh = a.wt + g.ab[l1 + 2];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      if (o < dg) {
        float s = __ldg(bh + o);
#pragma unroll
        for (int i = 0; i < kFHalf; ++i) s = fmaf(__ldg(wt_h + i * dg + o), hgr[i], s);
        out[oo + o] = s;
      }
    }
    dense_t<kFHalf, kFW>(a.wt + g.aw[kLZ1] + (size_t)b * kFHalf * kFW, kFW, hgr, v);
  }
  if (act) store_slots<kFW>(act, P, g.sv, p, v);
  put_relu<kFW>(frow, v);
  const float* vr = frow;
  // dz = Z2 relu(v) + b, in column chunks of at most 32.
  constexpr int ZC = D < 32 ? D : 32;
#pragma unroll
  for (int c0 = 0; c0 < D; c0 += ZC) {
    float2 z[ZC / 2];
    load_bias<ZC>(a.wt + g.ab[kLZ2] + c0, z);
    dense_t<kFW, ZC>(a.wt + g.aw[kLZ2] + c0, D, vr, z);
#pragma unroll
    for (int q = 0; q < ZC / 2; ++q) {
      const size_t i0 = (size_t)p * D + c0 + 2 * q;
      store_feat(a.feat_t, a.feat_bf16, i0, load_feat(a.feat, a.feat_bf16, i0) + z[q].x);
      store_feat(a.feat_t, a.feat_bf16, i0 + 1, load_feat(a.feat, a.feat_bf16, i0 + 1) + z[q].y);
    }
  }
  // Deformed Gaussian (Eq. 6): offsets added to the canonical parameters.
#pragma unroll
  for (int k = 0; k < 3; ++k) a.means_t[(size_t)p * 3 + k] = mu[k] + out[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) a.quats_t[(size_t)p * 4 + k] = a.quats[(size_t)p * 4 + k] + out[3 + k];
#pragma unroll
  for (int k = 0; k < 3; ++k) a.log_scales_t[(size_t)p * 3 + k] = a.log_scales[(size_t)p * 3 + k] + out[7 + k];
  a.logits_t[p] = a.logits[p] + out[10];
}

// ---------------------------------------------------------------------------
// Reverse.
// ---------------------------------------------------------------------------
struct BwdArgs {
  FstGeom g;
  const float *planes, *wn, *act;
  const float *means;
  float t;
  const float *d_means_t, *d_quats_t, *d_log_scales_t, *d_logits_t, *d_feat_t;
  float *d_means, *d_planes;
  float* dv;    // [64][P]: delta of F_feat's first layer
  float* part;  // [gridDim.x][mlp_aligned]
};

// pw[o * ldw + i] (+)= sum over the block's 128 Gaussians of
// s_d[g][o] * s_x[g][i], o < NO (<= 64), i < NI (multiple of 8, <= 64);
// pb[o] (+)= sum_g s_d[g][o] when pb is set.  Ends with a barrier.
__device__ void block_outer(const float* s_d, const float* s_x, int NO, int NI, float* pw, int ldw, float* pb,
                            bool first) {
  __syncthreads();
  const int nog = (NO + 3) / 4, ntile = nog * (NI / 8);
  for (int tile = threadIdx.x; tile < ntile; tile += kFThreads) {
    const int o0 = (tile % nog) * 4, i0 = (tile / nog) * 8;
    float2 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.0f, 0.0f);
#pragma unroll 4
    for (int gg = 0; gg < kFThreads; ++gg) {
      const float4 d = *reinterpret_cast<const float4*>(s_d + gg * kFRow + o0);
      const float4 x0 = *reinterpret_cast<const float4*>(s_x + gg * kFRow + i0);
      const float4 x1 = *reinterpret_cast<const float4*>(s_x + gg * kFRow + i0 + 4);
      const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 dd = make_float2(dv[r], dv[r]);
        acc[r][0] = __ffma2_rn(dd, make_float2(x0.x, x0.y), acc[r][0]);
        acc[r][1] = __ffma2_rn(dd, make_float2(x0.z, x0.w), acc[r][1]);
        acc[r][2] = __ffma2_rn(dd, make_float2(x1.x, x1.y), acc[r][2]);
        acc[r][3] = __ffma2_rn(dd, make_float2(x1.z, x1.w), acc[r][3]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (o0 + r < NO) {
        float* row = pw + (size_t)(o0 + r) * ldw + i0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float2 v = acc[r][c];
          if (!first) {
            v.x += row[2 * c];
            v.y += row[2 * c + 1];
          }
          row[2 * c] = v.x;
          row[2 * c + 1] = v.y;
        }
      }
    }
  }
  if (pb) {
    for (int o = threadIdx.x; o < NO; o += kFThreads) {
      float s = 0.0f;
      for (int gg = 0; gg < kFThreads; ++gg) s += s_d[gg * kFRow + o];
      pb[o] = first ? s : pb[o] + s;
    }
  }
  __syncthreads();
}

template <int N>
__device__ __forceinline__ void put_row(float* s, const float* x) {
#pragma unroll
  for (int q = 0; q < N / 4; ++q) reinterpret_cast<float4*>(s)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}
template <int N>
__device__ __forceinline__ void put_row_relu(float* s, const float* z) {
#pragma unroll
  for (int q = 0; q < N / 4; ++q)
    reinterpret_cast<float4*>(s)[q] = make_float4(fmaxf(z[4 * q], 0.f), fmaxf(z[4 * q + 1], 0.f),
                                                  fmaxf(z[4 * q + 2], 0.f), fmaxf(z[4 * q + 3], 0.f));
}
template <int N>
__device__ __forceinline__ void mask_pairs(const float2* dx, const float* z, float* delta) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    delta[2 * q] = z[2 * q] > 0.0f ? dx[q].x : 0.0f;
    delta[2 * q + 1] = z[2 * q + 1] > 0.0f ? dx[q].y : 0.0f;
  }
}

// delta[i] = dx[i] where the stored pre-activation z[i] > 0, else 0.
template <int N>
__device__ __forceinline__ void mask_slots(const float2* dx, const float* act, int P, int slot, int p, bool valid,
                                           float* delta) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    const float z0 = valid ? __ldg(act + (size_t)(slot + 2 * q) * P + p) : 0.0f;
    const float z1 = valid ? __ldg(act + (size_t)(slot + 2 * q + 1) * P + p) : 0.0f;
    delta[2 * q] = z0 > 0.0f ? dx[q].x : 0.0f;
    delta[2 * q + 1] = z1 > 0.0f ? dx[q].y : 0.0f;
  }
}
template <int N>
__device__ __forceinline__ void store_rows(float* dst, int P, int p, bool valid, const float* x) {
  if (!valid) return;
#pragma unroll
  for (int q = 0; q < N; ++q) dst[(size_t)q * P + p] = x[q];
}
// dx (pairs) += W^T delta with delta read from rows [NOUT][P] of src.
template <int NOUT, int NIN>
__device__ __forceinline__ void dense_back_rows(const float* __restrict__ wn, int ld, const float* src, int P, int p,
                                                bool valid, float2* dx) {
#pragma unroll 2
  for (int o = 0; o < NOUT; ++o) {
    const float dv = valid ? src[(size_t)o * P + p] : 0.0f;
    const float2 d = make_float2(dv, dv);
    const float4* w4 = reinterpret_cast<const float4*>(wn + (size_t)o * ld);
#pragma unroll
    for (int q = 0; q < NIN / 4; ++q) {
      const float4 w = __ldg(w4 + q);
      dx[2 * q] = __ffma2_rn(make_float2(w.x, w.y), d, dx[2 * q]);
      dx[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), d, dx[2 * q + 1]);
    }
  }
}

// Lane-cooperative reverse of one level's HexPlane sample for one Gaussian
// (lane = channel, dfc = d f of this channel): plane gradients by atomics,
// coordinate gradients summed over the warp into dc[0..2] (lane 0 adds).
__device__ __forceinline__ void plane_backward(const FstGeom& g, const float* __restrict__ planes, float* d_planes,
                                               int lv, const int* ci, const float* cf, float dfc, int lane,
                                               float* dc) {
  float smp[6], q00[6], q01[6], q10[6], q11[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int ia = ci[lv * 4 + pair_a(k)] & 0x3FFFFFFF, ib = ci[lv * 4 + pair_b(k)] & 0x3FFFFFFF;
    const float fa = cf[lv * 4 + pair_a(k)], fb = cf[lv * 4 + pair_b(k)];
    const int rb = g.prb[lv * 6 + k];
    const float* base = planes + g.poff[lv * 6 + k] + ((size_t)ia * rb + ib) * kFC + lane;
    q00[k] = __ldg(base);
    q01[k] = __ldg(base + kFC);
    q10[k] = __ldg(base + (size_t)rb * kFC);
    q11[k] = __ldg(base + (size_t)rb * kFC + kFC);
    smp[k] = (1.0f - fa) * ((1.0f - fb) * q00[k] + fb * q01[k]) + fa * ((1.0f - fb) * q10[k] + fb * q11[k]);
  }
  float dcl[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float others = 1.0f;
#pragma unroll
    for (int m = 0; m < 6; ++m)
      if (m != k) others *= smp[m];
    const float ds = dfc * others;
    const int A = pair_a(k), B = pair_b(k);
    const int ca = ci[lv * 4 + A], cb = ci[lv * 4 + B];
    const int ia = ca & 0x3FFFFFFF, ib = cb & 0x3FFFFFFF;
    const float fa = cf[lv * 4 + A], fb = cf[lv * 4 + B];
    const int rb = g.prb[lv * 6 + k];
    float* dbase = d_planes + g.poff[lv * 6 + k] + ((size_t)ia * rb + ib) * kFC + lane;
    atomicAdd(dbase, (1.0f - fa) * (1.0f - fb) * ds);
    atomicAdd(dbase + kFC, (1.0f - fa) * fb * ds);
    atomicAdd(dbase + (size_t)rb * kFC, fa * (1.0f - fb) * ds);
    atomicAdd(dbase + (size_t)rb * kFC + kFC, fa * fb * ds);
    if (!(ca >> 30))  // A is always a spatial axis
      dcl[A] += ds * ((1.0f - fb) * (q10[k] - q00[k]) + fb * (q11[k] - q01[k])) * 0.5f * (float)(g.pra[lv * 6 + k] - 1);
    if (B < 3 && !(cb >> 30))
      dcl[B < 3 ? B : 0] += ds * ((1.0f - fa) * (q01[k] - q00[k]) + fa * (q11[k] - q10[k])) * 0.5f * (float)(rb - 1);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = dcl[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    dcl[k] = s;
  }
  if (lane == 0) {
    dc[0] += dcl[0];
    dc[1] += dcl[1];
    dc[2] += dcl[2];
  }
}

template <int D>
__global__ void __launch_bounds__(kFThreads, 2) fst_bwd_kernel(const BwdArgs a) {
  extern __shared__ __align__(16) float s_dyn[];
  float* s_d = s_dyn;                       // [128][kFRow]: deltas of a layer
  float* s_x = s_dyn + kFThreads * kFRow;   // [128][kFRow]: inputs of a layer
  __shared__ int s_ci[kFThreads][kFMaxL * 4];
  __shared__ float s_cf[kFThreads][kFMaxL * 4];
  __shared__ float s_dc[kFThreads][4];
  const FstGeom& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = g.P;
  const int nchunk = (P + kFThreads - 1) / kFThreads;
  float* part = a.part + (size_t)blockIdx.x * g.mlp_aligned;
  float* sd = s_d + tid * kFRow;
  float* sx = s_x + tid * kFRow;
  const float* act = a.act;
  for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
    const bool first = chunk == (int)blockIdx.x;
    const int p = chunk * kFThreads + tid;
    const bool valid = p < P;
    const int pc = valid ? p : 0;
    // ---- F_feat, second layer: delta = d dz, input relu(v).
    {
      float v[kFW];
      load_slots<kFW>(act, P, g.sv, pc, valid, v);
      put_row_relu<kFW>(sx, v);
    }
    float2 dx[kFW / 2];
    zero2<kFW>(dx);
#pragma unroll
    for (int c0 = 0; c0 < D; c0 += 64) {
      constexpr int NC = D < 64 ? D : 64;
      {
        float dz[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) dz[q] = valid ? __ldg(a.d_feat_t + (size_t)p * D + c0 + q) : 0.0f;
        put_row<NC>(sd, dz);
        dense_back<NC, kFW>(a.wn + g.aw[kLZ2] + (size_t)c0 * kFW, kFW, sd, dx);
      }
      block_outer(s_d, s_x, NC, kFW, part + g.aw[kLZ2] + (size_t)c0 * kFW, kFW, part + g.ab[kLZ2] + c0, first);
    }
    // delta of F_feat's first layer; kept in the workspace for the branches.
    {
      float dv[kFW];
      mask_slots<kFW>(dx, act, P, g.sv, pc, valid, dv);
      put_row<kFW>(sd, dv);
      store_rows<kFW>(a.dv, P, pc, valid, dv);
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      {
        float u[kFW];
        load_slots<kFW>(act, P, g.shg + half * kFW, pc, valid, u);
        put_row_relu<kFW>(sx, u);
      }
      block_outer(s_d, s_x, kFW, kFW, part + g.aw[kLZ1] + half * kFW, 4 * kFHalf, half ? nullptr : part + g.ab[kLZ1],
                  first);
    }
    // ---- Branches.
    float2 drh[kFW / 2];
    zero2<kFW>(drh);
    const float* dsrc[4] = {a.d_means_t, a.d_quats_t, a.d_log_scales_t, a.d_logits_t};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      constexpr int dgs[4] = {3, 4, 3, 1};
      const int dg = dgs[b], l1 = branch_e1(b);
      float dhg[kFHalf];
      {
        float hg[kFHalf];
        load_slots<kFHalf>(act, P, g.shg + b * kFHalf, pc, valid, hg);
        float dh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 4; ++o)
          if (o < dg && valid) dh[o] = __ldg(dsrc[b] + (size_t)p * dg + o);
        // head: delta = d offset, input relu(h_g).
        put_row<4>(sd, dh);
        put_row_relu<kFHalf>(sx, hg);
        // d relu(h_g): from the head and from F_feat's first layer.
        float2 d2[kFHalf / 2];
        zero2<kFHalf>(d2);
        const float* wh = a.wn + g.aw[l1 + 2];  // [dg][32]
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          if (o < dg) {
            const float2 d = make_float2(dh[o], dh[o]);
#pragma unroll
            for (int q = 0; q < kFHalf / 4; ++q) {
              const float4 w = __ldg(reinterpret_cast<const float4*>(wh + o * kFHalf) + q);
              d2[2 * q] = __ffma2_rn(make_float2(w.x, w.y), d, d2[2 * q]);
              d2[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), d, d2[2 * q + 1]);
            }
          }
        }
        dense_back_rows<kFW, kFHalf>(a.wn + g.aw[kLZ1] + b * kFHalf, 4 * kFHalf, a.dv, P, pc, valid, d2);
        mask_pairs<kFHalf>(d2, hg, dhg);
      }
      block_outer(s_d, s_x, dg, kFHalf, part + g.aw[l1 + 2], kFHalf, part + g.ab[l1 + 2], first);
      // E2: input relu(e1).
      float de1[kFHalf];
      {
        float e1[kFHalf];
        load_slots<kFHalf>(act, P, g.se1 + b * kFHalf, pc, valid, e1);
        put_row<kFHalf>(sd, dhg);
        put_row_relu<kFHalf>(sx, e1);
        float2 de[kFHalf / 2];
        zero2<kFHalf>(de);
        dense_back<kFHalf, kFHalf>(a.wn + g.aw[l1 + 1], kFHalf, sd, de);
        mask_pairs<kFHalf>(de, e1, de1);
      }
      block_outer(s_d, s_x, kFHalf, kFHalf, part + g.aw[l1 + 1], kFHalf, part + g.ab[l1 + 1], first);
      // E1: input relu(h).
      {
        float h7[kFW];
        load_slots<kFW>(act, P, g.sz + (kFDepth - 1) * kFW, pc, valid, h7);
        put_row_relu<kFW>(sx, h7);
      }
      put_row<kFHalf>(sd, de1);
      dense_back<kFHalf, kFW>(a.wn + g.aw[l1], kFW, sd, drh);
      block_outer(s_d, s_x, kFHalf, kFW, part + g.aw[l1], kFW, part + g.ab[l1], first);
    }
    // ---- F_out, last layer first.
    float delta[kFW];
    mask_slots<kFW>(drh, act, P, g.sz + (kFDepth - 1) * kFW, pc, valid, delta);
    for (int j = kFDepth - 1; j >= 1; --j) {
      {
        float zp[kFW];
        load_slots<kFW>(act, P, g.sz + (j - 1) * kFW, pc, valid, zp);
        put_row_relu<kFW>(sx, zp);
      }
      put_row<kFW>(sd, delta);
      float2 d3[kFW / 2];
      zero2<kFW>(d3);
      dense_back<kFW, kFW>(a.wn + g.aw[j], kFW, sd, d3);
      block_outer(s_d, s_x, kFW, kFW, part + g.aw[j], kFW, part + g.ab[j], first);
      mask_slots<kFW>(d3, act, P, g.sz + (j - 1) * kFW, pc, valid, delta);
    }
    // First layer: input f.
    const int nf = g.levels * kFC;
    put_row<kFW>(sd, delta);
    for (int c0 = 0; c0 < nf; c0 += kFW) {
      const int nc = nf - c0 < kFW ? nf - c0 : kFW;
      {
        float f[kFW];
        load_slots<kFW>(act, P, g.sf + c0, pc, valid, f);
        if (nc < kFW) {
#pragma unroll
          for (int q = kFC; q < kFW; ++q) f[q] = 0.0f;
        }
        put_row<kFW>(sx, f);
      }
      block_outer(s_d, s_x, kFW, nc, part + g.aw[0] + c0, nf, c0 ? nullptr : part + g.ab[0], first);
    }
    // ---- HexPlane: d f per level, lane-cooperative over the warp's Gaussians.
    float mu[3] = {0.f, 0.f, 0.f};
    if (valid) {
#pragma unroll
      for (int k = 0; k < 3; ++k) mu[k] = a.means[(size_t)p * 3 + k];
    }
    grid_axes(g, mu, a.t, s_ci[tid], s_cf[tid]);
    s_dc[tid][0] = s_dc[tid][1] = s_dc[tid][2] = 0.0f;
    const int gbase = chunk * kFThreads + warp * 32;
    for (int lv = 0; lv < g.levels; ++lv) {
      float2 dfl[kFC / 2];
      zero2<kFC>(dfl);
      dense_back<kFW, kFC>(a.wn + g.aw[0] + lv * kFC, nf, sd, dfl);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kFC / 2; ++q) {
        sx[2 * q] = dfl[q].x;
        sx[2 * q + 1] = dfl[q].y;
      }
      __syncwarp();
      for (int j = 0; j < 32 && gbase + j < P; ++j) {
        const int r = warp * 32 + j;
        plane_backward(g, a.planes, a.d_planes, lv, s_ci[r], s_cf[r], s_x[r * kFRow + lane], lane, s_dc[r]);
      }
    }
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        a.d_means[(size_t)p * 3 + k] = a.d_means_t[(size_t)p * 3 + k] + s_dc[tid][k] * g.scale[k];
    }
    __syncthreads();  // s_x rows are rewritten by the next chunk's products
  }
}


// d_mlp (caller's packed layout) = sum over blocks, in block order, of the
// partials (aligned layout).
__global__ void fst_reduce_kernel(const FstGeom g, const float* __restrict__ part, int nblk, float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.mlp_packed;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < kFLayers && e >= g.pw[k + 1]) ++k;
    const int64_t src = e < g.pb[k] ? g.aw[k] + (e - g.pw[k]) : g.ab[k] + (e - g.pb[k]);
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * g.mlp_aligned + src];
    out[e] = s;
  }
}

// ---------------------------------------------------------------------------
// Total variation of the planes (L_TV of Eq. 11).
// ---------------------------------------------------------------------------
struct TvArgs {
  FstGeom g;
  const float* planes;
  float* d_planes;
  float weight;
  float* partial;  // [planes][kTvBlocks]
};

constexpr int kTvBlocks = 40;  // blocks per plane (grid.y = plane)

// One plane per grid row; each thread takes four channels of a node (the
// planes are channels-last, so a float4 per neighbour).  The loss partials
// are summed in a fixed order afterwards.
__global__ void __launch_bounds__(256) fst_tv_kernel(const TvArgs a) {
  __shared__ float s_w[8];
  const FstGeom& g = a.g;
  const int k = blockIdx.y;
  const int ra = g.pra[k], rb = g.prb[k];
  const float4* pl = reinterpret_cast<const float4*>(a.planes + g.poff[k]);
  float4* dp = reinterpret_cast<float4*>(a.d_planes + g.poff[k]);
  const int q4 = kFC / 4;
  const int total = ra * rb * q4;
  const float ia = 1.0f / (float)((int64_t)(ra - 1) * rb * kFC), ib = 1.0f / (float)((int64_t)ra * (rb - 1) * kFC);
  float acc = 0.0f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int node = e / q4;
    const int i = node / rb, j = node - i * rb;
    const float4 v = pl[e];
    float4 gr = make_float4(0.f, 0.f, 0.f, 0.f);
    auto term = [&](const float4 n, float w, bool forward) {
      // forward: n is the next node (difference n - v, counted in the loss)
      const float4 d = forward ? make_float4(n.x - v.x, n.y - v.y, n.z - v.z, n.w - v.w)
                               : make_float4(v.x - n.x, v.y - n.y, v.z - n.z, v.w - n.w);
      if (forward) acc += (d.x * d.x + d.y * d.y + d.z * d.z + d.w * d.w) * w;
      const float s = forward ? -2.0f * w : 2.0f * w;
      gr.x += s * d.x; gr.y += s * d.y; gr.z += s * d.z; gr.w += s * d.w;
    };
    if (i + 1 < ra) term(pl[e + rb * q4], ia, true);
    if (i > 0) term(pl[e - rb * q4], ia, false);
    if (j + 1 < rb) term(pl[e + q4], ib, true);
    if (j > 0) term(pl[e - q4], ib, false);
    float4 o = dp[e];
    o.x += a.weight * gr.x; o.y += a.weight * gr.y; o.z += a.weight * gr.z; o.w += a.weight * gr.w;
    dp[e] = o;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    a.partial[k * kTvBlocks + blockIdx.x] = t;
  }
}

__global__ void fst_tv_finish(const float* __restrict__ partial, int n, float weight, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.0f;
    for (int b = 0; b < n; ++b) s += partial[b];
    *loss = weight * s;
  }
}

bool al16p(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

}  // namespace fe

using namespace fe;

extern "C" int64_t fe_fst_plane_floats(int levels, int rs, int rt) {
  fe_fst f{};
  f.levels = levels;
  f.rs = rs;
  f.rt = rt;
  f.D = 32;
  for (int a = 0; a < 3; ++a) f.bbox_max[a] = 1.0f;
  FstGeom g;
  return make_geom(&f, 0, g) ? plane_floats(g) : 0;
}

extern "C" int64_t fe_fst_mlp_floats(int levels, int D) {
  fe_fst f{};
  f.levels = levels;
  f.rs = 2;
  f.rt = 2;
  f.D = D;
  for (int a = 0; a < 3; ++a) f.bbox_max[a] = 1.0f;
  FstGeom g;
  return make_geom(&f, 0, g) ? g.mlp_packed : 0;
}

extern "C" fe_status fe_fst_workspace_size(int P, int levels, int D, int with_backward, size_t* bytes) {
  if (!bytes) return FE_ERR_INVALID_ARG;
  fe_fst f{};
  f.levels = levels;
  f.rs = 2;
  f.rt = 2;
  f.D = D;
  for (int a = 0; a < 3; ++a) f.bbox_max[a] = 1.0f;
  FstGeom g;
  if (!make_geom(&f, P, g)) return (D == 16 || D == 32 || D == 64 || D == 128) ? FE_ERR_INVALID_ARG : FE_ERR_UNSUPPORTED;
  *bytes = ws_layout(g, with_backward ? 1 : 0).total;
  return FE_OK;
}

namespace {

template <int D>
cudaError_t launch_fst_fwd(const FwdArgs& a, cudaStream_t st) {
  const int blocks = (a.g.P + kFThreads - 1) / kFThreads;
  const size_t smem = (size_t)kFThreads * fwd_row(a.g.levels) * 4;
  auto k = fst_fwd_kernel<D>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<blocks, kFThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_fst_bwd(const BwdArgs& a, int nblk, cudaStream_t st) {
  const size_t smem = (size_t)2 * kFThreads * kFRow * 4;
  auto k = fst_bwd_kernel<D>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<nblk, kFThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

extern "C" fe_status fe_fst_forward(const fe_fst* fst, int P, const float* means, const float* quats,
                                    const float* log_scales, const float* opacity_logits, const void* feat,
                                    int feat_bf16, float t, float* means_t, float* quats_t, float* log_scales_t,
                                    float* opacity_logits_t, void* feat_t, void* workspace, size_t workspace_bytes,
                                    int with_backward, void* stream) {
  FstGeom g;
  if (!fst || !make_geom(fst, P, g)) {
    if (fst && !(fst->D == 16 || fst->D == 32 || fst->D == 64 || fst->D == 128)) return FE_ERR_UNSUPPORTED;
    return FE_ERR_INVALID_ARG;
  }
  if (!workspace || !al16p(workspace)) return FE_ERR_INVALID_ARG;
  const WsLayout w = ws_layout(g, with_backward ? 1 : 0);
  if (workspace_bytes < w.total) return FE_ERR_WORKSPACE;
  if (P == 0) return FE_OK;
  if (!fst->planes || !fst->mlp || !means || !quats || !log_scales || !opacity_logits || !feat || !means_t ||
      !quats_t || !log_scales_t || !opacity_logits_t || !feat_t || !al16p(fst->planes) || !al16p(fst->mlp))
    return FE_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  float* wt = reinterpret_cast<float*>(ws + w.wt);
  float* wn = reinterpret_cast<float*>(ws + w.wn);
  if (cudaMemsetAsync(wt, 0, w.act - w.wt, st) != cudaSuccess) return FE_ERR_CUDA;
  fst_pack_kernel<<<(int)((g.mlp_packed + 255) / 256), 256, 0, st>>>(g, fst->mlp, wt, wn);
  FwdArgs a{};
  a.g = g;
  a.planes = fst->planes;
  a.wt = wt;
  a.means = means;
  a.quats = quats;
  a.log_scales = log_scales;
  a.logits = opacity_logits;
  a.feat = feat;
  a.feat_bf16 = feat_bf16 ? 1 : 0;
  a.t = t;
  a.means_t = means_t;
  a.quats_t = quats_t;
  a.log_scales_t = log_scales_t;
  a.logits_t = opacity_logits_t;
  a.feat_t = feat_t;
  a.act = with_backward ? reinterpret_cast<float*>(ws + w.act) : nullptr;
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.D) {
    case 16: e = launch_fst_fwd<16>(a, st); break;
    case 32: e = launch_fst_fwd<32>(a, st); break;
    case 64: e = launch_fst_fwd<64>(a, st); break;
    case 128: e = launch_fst_fwd<128>(a, st); break;
  }
  return e == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" fe_status fe_fst_backward(const fe_fst* fst, int P, const float* means, float t, const float* d_means_t,
                                     const float* d_quats_t, const float* d_log_scales_t,
                                     const float* d_opacity_logits_t, const float* d_feat_t, float* d_means,
                                     float* d_planes, float* d_mlp, void* workspace, size_t workspace_bytes,
                                     void* stream) {
  FstGeom g;
  if (!fst || !make_geom(fst, P, g)) {
    if (fst && !(fst->D == 16 || fst->D == 32 || fst->D == 64 || fst->D == 128)) return FE_ERR_UNSUPPORTED;
    return FE_ERR_INVALID_ARG;
  }
  if (!workspace || !al16p(workspace) || !d_planes || !d_mlp) return FE_ERR_INVALID_ARG;
  const WsLayout w = ws_layout(g, 1);
  if (workspace_bytes < w.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_planes, 0, (size_t)plane_floats(g) * 4, st) != cudaSuccess) return FE_ERR_CUDA;
  if (P == 0) return cudaMemsetAsync(d_mlp, 0, (size_t)g.mlp_packed * 4, st) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
  if (!fst->planes || !means || !d_means_t || !d_quats_t || !d_log_scales_t || !d_opacity_logits_t || !d_feat_t ||
      !d_means)
    return FE_ERR_INVALID_ARG;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  BwdArgs a{};
  a.g = g;
  a.planes = fst->planes;
  a.wn = reinterpret_cast<const float*>(ws + w.wn);
  a.act = reinterpret_cast<const float*>(ws + w.act);
  a.means = means;
  a.t = t;
  a.d_means_t = d_means_t;
  a.d_quats_t = d_quats_t;
  a.d_log_scales_t = d_log_scales_t;
  a.d_logits_t = d_opacity_logits_t;
  a.d_feat_t = d_feat_t;
  a.d_means = d_means;
  a.d_planes = d_planes;
  a.dv = reinterpret_cast<float*>(ws + w.dv);
  a.part = reinterpret_cast<float*>(ws + w.part);
  const int nblk = bwd_blocks(P);
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.D) {
    case 16: e = launch_fst_bwd<16>(a, nblk, st); break;
    case 32: e = launch_fst_bwd<32>(a, nblk, st); break;
    case 64: e = launch_fst_bwd<64>(a, nblk, st); break;
    case 128: e = launch_fst_bwd<128>(a, nblk, st); break;
  }
  if (e != cudaSuccess) return FE_ERR_CUDA;
  fst_reduce_kernel<<<(int)((g.mlp_packed + 255) / 256), 256, 0, st>>>(g, a.part, nblk, d_mlp);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" fe_status fe_fst_tv(const fe_fst* fst, float weight, float* loss, float* d_planes, float* scratch,
                               void* stream) {
  FstGeom g;
  if (!fst || !make_geom(fst, 0, g)) return FE_ERR_INVALID_ARG;
  if (!fst->planes || !loss || !d_planes || !scratch) return FE_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TvArgs a{};
  a.g = g;
  a.planes = fst->planes;
  a.d_planes = d_planes;
  a.weight = weight;
  a.partial = scratch;
  const int np = g.levels * 6;  // at most 24 planes x kTvBlocks partials <= 1024 scratch floats
  fst_tv_kernel<<<dim3(kTvBlocks, np), 256, 0, st>>>(a);
  fst_tv_finish<<<1, 32, 0, st>>>(scratch, np * kTvBlocks, weight, loss);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
