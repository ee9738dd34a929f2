// Full FST deformation module (Sec. 3.2, Eq. 4-6; Appendix A): the
// multi-resolution HexPlane encoding of (mu, t), the decoder MLP F_out
// (width 64, depth 8), the four branches (mu, R, S, o) with their feature
// extractors and heads, and the semantic updater F_feat giving dz; forward
// and reverse, including the gradients of the planes and of every weight.
//
// Kernels, in launch order:
//   fst_pack_kernel     16-byte-aligned transposed and row-major copies of
//                       the weights in the workspace;
//   fst_sample_kernel   HexPlane features f, lane-cooperative (the warp takes
//                       its Gaussians four at a time, lane = channel, so each
//                       corner fetch is one coalesced 128-byte line of the
//                       channels-last planes), written Gaussian-major;
//   fst_fwd_kernel      the MLP: a block holds 128 Gaussians and every layer
//                       is a block product -- activations in shared memory
//                       (a row per Gaussian), each thread a register tile of
//                       packed FP32 FMAs, weight tiles staged by cp.async --
//                       writing the deformed Gaussians and relu(z) of every
//                       hidden layer for the reverse;
//   fst_bwd_kernel      (persistent blocks) per layer the input gradient
//                       delta W as the same tile product, the ReLU masks from
//                       the stored relu(z), and the weight gradient
//                       sum_g delta_g x_g^T as a second block product added
//                       into the block's own partial; writes d f;
//   fst_hex_bwd_kernel  the HexPlane reverse: plane gradients by coalesced
//                       float atomics (the only order-dependent sum of this
//                       file), the canonical mean's gradient;
//   fst_reduce_kernel   the weight gradients: the blocks' partials summed in
//                       block order (reproducible bit for bit);
//   fst_tv_kernel       the TV term and its plane gradient.
#include <cstdint>

#include "common.cuh"

namespace fe {

namespace {

constexpr int kFW = 64, kFHalf = 32, kFDepth = 8, kFC = 32, kFMaxL = 4;
constexpr int kFLayers = kFDepth + 12 + 2;
constexpr int kFThreads = 128;     // threads of the reverse product kernel
constexpr int kFM = 128;           // Gaussians per block of the product kernels
constexpr int kFwdThreads = 256;   // threads of the forward product kernel
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
// (aligned) | f [P][levels*32] | with the reverse: relu activations
// [nslots][P], F_feat delta [64][P], d f [P][levels*32], per-block partials
// of the weight gradients [nblk][mlp_aligned].
constexpr size_t kWsHeader = 256;
int bwd_blocks(int P) {
  const int chunks = (P + kFThreads - 1) / kFThreads;
  return chunks < 2 * 152 ? chunks : 2 * 152;
}
size_t al256(size_t x) { return (x + 255) / 256 * 256; }
// acc: with the reverse pass, the exact plane-gradient accumulators, two
// uint64 arrays (hi, lo) of one entry per plane float (see fixed_add).
struct WsLayout {
  size_t wt, wn, f, act, dv, df, part, acc, total;
};
WsLayout ws_layout(const FstGeom& g, int with_backward) {
  WsLayout w{};
  w.wt = kWsHeader;
  w.wn = w.wt + al256((size_t)g.mlp_aligned * 4);
  w.f = w.wn + al256((size_t)g.mlp_aligned * 4);
  w.act = w.f + al256((size_t)g.levels * kFC * g.P * 4);
  w.dv = w.act + (with_backward ? al256((size_t)g.nslots * g.P * 4) : 0);
  w.df = w.dv + (with_backward ? al256((size_t)kFW * g.P * 4) : 0);
  w.part = w.df + (with_backward ? al256((size_t)g.levels * kFC * g.P * 4) : 0);
  w.acc = w.part + (with_backward ? al256((size_t)bwd_blocks(g.P) * g.mlp_aligned * 4) : 0);
  w.total = w.acc + (with_backward == 2 ? al256((size_t)plane_floats(g) * 16) : 0);
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
// Block products.  A block holds 128 Gaussians; activations live in shared
// memory row-major per Gaussian ([128][kFRow] floats).  Thread (mt, nt)
// owns rows mt + (128 / TM) r (r < TM) and TN consecutive output columns
// from n0 = nt * TN (TM = 8 with 128 threads: mt = tid % 16, nt = tid / 16;
// TM = 4 with 256 threads: mt = tid % 32, nt = tid / 32): per step of four
// inputs it reads TM 16-byte row slices from shared memory and TN weights
// per input, then issues 2 TM TN packed FMAs.
// ---------------------------------------------------------------------------
template <int TN, int TM = 8>
__device__ __forceinline__ void tile_zero(float2 (&acc)[TM][TN / 2]) {
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN / 2; ++c) acc[r][c] = make_float2(0.0f, 0.0f);
}

// acc[r][c] += sum_k X[(mt + RG r) * kFRow + k] * B[k * ldb + n0 + (2c, 2c+1)],
// RG = 128 / TM, k < K (multiple of 8); B rows 8-byte aligned at n0.
template <int TN, bool kSharedB = false, int TM = 8>
__device__ __forceinline__ void tile_mma(const float* X, int K, const float* __restrict__ B, int ldb, int mt, int n0,
                                         float2 (&acc)[TM][TN / 2]) {
  constexpr int RG = kFM / TM;  // row groups: thread rows are mt + RG r
#pragma unroll 2
  for (int k = 0; k < K; k += 4) {
    float4 xv[TM];
#pragma unroll
    for (int r = 0; r < TM; ++r) xv[r] = *reinterpret_cast<const float4*>(X + (mt + RG * r) * kFRow + k);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      float2 b[TN / 2];
      const float2* brow = reinterpret_cast<const float2*>(B + (size_t)(k + kk) * ldb + n0);
#pragma unroll
      for (int c = 0; c < TN / 2; ++c) b[c] = kSharedB ? brow[c] : __ldg(brow + c);
#pragma unroll
      for (int r = 0; r < TM; ++r) {
        const float xk = kk == 0 ? xv[r].x : (kk == 1 ? xv[r].y : (kk == 2 ? xv[r].z : xv[r].w));
        const float2 x2 = make_float2(xk, xk);
#pragma unroll
        for (int c = 0; c < TN / 2; ++c) acc[r][c] = __ffma2_rn(x2, b[c], acc[r][c]);
      }
    }
  }
}

// Layer epilogue: z = acc + bias; relu(z) -> Y (shared, column offset yc)
// and optionally -> act slots (valid rows only).  The reverse pass needs
// only relu(z): it is the next layer's input, and z > 0 iff relu(z) > 0.
template <int TN, int TM = 8>
__device__ __forceinline__ void tile_out(const float2 (&acc)[TM][TN / 2], const float* __restrict__ bias, int mt,
                                         int n0, float* act, int P, int slot, int p0, float* Y, int yc) {
  constexpr int RG = kFM / TM;
  float2 bb[TN / 2];
#pragma unroll
  for (int c = 0; c < TN / 2; ++c) bb[c] = __ldg(reinterpret_cast<const float2*>(bias + n0) + c);
#pragma unroll
  for (int r = 0; r < TM; ++r) {
    const int m = mt + RG * r;
#pragma unroll
    for (int c = 0; c < TN / 2; ++c) {
      const float z0 = fmaxf(acc[r][c].x + bb[c].x, 0.0f), z1 = fmaxf(acc[r][c].y + bb[c].y, 0.0f);
      if (act && p0 + m < P) {
        act[(size_t)(slot + n0 + 2 * c) * P + p0 + m] = z0;
        act[(size_t)(slot + n0 + 2 * c + 1) * P + p0 + m] = z1;
      }
      *reinterpret_cast<float2*>(Y + m * kFRow + yc + n0 + 2 * c) = make_float2(z0, z1);
    }
  }
}

// Row m of Y (columns [yc, yc + N)) <- rows [slot, slot + N) of the
// [slot][P] array src at Gaussian p0 + m (zeros past the end), as 4-byte
// asynchronous copies; complete after cp_async_wait_all() and a barrier.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void rows_async(float* Y, int yc, const float* src, int P, int slot, int p0, int m,
                                           int ys = kFRow) {
  const bool valid = p0 + m < P;
  const float* s0 = src + (size_t)slot * P + (valid ? p0 + m : 0);
#pragma unroll 16
  for (int q = 0; q < N; ++q) cp_async4(Y + m * ys + yc + q, s0 + (size_t)q * P, valid);
}


// Weight tiles staged into shared memory with cp.async, two buffers: the
// tile of the next product is in flight while the current one runs.  (The
// waits are the hardware's group waits: no spinning.)
struct WTile {
  int64_t off;           // float offset of the tile's first element
  int rows, cols, ld;    // copied as [rows][cols] from rows of `ld` floats
};
constexpr int kMaxWTiles = 40;
constexpr int kWBuf = 4096;   // floats per staging buffer (forward)
constexpr int kWBufR = 2048;  // floats per staging buffer (reverse)

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Issue the copy of tile t (if any) into buffer t & 1; always commits a
// group so that "all but the newest group" names tile t - 1.  The caller
// guarantees no thread still reads buffer t & 1.
template <int kBuf = kWBuf>
__device__ __forceinline__ void stage_tile(const WTile* tiles, int ntiles, int t, const float* __restrict__ base,
                                           float* wbuf) {
  if (t < ntiles) {
    const WTile w = tiles[t];
    float* dst = wbuf + (t & 1) * kBuf;
    const int c4 = w.cols / 4, n = w.rows * c4;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = i / c4, c = i - r * c4;
      cp_async16(dst + r * w.cols + 4 * c, base + w.off + (size_t)r * w.ld + 4 * c);
    }
  }
  cp_async_commit();
}

// Tile t: start tile t + 1, wait for tile t, make it visible to the block.
template <int kBuf = kWBuf>
__device__ __forceinline__ const float* next_tile(const WTile* tiles, int ntiles, int& t, const float* base,
                                                  float* wbuf) {
  stage_tile<kBuf>(tiles, ntiles, t + 1, base, wbuf);
  cp_async_wait1();
  __syncthreads();
  const float* w = wbuf + (t & 1) * kBuf;
  ++t;
  return w;
}

struct FwdArgs {
  FstGeom g;
  const float *planes, *wt;
  WTile tiles[kMaxWTiles];
  int ntiles;
  const float *means, *quats, *log_scales, *logits;
  const void* feat;
  int feat_bf16;
  float t;
  float *means_t, *quats_t, *log_scales_t, *logits_t;
  void* feat_t;
  float* act;  // NULL: forward only
  const float* f;  // [P][levels * 32] HexPlane features from fst_sample_kernel
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

// HexPlane features f of every Gaussian (lane-cooperative, four Gaussians
// per iteration), written Gaussian-major [P][levels * 32] for the MLP
// kernel.  A light kernel with many warps per SM, so many corner fetches
// are in flight.
constexpr int kSampThreads = 256;
struct SampArgs {
  FstGeom g;
  const float *planes, *means;
  float t;
  float* f;
};

__global__ void __launch_bounds__(kSampThreads, 2) fst_sample_kernel(const SampArgs a) {
  __shared__ int s_ci[kSampThreads][kFMaxL * 4];
  __shared__ float s_cf[kSampThreads][kFMaxL * 4];
  const FstGeom& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = g.P, nf = g.levels * kFC;
  const int p0 = blockIdx.x * kSampThreads;
  const int p = p0 + tid;
  float mu[3] = {0.0f, 0.0f, 0.0f};
  if (p < P) {
#pragma unroll
    for (int k = 0; k < 3; ++k) mu[k] = a.means[(size_t)p * 3 + k];
  }
  grid_axes(g, mu, a.t, s_ci[tid], s_cf[tid]);
  __syncwarp();
  const int nw = P - (p0 + warp * 32) < 32 ? P - (p0 + warp * 32) : 32;  // Gaussians of this warp (may be <= 0)
  for (int j = 0; j < nw; j += 4) {
    // Four Gaussians at a time (a missing one repeats a valid row and is
    // not stored).
    const int r = warp * 32 + j;
    const int* ci[4];
    const float* cf[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rq = j + q < nw ? r + q : r;
      ci[q] = s_ci[rq];
      cf[q] = s_cf[rq];
    }
    for (int lv = 0; lv < g.levels; ++lv) {
      float f[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] = level_feature(g, a.planes, lv, ci[q], cf[q], lane);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j + q < nw) a.f[(size_t)(p0 + r + q) * nf + lv * kFC + lane] = f[q];
    }
  }
}

constexpr size_t kFwdSmem = ((size_t)2 * kFM * kFRow + 2 * kWBuf) * 4;

template <int D>
__global__ void __launch_bounds__(kFwdThreads, 2) fst_fwd_kernel(const FwdArgs a) {
  // 256 threads over 128 Gaussians: thread (mt, nt) = (tid % 32, tid / 32)
  // owns rows mt + 32 r (r < 4) of every product; threads below 128 also own
  // Gaussian p0 + tid for the per-Gaussian parts (f rows, heads, outputs).
  constexpr int TM = 4;
  extern __shared__ __align__(16) float s_buf[];
  float* A = s_buf;                        // [128][kFRow]
  float* B = s_buf + kFM * kFRow;          // [128][kFRow]
  float* wbuf = s_buf + 2 * kFM * kFRow;   // [2][kWBuf] staged weight tiles
  int wt_i = 0;
  stage_tile(a.tiles, a.ntiles, 0, a.wt, wbuf);
  const FstGeom& g = a.g;
  const int tid = threadIdx.x;
  const int mt = tid & 31, nt = tid >> 5;
  const bool owner = tid < kFM;
  const int p0 = blockIdx.x * kFM;
  const int p = p0 + tid;
  const bool valid = owner && p < g.P;
  const int P = g.P;
  float* act = a.act;
  float mu[3] = {0.0f, 0.0f, 0.0f};
  if (valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k) mu[k] = a.means[(size_t)p * 3 + k];
  }
  // F_out layer 0 over f (written Gaussian-major by the sampling kernel),
  // two levels (64 columns) at a time, copied into A asynchronously.
  const int nf = g.levels * kFC;
  float2 acc[TM][4];
  tile_zero<8, TM>(acc);
  for (int l0 = 0; l0 < g.levels; l0 += 2) {
    const int nl = g.levels - l0 < 2 ? g.levels - l0 : 2;
    if (owner) {
      const float* src = a.f + (size_t)(valid ? p : 0) * nf + l0 * kFC;
      for (int q = 0; q < nl * kFC; q += 4) cp_async16_zfill(A + tid * kFRow + q, src + q, valid);
      cp_async_wait_all();
    }
    __syncthreads();
    if (act && valid) {
      for (int c = 0; c < nl * kFC; ++c) act[(size_t)(g.sf + l0 * kFC + c) * P + p] = A[tid * kFRow + c];
    }
    {
      const float* w = next_tile(a.tiles, a.ntiles, wt_i, a.wt, wbuf);
      tile_mma<8, true, TM>(A, nl * kFC, w, kFW, mt, nt * 8, acc);
    }
    __syncthreads();
  }
  tile_out<8, TM>(acc, a.wt + g.ab[0], mt, nt * 8, act, P, g.sz, p0, B, 0);
  __syncthreads();
  // z_j = W_j relu(z_{j-1}) + b_j; layer j reads (j odd ? B : A).
  for (int j = 1; j < kFDepth; ++j) {
    float* src = (j & 1) ? B : A;
    float* dst = (j & 1) ? A : B;
    tile_zero<8, TM>(acc);
    tile_mma<8, true, TM>(src, kFW, next_tile(a.tiles, a.ntiles, wt_i, a.wt, wbuf), kFW, mt, nt * 8, acc);
    tile_out<8, TM>(acc, a.wt + g.ab[j], mt, nt * 8, act, P, g.sz + j * kFW, p0, dst, 0);
    __syncthreads();
  }
  // relu(h) is in A.  Branches: e1 -> B[0, 32), h_g -> B[32, 64); the
  // semantic updater's first layer accumulates over the branches.
  float2 v[TM][4];
  tile_zero<8, TM>(v);
  float out[11];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int l1 = branch_e1(b);
    {
      float2 e[TM][2];
      tile_zero<4, TM>(e);
      tile_mma<4, true, TM>(A, kFW, next_tile(a.tiles, a.ntiles, wt_i, a.wt, wbuf), kFHalf, mt, nt * 4, e);
      tile_out<4, TM>(e, a.wt + g.ab[l1], mt, nt * 4, act, P, g.se1 + b * kFHalf, p0, B, 0);
    }
    __syncthreads();
    {
      float2 e[TM][2];
      tile_zero<4, TM>(e);
      tile_mma<4, true, TM>(B, kFHalf, next_tile(a.tiles, a.ntiles, wt_i, a.wt, wbuf), kFHalf, mt, nt * 4, e);
      tile_out<4, TM>(e, a.wt + g.ab[l1 + 1], mt, nt * 4, act, P, g.shg + b * kFHalf, p0, B, kFHalf);
    }
    __syncthreads();
    // Head (the owner thread's own Gaussian): offset = H relu(h_g) + b.
    constexpr int dgs[4] = {3, 4, 3, 1}, oos[4] = {0, 3, 7, 10};
    if (owner) {
      const float* hgr = B + tid * kFRow + kFHalf;
      const float* wt_h = a.wt + g.aw[l1 + 2];  // [32][dg]
      const float* bh = a.wt + g.ab[l1 + 2];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        if (o < dgs[b]) {
          float s = __ldg(bh + o);
#pragma unroll 8
          for (int i = 0; i < kFHalf; ++i) s = fmaf(__ldg(wt_h + i * dgs[b] + o), hgr[i], s);
          out[oos[b] + o] = s;
        }
      }
    }
    tile_mma<8, true, TM>(B + kFHalf, kFHalf, next_tile(a.tiles, a.ntiles, wt_i, a.wt, wbuf), kFW, mt, nt * 8, v);
    __syncthreads();
  }
  tile_out<8, TM>(v, a.wt + g.ab[kLZ1], mt, nt * 8, act, P, g.sv, p0, A, 0);
  __syncthreads();
  // dz = Z2 relu(v) + b, 64 columns at a time.
  constexpr int ZN = D < 64 ? D : 64, ZT = ZN / 8;
#pragma unroll
  for (int c0 = 0; c0 < D; c0 += ZN) {
    float2 z[TM][ZT / 2];
    tile_zero<ZT, TM>(z);
    tile_mma<ZT, true, TM>(A, kFW, next_tile(a.tiles, a.ntiles, wt_i, a.wt, wbuf), ZN, mt, nt * ZT, z);
    float2 bb[ZT / 2];
#pragma unroll
    for (int c = 0; c < ZT / 2; ++c) bb[c] = __ldg(reinterpret_cast<const float2*>(a.wt + g.ab[kLZ2] + c0 + nt * ZT) + c);
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      const int pm = p0 + mt + (kFM / TM) * r;
      if (pm < P) {
#pragma unroll
        for (int c = 0; c < ZT / 2; ++c) {
          const size_t i0 = (size_t)pm * D + c0 + nt * ZT + 2 * c;
          store_feat(a.feat_t, a.feat_bf16, i0, load_feat(a.feat, a.feat_bf16, i0) + z[r][c].x + bb[c].x);
          store_feat(a.feat_t, a.feat_bf16, i0 + 1, load_feat(a.feat, a.feat_bf16, i0 + 1) + z[r][c].y + bb[c].y);
        }
      }
    }
    __syncthreads();
  }
  if (!valid) return;
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
  float* df;    // [P][levels * 32]: d f, read by the HexPlane reverse kernel
  float* part;  // [gridDim.x][mlp_aligned]
  WTile tiles[kMaxWTiles];  // row-major weight tiles in order of use (per chunk)
  int ntiles;
};

// pw[o * ldw + i] (+)= sum over the block's 128 Gaussians of
// s_d[g][o] * s_x[g][i], o < NO (<= 64), i < NI (multiple of 8, <= 64);
// pb[o] (+)= sum_g s_d[g][o] when pb is set.  Tiles of TO outputs x 8
// inputs per thread (TO chosen so that the 128 threads have work); the bias
// sum runs as two fixed-order halves of independent partial sums.  Starts
// and ends with a barrier.
template <int TO>
__device__ __forceinline__ void outer_tiles(const float* s_d, int ds, const float* s_x, int xs, int NO, int NI,
                                            float* pw, int ldw, bool first) {
  const int nog = (NO + TO - 1) / TO, ntile = nog * (NI / 8);
  for (int tile = threadIdx.x; tile < ntile; tile += kFThreads) {
    const int o0 = (tile % nog) * TO, i0 = (tile / nog) * 8;
    // The block's partial rows of this tile are loaded before the product,
    // so their L2 round trip overlaps it.
    float4 prev[TO][2];
#pragma unroll
    for (int r = 0; r < TO; ++r) {
      prev[r][0] = prev[r][1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (!first && o0 + r < NO) {
        const float4* row = reinterpret_cast<const float4*>(pw + (size_t)(o0 + r) * ldw + i0);
        prev[r][0] = row[0];
        prev[r][1] = row[1];
      }
    }
    float2 acc[TO][4];
#pragma unroll
    for (int r = 0; r < TO; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.0f, 0.0f);
#pragma unroll 4
    for (int gg = 0; gg < kFThreads; ++gg) {
      float dv[TO];
      if (TO == 4) {
        const float4 d = *reinterpret_cast<const float4*>(s_d + gg * ds + o0);
        dv[0] = d.x; dv[TO > 1 ? 1 : 0] = d.y; dv[TO > 2 ? 2 : 0] = d.z; dv[TO > 3 ? 3 : 0] = d.w;
      } else if (TO == 2) {
        const float2 d = *reinterpret_cast<const float2*>(s_d + gg * ds + o0);
        dv[0] = d.x; dv[TO > 1 ? 1 : 0] = d.y;
      } else {
        dv[0] = s_d[gg * ds + o0];
      }
      const float4 x0 = *reinterpret_cast<const float4*>(s_x + gg * xs + i0);
      const float4 x1 = *reinterpret_cast<const float4*>(s_x + gg * xs + i0 + 4);
#pragma unroll
      for (int r = 0; r < TO; ++r) {
        const float2 dd = make_float2(dv[r], dv[r]);
        acc[r][0] = __ffma2_rn(dd, make_float2(x0.x, x0.y), acc[r][0]);
        acc[r][1] = __ffma2_rn(dd, make_float2(x0.z, x0.w), acc[r][1]);
        acc[r][2] = __ffma2_rn(dd, make_float2(x1.x, x1.y), acc[r][2]);
        acc[r][3] = __ffma2_rn(dd, make_float2(x1.z, x1.w), acc[r][3]);
      }
    }
    // Partial += this chunk's sums (the partial loaded above; zero for the
    // block's first chunk, whose sums are stored as they are).
#pragma unroll
    for (int r = 0; r < TO; ++r) {
      if (o0 + r < NO) {
        float4* row = reinterpret_cast<float4*>(pw + (size_t)(o0 + r) * ldw + i0);
        float4 v0 = make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
        float4 v1 = make_float4(acc[r][2].x, acc[r][2].y, acc[r][3].x, acc[r][3].y);
        if (!first) {
          const float4 a0 = prev[r][0], a1 = prev[r][1];
          v0.x += a0.x; v0.y += a0.y; v0.z += a0.z; v0.w += a0.w;
          v1.x += a1.x; v1.y += a1.y; v1.z += a1.z; v1.w += a1.w;
        }
        row[0] = v0;
        row[1] = v1;
      }
    }
  }
}

__device__ void block_outer(const float* s_d, int ds, const float* s_x, int xs, int NO, int NI, float* pw, int ldw,
                            float* pb, bool first) {
  __shared__ float s_red[kFThreads];
  __syncthreads();
  if (NO >= 4 && (NO / 4) * (NI / 8) >= kFThreads)
    outer_tiles<4>(s_d, ds, s_x, xs, NO, NI, pw, ldw, first);
  else if (NO >= 2 && (NO / 2) * (NI / 8) >= kFThreads / 2)
    outer_tiles<2>(s_d, ds, s_x, xs, NO, NI, pw, ldw, first);
  else
    outer_tiles<1>(s_d, ds, s_x, xs, NO, NI, pw, ldw, first);
  if (pb) {
    const int o = threadIdx.x & 63, half = threadIdx.x >> 6;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (o < NO) {
#pragma unroll 4
      for (int gg = half * 64; gg < half * 64 + 64; gg += 4) {
        s0 += s_d[gg * ds + o];
        s1 += s_d[(gg + 1) * ds + o];
        s2 += s_d[(gg + 2) * ds + o];
        s3 += s_d[(gg + 3) * ds + o];
      }
    }
    s_red[threadIdx.x] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (threadIdx.x < NO) {
      const float v = s_red[threadIdx.x] + s_red[threadIdx.x + 64];
      pb[threadIdx.x] = first ? v : pb[threadIdx.x] + v;
    }
  }
  __syncthreads();
}

// Exact, order-independent plane-gradient sums.  Each float contribution x
// is the integer X = x 2^72 (exact for |x| >= 2^-49; smaller ones rounded to
// the nearest multiple of 2^-72), held as hi 2^32 + lo with 0 <= lo < 2^32,
// and added with 64-bit integer atomics into hi[i] (two's complement) and
// lo[i]: integer sums do not depend on the order of the additions, so the
// result is the same bits however the Gaussians are scheduled.  |sum| must
// stay below 2^23 (contributions at or above it are clamped and flagged).
__device__ __forceinline__ void fixed_add(unsigned long long* hi, unsigned long long* lo, size_t i, float x,
                                          uint32_t* err) {
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFFu);
  if (e == 0) return;  // zero or below 2^-126: under the resolution
  uint64_t m = (u & 0x7FFFFFu) | 0x800000u;  // |x| = m 2^(e - 150)
  int sh = e - 150 + 72;                      // |X| = m 2^sh
  if (sh > 71) {                              // |x| >= 2^23
    set_err(err, kErrOverflow);
    m = 0xFFFFFFu;
    sh = 71;
  }
  uint64_t h, l;
  if (sh >= 32) {
    h = m << (sh - 32);
    l = 0;
  } else if (sh >= 0) {
    const uint64_t X = m << sh;
    h = X >> 32;
    l = X & 0xFFFFFFFFull;
  } else if (sh > -25) {
    h = 0;
    l = (m + (1ull << (-sh - 1))) >> (-sh);  // nearest, ties up
  } else {
    return;
  }
  if (u >> 31) {  // -(h 2^32 + l)
    if (l) {
      h = ~h;            // -h - 1
      l = 0x100000000ull - l;
    } else {
      h = ~h + 1ull;     // -h
    }
  }
  if (h) atomicAdd(hi + i, (unsigned long long)h);
  if (l) atomicAdd(lo + i, (unsigned long long)l);
}

// Lane-cooperative reverse of one level's HexPlane sample for NG Gaussians
// at once (lane = channel, dfc[q] = d f of this channel for Gaussian q): all
// corner fetches are issued before any arithmetic, plane gradients by
// atomics, coordinate gradients summed over the warp into dc[q][0..2]
// (lane 0 adds).
template <int NG>
__device__ __forceinline__ void plane_backward(const FstGeom& g, const float* __restrict__ planes, float* d_planes,
                                               unsigned long long* acc_hi, unsigned long long* acc_lo, uint32_t* err,
                                               int lv, const int* const* ci, const float* const* cf, const float* dfc,
                                               int lane, float* const* dc) {
  float q00[NG][6], q01[NG][6], q10[NG][6], q11[NG][6];
#pragma unroll
  for (int n = 0; n < NG; ++n) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int ia = ci[n][lv * 4 + pair_a(k)] & 0x3FFFFFFF, ib = ci[n][lv * 4 + pair_b(k)] & 0x3FFFFFFF;
      const int rb = g.prb[lv * 6 + k];
      const float* base = planes + g.poff[lv * 6 + k] + ((size_t)ia * rb + ib) * kFC + lane;
      q00[n][k] = __ldg(base);
      q01[n][k] = __ldg(base + kFC);
      q10[n][k] = __ldg(base + (size_t)rb * kFC);
      q11[n][k] = __ldg(base + (size_t)rb * kFC + kFC);
    }
  }
#pragma unroll
  for (int n = 0; n < NG; ++n) {
    float smp[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float fa = cf[n][lv * 4 + pair_a(k)], fb = cf[n][lv * 4 + pair_b(k)];
      smp[k] = (1.0f - fa) * ((1.0f - fb) * q00[n][k] + fb * q01[n][k]) + fa * ((1.0f - fb) * q10[n][k] + fb * q11[n][k]);
    }
    float dcl[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float others = 1.0f;
#pragma unroll
      for (int m = 0; m < 6; ++m)
        if (m != k) others *= smp[m];
      const float ds = dfc[n] * others;
      const int A = pair_a(k), B = pair_b(k);
      const int ca = ci[n][lv * 4 + A], cb = ci[n][lv * 4 + B];
      const int ia = ca & 0x3FFFFFFF, ib = cb & 0x3FFFFFFF;
      const float fa = cf[n][lv * 4 + A], fb = cf[n][lv * 4 + B];
      const int rb = g.prb[lv * 6 + k];
      const size_t di = g.poff[lv * 6 + k] + ((size_t)ia * rb + ib) * kFC + lane;
      const float w00 = (1.0f - fa) * (1.0f - fb) * ds, w01 = (1.0f - fa) * fb * ds;
      const float w10 = fa * (1.0f - fb) * ds, w11 = fa * fb * ds;
      if (acc_hi) {
        fixed_add(acc_hi, acc_lo, di, w00, err);
        fixed_add(acc_hi, acc_lo, di + kFC, w01, err);
        fixed_add(acc_hi, acc_lo, di + (size_t)rb * kFC, w10, err);
        fixed_add(acc_hi, acc_lo, di + (size_t)rb * kFC + kFC, w11, err);
      } else {
        atomicAdd(d_planes + di, w00);
        atomicAdd(d_planes + di + kFC, w01);
        atomicAdd(d_planes + di + (size_t)rb * kFC, w10);
        atomicAdd(d_planes + di + (size_t)rb * kFC + kFC, w11);
      }
      if (!(ca >> 30))  // A is always a spatial axis
        dcl[A] += ds * ((1.0f - fb) * (q10[n][k] - q00[n][k]) + fb * (q11[n][k] - q01[n][k])) * 0.5f *
                  (float)(g.pra[lv * 6 + k] - 1);
      if (B < 3 && !(cb >> 30))
        dcl[B < 3 ? B : 0] += ds * ((1.0f - fa) * (q01[n][k] - q00[n][k]) + fa * (q11[n][k] - q10[n][k])) * 0.5f *
                              (float)(rb - 1);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float v = dcl[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      dcl[k] = v;
    }
    if (lane == 0) {
      dc[n][0] += dcl[0];
      dc[n][1] += dcl[1];
      dc[n][2] += dcl[2];
    }
  }
}

// Y[m][yc + n] <- (X[m][xc + n] > 0 ? acc : 0) for the thread's tile (the
// ReLU mask read from the stored relu(z) inputs); dv rows optionally copied
// to global [n][P].
template <int TN>
__device__ __forceinline__ void tile_mask(const float2 (&acc)[8][TN / 2], const float* X, int xc, float* Y, int yc,
                                          int mt, int n0, float* rows, int P, int p0, int xs = kFRow) {
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int m = mt + 16 * r;
#pragma unroll
    for (int c = 0; c < TN / 2; ++c) {
      const float2 x = *reinterpret_cast<const float2*>(X + m * xs + xc + n0 + 2 * c);
      const float2 d = make_float2(x.x > 0.0f ? acc[r][c].x : 0.0f, x.y > 0.0f ? acc[r][c].y : 0.0f);
      *reinterpret_cast<float2*>(Y + m * kFRow + yc + n0 + 2 * c) = d;
      if (rows && p0 + m < P) {
        rows[(size_t)(n0 + 2 * c) * P + p0 + m] = d.x;
        rows[(size_t)(n0 + 2 * c + 1) * P + p0 + m] = d.y;
      }
    }
  }
}

constexpr int kTRow = 36;  // row stride of the small third buffer
constexpr size_t kBwdSmem = ((size_t)(2 * kFRow + kTRow) * kFThreads + 2 * kWBufR) * 4;


template <int D>
__global__ void __launch_bounds__(kFThreads, 2) fst_bwd_kernel(const BwdArgs a) {
  extern __shared__ __align__(16) float s_dyn[];
  float* SD = s_dyn;                            // [128][kFRow]: deltas
  float* SX = s_dyn + kFThreads * kFRow;        // [128][kFRow]: layer inputs
  float* ST = s_dyn + 2 * kFThreads * kFRow;    // [128][kTRow]: relu(h_g) | head deltas; grid axes
  float* wbuf = ST + kFThreads * kTRow;         // [2][kWBufR] staged weight tiles
  const FstGeom& g = a.g;
  const int tid = threadIdx.x;
  const int mt = tid & 15, nt = tid >> 4;
  const int P = g.P;
  const int nchunk = (P + kFThreads - 1) / kFThreads;
  float* part = a.part + (size_t)blockIdx.x * g.mlp_aligned;
  const float* act = a.act;
  for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
    const bool first = chunk == (int)blockIdx.x;
    const int p0 = chunk * kFThreads;
    const int p = p0 + tid;
    const bool valid = p < P;
    int wt_i = 0;
    stage_tile<kWBufR>(a.tiles, a.ntiles, 0, a.wn, wbuf);
    // ---- F_feat second layer: delta = d dz; input relu(v).
    rows_async<kFW>(SX, 0, act, P, g.sv, p0, tid);
    float2 acc[8][4];
    tile_zero<8>(acc);
    constexpr int NC = D < 64 ? D : 64;
    for (int c0 = 0; c0 < D; c0 += NC) {
      for (int q = 0; q < NC; q += 4)
        *reinterpret_cast<float4*>(SD + tid * kFRow + q) =
            valid ? __ldg(reinterpret_cast<const float4*>(a.d_feat_t + (size_t)p * D + c0 + q)) : make_float4(0.f, 0.f, 0.f, 0.f);
      cp_async_wait_all();
      block_outer(SD, kFRow, SX, kFRow, NC, kFW, part + g.aw[kLZ2] + (size_t)c0 * kFW, kFW, part + g.ab[kLZ2] + c0, first);
      for (int r0 = 0; r0 < NC; r0 += 32) {
        if (r0) __syncthreads();
        const float* w = next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf);
        tile_mma<8, true>(SD + r0, NC - r0 < 32 ? NC - r0 : 32, w, kFW, mt, nt * 8, acc);
      }
      __syncthreads();
    }
    // delta_v (kept in SD and in the workspace for the branches).
    tile_mask<8>(acc, SX, 0, SD, 0, mt, nt * 8, a.dv, P, p0);
    // ---- F_feat first layer: input relu(u), u = [h_mu, h_R, h_S, h_o].
    for (int half = 0; half < 2; ++half) {
      __syncthreads();
      rows_async<kFW>(SX, 0, act, P, g.shg + half * kFW, p0, tid);
      cp_async_wait_all();
      block_outer(SD, kFRow, SX, kFRow, kFW, kFW, part + g.aw[kLZ1] + half * kFW, 4 * kFHalf, half ? nullptr : part + g.ab[kLZ1],
                  first);
    }
    // ---- Branches; d relu(h) accumulates over them.
    float2 drh[8][4];
    tile_zero<8>(drh);
    const float* dsrc[4] = {a.d_means_t, a.d_quats_t, a.d_log_scales_t, a.d_logits_t};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      constexpr int dgs[4] = {3, 4, 3, 1};
      const int dg = dgs[b], l1 = branch_e1(b);
      // delta_v rows -> SX; relu(h_g) and the head deltas -> ST.
      __syncthreads();
      rows_async<kFW>(SX, 0, a.dv, P, 0, p0, tid);
      rows_async<kFHalf>(ST, 0, act, P, g.shg + b * kFHalf, p0, tid, kTRow);
#pragma unroll
      for (int o = 0; o < 4; ++o) ST[tid * kTRow + kFHalf + o] = (o < dg && valid) ? __ldg(dsrc[b] + (size_t)p * dg + o) : 0.0f;
      cp_async_wait_all();
      __syncthreads();
      // d relu(h_g) = Z1[:, branch b]^T delta_v + H^T d offset, masked.
      float2 e[8][2];
      tile_zero<4>(e);
      tile_mma<4, true>(SX, kFW, next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf), kFHalf, mt, nt * 4, e);
      {
        const float* wh = a.wn + g.aw[l1 + 2];  // [dg][32]
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float* dh = ST + (mt + 16 * r) * kTRow + kFHalf;
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            if (o < dg) {
              const float2 d2 = make_float2(dh[o], dh[o]);
#pragma unroll
              for (int c = 0; c < 2; ++c)
                e[r][c] = __ffma2_rn(d2, __ldg(reinterpret_cast<const float2*>(wh + o * kFHalf + nt * 4) + c), e[r][c]);
            }
          }
        }
      }
      tile_mask<4>(e, ST, 0, SD, 0, mt, nt * 4, nullptr, P, p0, kTRow);   // delta_hg -> SD[0, 32)
      // head: delta = d offset (ST[32, 36)), input relu(h_g) (ST[0, 32)).
      block_outer(ST + kFHalf, kTRow, ST, kTRow, dg, kFHalf, part + g.aw[l1 + 2], kFHalf, part + g.ab[l1 + 2], first);
      // E2: delta_hg (SD[0, 32)), input relu(e1).
      rows_async<kFHalf>(SX, 0, act, P, g.se1 + b * kFHalf, p0, tid);
      cp_async_wait_all();
      block_outer(SD, kFRow, SX, kFRow, kFHalf, kFHalf, part + g.aw[l1 + 1], kFHalf, part + g.ab[l1 + 1], first);
      tile_zero<4>(e);
      tile_mma<4, true>(SD, kFHalf, next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf), kFHalf, mt, nt * 4, e);
      __syncthreads();
      tile_mask<4>(e, SX, 0, SD, 0, mt, nt * 4, nullptr, P, p0);   // delta_e1 -> SD[0, 32)
      __syncthreads();
      // E1: delta_e1, input relu(h).
      rows_async<kFW>(SX, 0, act, P, g.sz + (kFDepth - 1) * kFW, p0, tid);
      cp_async_wait_all();
      block_outer(SD, kFRow, SX, kFRow, kFHalf, kFW, part + g.aw[l1], kFW, part + g.ab[l1], first);
      tile_mma<8, true>(SD, kFHalf, next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf), kFW, mt, nt * 8, drh);
    }
    // ---- F_out, last layer first.  SX holds relu(h).
    __syncthreads();
    tile_mask<8>(drh, SX, 0, SD, 0, mt, nt * 8, nullptr, P, p0);
    for (int j = kFDepth - 1; j >= 1; --j) {
      __syncthreads();
      rows_async<kFW>(SX, 0, act, P, g.sz + (j - 1) * kFW, p0, tid);
      cp_async_wait_all();
      block_outer(SD, kFRow, SX, kFRow, kFW, kFW, part + g.aw[j], kFW, part + g.ab[j], first);
      tile_zero<8>(acc);
      tile_mma<8, true>(SD, 32, next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf), kFW, mt, nt * 8, acc);
      __syncthreads();
      tile_mma<8, true>(SD + 32, 32, next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf), kFW, mt, nt * 8, acc);
      __syncthreads();
      tile_mask<8>(acc, SX, 0, SD, 0, mt, nt * 8, nullptr, P, p0);
    }
    // First layer: input f.
    const int nf = g.levels * kFC;
    for (int c0 = 0; c0 < nf; c0 += kFW) {
      const int nc = nf - c0 < kFW ? nf - c0 : kFW;
      __syncthreads();
      if (nc == kFW) rows_async<kFW>(SX, 0, act, P, g.sf + c0, p0, tid);
      else rows_async<kFC>(SX, 0, act, P, g.sf + c0, p0, tid);
      cp_async_wait_all();
      block_outer(SD, kFRow, SX, kFRow, kFW, nc, part + g.aw[0] + c0, nf, c0 ? nullptr : part + g.ab[0], first);
    }
    // ---- d f = W0^T delta_0, 32 columns per level, staged in SX and
    // written Gaussian-major for the HexPlane reverse kernel.
    for (int lv = 0; lv < g.levels; ++lv) {
      float2 e[8][2];
      tile_zero<4>(e);
      tile_mma<4, true>(SD, kFW, next_tile<kWBufR>(a.tiles, a.ntiles, wt_i, a.wn, wbuf), kFC, mt, nt * 4, e);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          *reinterpret_cast<float2*>(SX + (mt + 16 * r) * kFRow + nt * 4 + 2 * c) = e[r][c];
      __syncthreads();
      if (valid) {
        float4* dst = reinterpret_cast<float4*>(a.df + (size_t)p * nf + lv * kFC);
#pragma unroll
        for (int q = 0; q < kFC / 4; ++q) dst[q] = *reinterpret_cast<const float4*>(SX + tid * kFRow + 4 * q);
      }
    }
    __syncthreads();  // the buffers are rewritten by the next chunk
  }
}

// HexPlane reverse: per Gaussian and level, d f (Gaussian-major rows) through
// the channel-wise product and the bilinear weights -- plane gradients by
// coalesced atomics, the canonical mean's gradient summed over the warp
// (one warp owns each Gaussian: reproducible).  A light kernel with many
// warps per SM, so many corner fetches are in flight.
constexpr int kHexThreads = 256;
struct HexArgs {
  FstGeom g;
  const float *planes, *means, *df, *d_means_t;
  float t;
  float* d_means;
  float* d_planes;                      // float-atomic plane sums (acc_hi == NULL)
  unsigned long long *acc_hi, *acc_lo;  // or exact plane-gradient sums (fixed_add)
  uint32_t* err;
};

// d_planes[i] = the exact sum hi 2^32 + lo, times 2^-72, rounded to float.
__global__ void __launch_bounds__(256) fst_planes_out_kernel(const unsigned long long* __restrict__ hi,
                                                             const unsigned long long* __restrict__ lo, int64_t n,
                                                             float* __restrict__ d_planes) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)(long long)hi[i] * 0x1p-40 + (double)lo[i] * 0x1p-72;
    d_planes[i] = (float)v;
  }
}

__global__ void __launch_bounds__(kHexThreads, 2) fst_hex_bwd_kernel(const HexArgs a) {
  __shared__ int s_ci[kHexThreads][kFMaxL * 4];
  __shared__ float s_cf[kHexThreads][kFMaxL * 4];
  __shared__ float s_dc[kHexThreads][4];
  const FstGeom& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = g.P, nf = g.levels * kFC;
  const int p0 = blockIdx.x * kHexThreads;
  const int p = p0 + tid;
  const bool valid = p < P;
  float mu[3] = {0.f, 0.f, 0.f};
  if (valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k) mu[k] = a.means[(size_t)p * 3 + k];
  }
  grid_axes(g, mu, a.t, s_ci[tid], s_cf[tid]);
  s_dc[tid][0] = s_dc[tid][1] = s_dc[tid][2] = 0.0f;
  __syncwarp();
  const int nw = P - (p0 + warp * 32) < 32 ? P - (p0 + warp * 32) : 32;  // Gaussians of this warp
  for (int lv = 0; lv < g.levels; ++lv) {
    int j = 0;
    for (; j + 1 < nw; j += 2) {
      const int r = warp * 32 + j;
      const int* ci[2] = {s_ci[r], s_ci[r + 1]};
      const float* cf[2] = {s_cf[r], s_cf[r + 1]};
      const float dfc[2] = {__ldg(a.df + (size_t)(p0 + r) * nf + lv * kFC + lane),
                            __ldg(a.df + (size_t)(p0 + r + 1) * nf + lv * kFC + lane)};
      float* dc[2] = {s_dc[r], s_dc[r + 1]};
      plane_backward<2>(g, a.planes, a.d_planes, a.acc_hi, a.acc_lo, a.err, lv, ci, cf, dfc, lane, dc);
    }
    if (j < nw) {
      const int r = warp * 32 + j;
      const int* ci[1] = {s_ci[r]};
      const float* cf[1] = {s_cf[r]};
      const float dfc[1] = {__ldg(a.df + (size_t)(p0 + r) * nf + lv * kFC + lane)};
      float* dc[1] = {s_dc[r]};
      plane_backward<1>(g, a.planes, a.d_planes, a.acc_hi, a.acc_lo, a.err, lv, ci, cf, dfc, lane, dc);
    }
  }
  __syncwarp();
  if (valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      a.d_means[(size_t)p * 3 + k] = a.d_means_t[(size_t)p * 3 + k] + s_dc[tid][k] * g.scale[k];
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
constexpr int kTvMaxBlocks = 1024;  // loss partials (the caller's scratch)

struct TvArgs {
  FstGeom g;
  const float* planes;
  float* d_planes;
  float weight;
  float* partial;                   // [gridDim.x]
  int bstart[kFMaxL * 6 + 1];       // first block of each plane (blocks in proportion to plane size)
};

// Each plane gets a share of the blocks in proportion to its size; each
// thread takes four channels of a node (the planes are channels-last, so a
// float4 per neighbour).  One loss partial per block, summed in a fixed
// order afterwards.
__global__ void __launch_bounds__(256) fst_tv_kernel(const TvArgs a) {
  __shared__ float s_w[8];
  const FstGeom& g = a.g;
  int k = 0;
  while (k + 1 < g.levels * 6 && (int)blockIdx.x >= a.bstart[k + 1]) ++k;
  const int b0 = a.bstart[k], nb = a.bstart[k + 1] - b0;
  const int ra = g.pra[k], rb = g.prb[k];
  const float4* pl = reinterpret_cast<const float4*>(a.planes + g.poff[k]);
  float4* dp = reinterpret_cast<float4*>(a.d_planes + g.poff[k]);
  const int q4 = kFC / 4;
  const int total = ra * rb * q4;
  const float ia = 1.0f / (float)((int64_t)(ra - 1) * rb * kFC), ib = 1.0f / (float)((int64_t)ra * (rb - 1) * kFC);
  float acc = 0.0f;
  for (int e = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x; e < total; e += nb * blockDim.x) {
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
    a.partial[blockIdx.x] = t;
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

extern "C" fe_status fe_fst_workspace_size(int P, int levels, int rs, int rt, int D, int with_backward,
                                           size_t* bytes) {
  if (!bytes) return FE_ERR_INVALID_ARG;
  fe_fst f{};
  f.levels = levels;
  f.rs = rs;
  f.rt = rt;
  f.D = D;
  for (int a = 0; a < 3; ++a) f.bbox_max[a] = 1.0f;
  FstGeom g;
  if (!make_geom(&f, P, g)) return (D == 16 || D == 32 || D == 64 || D == 128) ? FE_ERR_INVALID_ARG : FE_ERR_UNSUPPORTED;
  if (with_backward < 0 || with_backward > 2) return FE_ERR_INVALID_ARG;
  *bytes = ws_layout(g, with_backward).total;
  return FE_OK;
}

namespace {

template <int D>
cudaError_t launch_fst_fwd(const FwdArgs& a, cudaStream_t st) {
  const int blocks = (a.g.P + kFM - 1) / kFM;
  const size_t smem = kFwdSmem;
  auto k = fst_fwd_kernel<D>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<blocks, kFwdThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_fst_bwd(const BwdArgs& a, int nblk, cudaStream_t st) {
  const size_t smem = kBwdSmem;
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
  if (cudaMemsetAsync(wt, 0, w.f - w.wt, st) != cudaSuccess) return FE_ERR_CUDA;
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
  a.f = reinterpret_cast<const float*>(ws + w.f);
  {
    SampArgs sa{};
    sa.g = g;
    sa.planes = fst->planes;
    sa.means = means;
    sa.t = t;
    sa.f = reinterpret_cast<float*>(ws + w.f);
    fst_sample_kernel<<<(P + kSampThreads - 1) / kSampThreads, kSampThreads, 0, st>>>(sa);
  }
  // Weight tiles of the transposed copy in the order the kernel uses them.
  {
    int n = 0;
    auto add = [&](int64_t off, int rows, int cols, int ld) { a.tiles[n++] = WTile{off, rows, cols, ld}; };
    for (int l0 = 0; l0 < g.levels; l0 += 2) {
      const int nl = g.levels - l0 < 2 ? g.levels - l0 : 2;
      add(g.aw[0] + (int64_t)l0 * kFC * kFW, nl * kFC, kFW, kFW);
    }
    for (int j = 1; j < kFDepth; ++j) add(g.aw[j], kFW, kFW, kFW);
    for (int b = 0; b < 4; ++b) {
      add(g.aw[branch_e1(b)], kFW, kFHalf, kFHalf);
      add(g.aw[branch_e1(b) + 1], kFHalf, kFHalf, kFHalf);
      add(g.aw[kLZ1] + (int64_t)b * kFHalf * kFW, kFHalf, kFW, kFW);
    }
    const int zn = g.D < 64 ? g.D : 64;
    for (int c0 = 0; c0 < g.D; c0 += zn) add(g.aw[kLZ2] + c0, kFW, zn, g.D);
    a.ntiles = n;
  }
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
  const bool exact = fst->exact_planes != 0;
  const WsLayout w = ws_layout(g, exact ? 2 : 1);
  if (workspace_bytes < w.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t npl = plane_floats(g);
  if (P == 0) {
    if (cudaMemsetAsync(d_planes, 0, (size_t)npl * 4, st) != cudaSuccess) return FE_ERR_CUDA;
    return cudaMemsetAsync(d_mlp, 0, (size_t)g.mlp_packed * 4, st) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
  }
  if (!fst->planes || !means || !d_means_t || !d_quats_t || !d_log_scales_t || !d_opacity_logits_t || !d_feat_t ||
      !d_means || !al16p(d_feat_t))
    return FE_ERR_INVALID_ARG;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  unsigned long long* acc_hi = exact ? reinterpret_cast<unsigned long long*>(ws + w.acc) : nullptr;
  unsigned long long* acc_lo = exact ? acc_hi + npl : nullptr;
  if (cudaMemsetAsync(ws, 0, kWsHeader, st) != cudaSuccess) return FE_ERR_CUDA;
  if (exact) {
    if (cudaMemsetAsync(acc_hi, 0, (size_t)npl * 16, st) != cudaSuccess) return FE_ERR_CUDA;
  } else if (cudaMemsetAsync(d_planes, 0, (size_t)npl * 4, st) != cudaSuccess) {
    return FE_ERR_CUDA;
  }
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
  a.df = reinterpret_cast<float*>(ws + w.df);
  a.part = reinterpret_cast<float*>(ws + w.part);
  // Row-major weight tiles (at most 2048 floats) in the order the kernel
  // uses them for every chunk.
  {
    int n = 0;
    auto add = [&](int64_t off, int rows, int cols, int ld) { a.tiles[n++] = WTile{off, rows, cols, ld}; };
    const int nc = g.D < 64 ? g.D : 64;
    for (int c0 = 0; c0 < g.D; c0 += nc)
      for (int r0 = 0; r0 < nc; r0 += 32) add(g.aw[kLZ2] + (int64_t)(c0 + r0) * kFW, nc - r0 < 32 ? nc - r0 : 32, kFW, kFW);
    for (int b = 0; b < 4; ++b) {
      add(g.aw[kLZ1] + b * kFHalf, kFW, kFHalf, 4 * kFHalf);
      add(g.aw[branch_e1(b) + 1], kFHalf, kFHalf, kFHalf);
      add(g.aw[branch_e1(b)], kFHalf, kFW, kFW);
    }
    for (int j = kFDepth - 1; j >= 1; --j) {
      add(g.aw[j], 32, kFW, kFW);
      add(g.aw[j] + 32 * kFW, 32, kFW, kFW);
    }
    const int nf = g.levels * kFC;
    for (int lv = 0; lv < g.levels; ++lv) add(g.aw[0] + lv * kFC, kFW, kFC, nf);
    a.ntiles = n;
  }
  const int nblk = bwd_blocks(P);
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.D) {
    case 16: e = launch_fst_bwd<16>(a, nblk, st); break;
    case 32: e = launch_fst_bwd<32>(a, nblk, st); break;
    case 64: e = launch_fst_bwd<64>(a, nblk, st); break;
    case 128: e = launch_fst_bwd<128>(a, nblk, st); break;
  }
  if (e != cudaSuccess) return FE_ERR_CUDA;
  {
    HexArgs h{};
    h.g = g;
    h.planes = fst->planes;
    h.means = means;
    h.df = a.df;
    h.d_means_t = d_means_t;
    h.t = t;
    h.d_means = d_means;
    h.d_planes = d_planes;
    h.acc_hi = acc_hi;
    h.acc_lo = acc_lo;
    h.err = reinterpret_cast<uint32_t*>(ws);
    fst_hex_bwd_kernel<<<(P + kHexThreads - 1) / kHexThreads, kHexThreads, 0, st>>>(h);
    if (exact) {
      const int64_t nb = (npl + 255) / 256;
      fst_planes_out_kernel<<<(int)(nb < 152 * 16 ? nb : 152 * 16), 256, 0, st>>>(acc_hi, acc_lo, npl, d_planes);
    }
  }
  fst_reduce_kernel<<<(int)((g.mlp_packed + 255) / 256), 256, 0, st>>>(g, a.part, nblk, d_mlp);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" fe_status fe_fst_tv(const fe_fst* fst, float weight, float* loss, float* d_planes, float* scratch,
                               void* stream) {
  FstGeom g;
  if (!fst || !make_geom(fst, 0, g)) return FE_ERR_INVALID_ARG;
  if (!fst->planes || !loss || !d_planes || !scratch) return FE_ERR_INVALID_ARG;
  {
    // The gradient array must not overlap the planes (the kernel reads the
    // planes while it updates the gradient).
    const uintptr_t p0 = reinterpret_cast<uintptr_t>(fst->planes), d0 = reinterpret_cast<uintptr_t>(d_planes);
    const uintptr_t n = (uintptr_t)plane_floats(g) * sizeof(float);
    if (p0 < d0 + n && d0 < p0 + n) return FE_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TvArgs a{};
  a.g = g;
  a.planes = fst->planes;
  a.d_planes = d_planes;
  a.weight = weight;
  a.partial = scratch;
  // Blocks per plane in proportion to its size (at least one), at most
  // kTvMaxBlocks in all.
  const int np = g.levels * 6;
  const double total = (double)plane_floats(g);
  const int budget = kTvMaxBlocks - np;
  a.bstart[0] = 0;
  for (int k = 0; k < np; ++k) {
    const double n = (double)g.pra[k] * g.prb[k] * kFC;
    a.bstart[k + 1] = a.bstart[k] + 1 + (int)(budget * n / total);
  }
  const int nblk = a.bstart[np];
  fst_tv_kernel<<<nblk, 256, 0, st>>>(a);
  fst_tv_finish<<<1, 32, 0, st>>>(scratch, nblk, weight, loss);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
