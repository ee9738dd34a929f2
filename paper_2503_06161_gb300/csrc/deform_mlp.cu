// Deformation MLP of the FST query (Sec. 3.2, Eq. 4; App. A widths, single
// level): for every Gaussian, from its HexPlane feature f (C channels),
//   h1 = relu(W1 f + b1),  h2 = relu(W2 h1 + b2),  delta = Wh h2 + bh
// (64, 64 and 11 outputs), with the two ReLU unit masks kept for the
// reverse pass.  The products run on the 5th-generation tensor cores
// (tcgen05, kind::f16): every FP32 operand x is carried as three BF16 terms
// x = hi + mid + lo, each the BF16 rounding of what the previous terms
// leave (24 significant bits in all), and each layer's product as the six
// term products whose size is at most 2^-16 of |x||w| (hi.hi, hi.mid,
// mid.hi, hi.lo, mid.mid, lo.hi), accumulated in FP32 in tensor memory; the
// three dropped products are below 2^-24 of |x||w|, the rounding of FP32
// arithmetic itself.  The products are issued smallest first: added to an
// accumulator that already holds hi.hi, the tensor core's FP32 accumulation
// loses much of the 2^-16 terms (measured: forward errors against an FP64
// reference several times those of FP32 FMAs when issued largest first).
// The reverse of the MLP (deform_mlp_bwd_kernel, below) has the same form.
//
// Each CTA walks 128-Gaussian tiles (two CTAs per SM).  Warp roles:
//   warps 0-3  epilogue: one Gaussian (tensor-memory lane) per thread; bias,
//              ReLU, unit masks and the three-term split of the next
//              layer's input, written over the tile's operand buffer
//   warp 4     tensor-core issue (one thread) and tensor-memory allocation
//   warp 5     TMA loads of the split feature rows of each tile
// Per tile: the feature terms arrive (TMA), layer 1 (K = C), the epilogue
// writes h1's terms, layer 2 (K = 64), the epilogue writes h2's terms,
// layer 3 (K = 64, N = 16 with rows 11-15 zero), the epilogue writes delta
// and the masks.  The operand buffer is free again once layer 3's products
// complete, so the next tile's feature terms load while the epilogue
// finishes this tile.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace fe {

namespace {

using namespace tc;
using namespace tc_host;

constexpr int kMlpBM = 128;                 // Gaussians per tile (MMA M)
constexpr int kMlpEpiWarps = 4;
constexpr int kMlpWarpMma = 4, kMlpWarpTma = 5;
constexpr int kMlpThreads = 32 * 6;
constexpr uint32_t kMlpTmemCols = 256;      // D1 [0, 64), D2 [64, 128), D3 [128, 144)
constexpr uint32_t kColD1 = 0, kColD2 = 64, kColD3 = 128;
constexpr int kNTerms = 3;
// The six (input term, weight term) products of every layer, smallest
// first: lo.hi, mid.mid, hi.lo, mid.hi, hi.mid, hi.hi.
__device__ constexpr int kPairA[6] = {2, 1, 0, 1, 0, 0};
__device__ constexpr int kPairW[6] = {0, 1, 2, 0, 1, 0};

template <int C>
struct MlpCfg {
  static constexpr uint32_t row1 = C * 2;                    // bytes of a layer-1 row (K = C)
  static constexpr uint64_t layout1 = C == 32 ? kLayout64B : kLayout128B;
  static constexpr uint32_t w1_term = kHidden * row1;         // one term of W1 [64][C]
  static constexpr uint32_t w2_term = kHidden * 128;          // one term of W2 [64][64]
  static constexpr uint32_t wh_term = 16 * 128;               // one term of Wh [16][64]
  static constexpr uint32_t a_term = kMlpBM * 128;            // one term of a tile's operand rows
  static constexpr uint32_t off_w1 = 0;
  static constexpr uint32_t off_w2 = off_w1 + kNTerms * w1_term;
  static constexpr uint32_t off_wh = off_w2 + kNTerms * w2_term;
  static constexpr uint32_t off_a = off_wh + kNTerms * wh_term;
  static constexpr uint32_t off_bias = off_a + kNTerms * a_term;  // b1[64] b2[64] bh[16]
  static constexpr uint32_t off_bar = off_bias + 144 * 4;
  static constexpr uint32_t bytes = off_bar + 128;
  static constexpr size_t launch_bytes = bytes + 1024;  // slack for the 1024-byte alignment
  static_assert(C == 32 || C == 64, "HexPlane channels");
  static_assert(off_w2 % 1024 == 0 && off_wh % 1024 == 0 && off_a % 1024 == 0 && w1_term % 1024 == 0 &&
                    wh_term % 1024 == 0,
                "swizzled operands need 1024-byte aligned buffers");
  static_assert(2 * (launch_bytes + 1024) <= 233472, "two CTAs per SM");
};

enum : int { kBarA1Full = 0, kBarAFree, kBarD1, kBarA2, kBarD2, kBarA3, kBarD3, kBarDrain, kMlpBars };

// Byte offset of the 16-byte chunk `c` of row `r` in a K-major operand with
// 64-byte rows (64-byte swizzle) or 128-byte rows (128-byte swizzle): the
// layout a TMA box with that swizzle lands in and the descriptors read.
__device__ __forceinline__ uint32_t chunk_off(int r, int c, int row_bytes) {
  return row_bytes == 64 ? (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4))
                         : (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// Three-term BF16 split of a pair (low half = first value).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  auto pack = [](float x, float y) -> uint32_t {
    const __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&v);
  };
  hi = pack(a, b);
  a -= __uint_as_float(hi << 16);
  b -= __uint_as_float(hi & 0xFFFF0000u);
  mid = pack(a, b);
  a -= __uint_as_float(mid << 16);
  b -= __uint_as_float(mid & 0xFFFF0000u);
  lo = pack(a, b);
}

// Eight consecutive values as one 16-byte chunk of each term's row.
__device__ __forceinline__ void store_split8(unsigned char* base, uint32_t term_bytes, uint32_t off, const float* x) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_pair(x[2 * i], x[2 * i + 1], h[i], m[i], l[i]);
  *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(base + term_bytes + off) = make_uint4(m[0], m[1], m[2], m[3]);
  *reinterpret_cast<uint4*>(base + 2 * term_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ bool mlp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint32_t* err) {
  if (*abort) return false;
  if (mbar_wait(bar, parity)) return true;
  *abort = 1;
  set_err(err, kErrTimeout);
  return false;
}

struct MlpArgs {
  int P, ntiles;
  const float *w1, *b1, *w2, *b2, *wh, *bh;
  float* dstate;  // [P][kDStride]: delta (11), 0, m1 (2 words), m2 (2 words)
  uint32_t* err;
};

template <int C>
__global__ void __launch_bounds__(kMlpThreads, 2)
    deform_mlp_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_mid,
                      const __grid_constant__ CUtensorMap tm_lo, const MlpArgs a) {
  using K = MlpCfg<C>;
  extern __shared__ unsigned char dsmem_raw[];
  const uint32_t raw_addr = smem_addr(dsmem_raw);
  unsigned char* sm = dsmem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sb = smem_addr(sm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + K::off_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + K::off_bar + kMlpBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + K::off_bar + kMlpBars * 8 + 4);
  float* s_bias = reinterpret_cast<float*>(sm + K::off_bias);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_mine = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int i = 0; i < kMlpBars; ++i) mbar_init(&bars[i], (i == kBarA2 || i == kBarA3) ? kMlpEpiWarps : 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  if (warp < kMlpEpiWarps) {
    // Weights as three BF16 terms in the operand layouts, one 16-byte chunk
    // (8 consecutive inputs of one output row) at a time; bias in FP32.
    // All of a thread's loads are issued before its first split.
    constexpr int n1 = kHidden * C / 8, n2 = kHidden * 64 / 8, nh = 16 * 64 / 8;
    constexpr int kPer = (n1 + n2 + nh + 32 * kMlpEpiWarps - 1) / (32 * kMlpEpiWarps);
    float xs[kPer][8];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int q = tid + j * 32 * kMlpEpiWarps;
      const float* src = nullptr;
      if (q < n1) src = a.w1 + (q / (C / 8)) * C + 8 * (q % (C / 8));
      else if (q < n1 + n2) src = a.w2 + ((q - n1) / 8) * kHidden + 8 * ((q - n1) % 8);  // W2[out][in]
      else if (q < n1 + n2 + nh && (q - n1 - n2) / 8 < kHeads) src = a.wh + ((q - n1 - n2) / 8) * kHidden + 8 * ((q - n1 - n2) % 8);
#pragma unroll
      for (int i = 0; i < 8; ++i) xs[j][i] = src ? __ldg(src + i) : 0.0f;  // Wh rows 11-15: zero
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int q = tid + j * 32 * kMlpEpiWarps;
      if (q < n1) store_split8(sm + K::off_w1, K::w1_term, chunk_off(q / (C / 8), q % (C / 8), K::row1), xs[j]);
      else if (q < n1 + n2) store_split8(sm + K::off_w2, K::w2_term, chunk_off((q - n1) / 8, (q - n1) % 8, 128), xs[j]);
      else if (q < n1 + n2 + nh)
        store_split8(sm + K::off_wh, K::wh_term, chunk_off((q - n1 - n2) / 8, (q - n1 - n2) % 8, 128), xs[j]);
    }
    for (int i = tid; i < 144; i += 32 * kMlpEpiWarps)
      s_bias[i] = i < 64 ? a.b1[i] : (i < 128 ? a.b2[i - 64] : (i - 128 < kHeads ? a.bh[i - 128] : 0.0f));
    fence_proxy_async();  // weight stores -> tensor-core reads
  }
  if (warp == kMlpWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(kMlpTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == kMlpWarpTma) {
    // ---------------- feature terms of each tile ----------------
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < n_mine; ++i) {
        if (i > 0 && !mlp_wait(&bars[kBarAFree], (i - 1) & 1, s_abort, a.err)) break;
        const int row0 = ((int)blockIdx.x + i * (int)gridDim.x) * kMlpBM;
        mbar_arrive_expect_tx(&bars[kBarA1Full], kNTerms * kMlpBM * K::row1);
        tma_2d(sm + K::off_a, &tm_hi, 0, row0, &bars[kBarA1Full]);
        tma_2d(sm + K::off_a + K::a_term, &tm_mid, 0, row0, &bars[kBarA1Full]);
        tma_2d(sm + K::off_a + 2 * K::a_term, &tm_lo, 0, row0, &bars[kBarA1Full]);
        issued = i + 1;
      }
      // The last copies issued land before the block leaves.
      if (issued > 0 && !mbar_wait(&bars[kBarA1Full], (issued - 1) & 1)) set_err(a.err, kErrTimeout);
    }
  } else if (warp == kMlpWarpMma) {
    // ---------------- tensor-core issue ----------------
    if (lane == 0) {
      const uint32_t s_a = sb + K::off_a;
      constexpr uint32_t id64 = mma_idesc(128, 64, 0, 0), id16 = mma_idesc(128, 16, 0, 0);
      // One layer: the six term products, K in 16-input steps (32 bytes of
      // a swizzled row).
      auto layer = [&](uint32_t col, uint32_t w_base, uint32_t w_term, uint32_t row_bytes, uint64_t layout, int ksteps,
                       uint32_t idesc) {
#pragma unroll
        for (int p = 0; p < 6; ++p)
          for (int k = 0; k < ksteps; ++k)
            mma_bf16(tmem + col, smem_desc(s_a + kPairA[p] * K::a_term + 32u * k, 16, 8 * row_bytes, layout),
                     smem_desc(w_base + kPairW[p] * w_term + 32u * k, 16, 8 * row_bytes, layout), idesc,
                     (p > 0 || k > 0) ? 1u : 0u);
      };
      for (int i = 0; i < n_mine; ++i) {
        const uint32_t ph = i & 1;
        if (!mlp_wait(&bars[kBarA1Full], ph, s_abort, a.err)) break;
        tc_fence_after();
        layer(kColD1, sb + K::off_w1, K::w1_term, K::row1, K::layout1, C / 16, id64);
        mma_commit(&bars[kBarD1]);
        if (!mlp_wait(&bars[kBarA2], ph, s_abort, a.err)) break;
        tc_fence_after();
        layer(kColD2, sb + K::off_w2, K::w2_term, 128, kLayout128B, 4, id64);
        mma_commit(&bars[kBarD2]);
        if (!mlp_wait(&bars[kBarA3], ph, s_abort, a.err)) break;
        tc_fence_after();
        layer(kColD3, sb + K::off_wh, K::wh_term, 128, kLayout128B, 4, id16);
        mma_commit(&bars[kBarD3]);
        mma_commit(&bars[kBarAFree]);
      }
      // Every issued product completes before tensor memory is freed.
      mma_commit(&bars[kBarDrain]);
      if (!mbar_wait(&bars[kBarDrain], 0)) set_err(a.err, kErrTimeout);
    }
  } else {
    // ---------------- epilogue: one Gaussian per thread ----------------
    const int r = warp * 32 + lane;  // tile row = tensor-memory lane
    const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
    unsigned char* s_a = sm + K::off_a;
    // Hidden layer from its accumulator: bias, ReLU, mask bits, and the
    // three terms of the next layer's input row.
    auto hidden = [&](uint32_t col, const float* bias, uint64_t& mask) {
      uint32_t v[32];
      mask = 0;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        tmem_ld32(t_row + col + 32 * half, v);
        tmem_wait_ld(v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int o = 32 * half + 8 * c + j;
            const float h = __uint_as_float(v[8 * c + j]) + bias[o];
            mask |= (uint64_t)(h > 0.0f) << o;
            x[j] = fmaxf(h, 0.0f);
          }
          store_split8(s_a, K::a_term, chunk_off(r, 4 * half + c, 128), x);
        }
      }
    };
    bool ok = true;
    for (int i = 0; ok && i < n_mine; ++i) {
      const uint32_t ph = i & 1;
      const int64_t g = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kMlpBM + r;
      uint64_t m1 = 0, m2 = 0;
      if (!mlp_wait(&bars[kBarD1], ph, s_abort, a.err)) break;
      tc_fence_after();
      hidden(kColD1, s_bias, m1);
      fence_proxy_async();  // operand stores -> tensor-core reads
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBarA2]);
      if (!mlp_wait(&bars[kBarD2], ph, s_abort, a.err)) break;
      tc_fence_after();
      hidden(kColD2, s_bias + 64, m2);
      fence_proxy_async();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBarA3]);
      if (!mlp_wait(&bars[kBarD3], ph, s_abort, a.err)) break;
      tc_fence_after();
      uint32_t v[32];
      tmem_ld16(t_row + kColD3, v);
      tmem_wait_ld(v);
      tc_fence_before();
      if (g < a.P) {
        float d[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) d[k] = k < kHeads ? __uint_as_float(v[k]) + s_bias[128 + k] : 0.0f;
        float4* o = reinterpret_cast<float4*>(a.dstate + g * kDStride);
        o[0] = make_float4(d[0], d[1], d[2], d[3]);
        o[1] = make_float4(d[4], d[5], d[6], d[7]);
        o[2] = make_float4(d[8], d[9], d[10], 0.0f);
        reinterpret_cast<uint4*>(o)[3] =
            make_uint4((uint32_t)m1, (uint32_t)(m1 >> 32), (uint32_t)m2, (uint32_t)(m2 >> 32));
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == kMlpWarpMma) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpTmemCols) : "memory");
  }
}

// Reverse of the MLP for the mean gradient (the offsets' gradient dd, 11
// values, back to the HexPlane feature): with the forward's unit masks m1,
// m2,
//   g2 = m2 . (Wh^T dd),  d1 = m1 . (W2^T g2),  df = W1^T d1,
// as three tensor-core layers of the same three-term form (K = 16 padded to
// 32, then 64 and 64; N = 64, 64 and C).  The epilogue warps write each
// tile's dd terms themselves (no TMA) and apply the masks between layers;
// df goes to a [P][C] FP32 array for the HexPlane reverse.
struct MlpBwdArgs {
  int P, ntiles;
  const float *w1, *w2, *wh;
  const float* ddstate;  // [P][12]: dd (11), active flag
  const float* dstate;   // [P][kDStride]: the masks in words 12-15
  float* df;             // [P][C]
  uint32_t* err;
};

template <int C>
struct MlpBwdCfg {
  static constexpr uint32_t b1_term = kHidden * 64;   // Wh^T [64][32] (K padded to 32: 64-byte rows)
  static constexpr uint32_t b2_term = kHidden * 128;  // W2^T [64][64]
  static constexpr uint32_t b3_term = C * 128;        // W1^T [C][64]
  static constexpr uint32_t a_term = kMlpBM * 128;
  static constexpr uint32_t off_b1 = 0;
  static constexpr uint32_t off_b2 = off_b1 + kNTerms * b1_term;
  static constexpr uint32_t off_b3 = off_b2 + kNTerms * b2_term;
  static constexpr uint32_t off_a = off_b3 + kNTerms * b3_term;
  static constexpr uint32_t off_bar = off_a + kNTerms * a_term;
  static constexpr uint32_t bytes = off_bar + 128;
  static constexpr size_t launch_bytes = bytes + 1024;
  static_assert(off_b2 % 1024 == 0 && off_b3 % 1024 == 0 && off_a % 1024 == 0, "1024-byte aligned operands");
  static_assert(2 * (launch_bytes + 1024) <= 233472, "two CTAs per SM");
};

enum : int { kBwA0 = 0, kBwD1, kBwA2, kBwD2, kBwA3, kBwD3, kBwDrain, kBwBars };
constexpr int kMlpBwdThreads = 32 * 5;  // 4 epilogue warps + the MMA warp

template <int C>
__global__ void __launch_bounds__(kMlpBwdThreads, 2) deform_mlp_bwd_kernel(const MlpBwdArgs a) {
  using K = MlpBwdCfg<C>;
  extern __shared__ unsigned char dsmem_raw[];
  const uint32_t raw_addr = smem_addr(dsmem_raw);
  unsigned char* sm = dsmem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sb = smem_addr(sm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + K::off_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + K::off_bar + kBwBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + K::off_bar + kBwBars * 8 + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_mine = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int i = 0; i < kBwBars; ++i) mbar_init(&bars[i], (i == kBwA0 || i == kBwA2 || i == kBwA3) ? kMlpEpiWarps : 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  if (warp < kMlpEpiWarps) {
    // Transposed weights as three BF16 terms, one 16-byte chunk (8
    // consecutive K values of one output row) at a time; all of a thread's
    // loads issued before its first split.
    constexpr int n1 = kHidden * 4, n2 = kHidden * 8, n3 = C * 8;
    constexpr int kPer = (n1 + n2 + n3 + 32 * kMlpEpiWarps - 1) / (32 * kMlpEpiWarps);
    float xs[kPer][8];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int q = tid + j * 32 * kMlpEpiWarps;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float x = 0.0f;
        if (q < n1) {
          const int o = q / 4, k = 8 * (q % 4) + i;  // Wh^T[o][k] = Wh[k][o], k < 11
          if (k < kHeads) x = __ldg(a.wh + k * kHidden + o);
        } else if (q < n1 + n2) {
          const int o1 = (q - n1) / 8, o = 8 * ((q - n1) % 8) + i;  // W2^T[o1][o] = W2[o][o1]
          x = __ldg(a.w2 + o * kHidden + o1);
        } else if (q < n1 + n2 + n3) {
          const int c = (q - n1 - n2) / 8, o1 = 8 * ((q - n1 - n2) % 8) + i;  // W1^T[c][o1] = W1[o1][c]
          x = __ldg(a.w1 + o1 * C + c);
        }
        xs[j][i] = x;
      }
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int q = tid + j * 32 * kMlpEpiWarps;
      if (q < n1) store_split8(sm + K::off_b1, K::b1_term, chunk_off(q / 4, q % 4, 64), xs[j]);
      else if (q < n1 + n2) store_split8(sm + K::off_b2, K::b2_term, chunk_off((q - n1) / 8, (q - n1) % 8, 128), xs[j]);
      else if (q < n1 + n2 + n3)
        store_split8(sm + K::off_b3, K::b3_term, chunk_off((q - n1 - n2) / 8, (q - n1 - n2) % 8, 128), xs[j]);
    }
    fence_proxy_async();
  }
  if (warp == kMlpEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(kMlpTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == kMlpEpiWarps) {
    // ---------------- tensor-core issue ----------------
    if (lane == 0) {
      const uint32_t s_a = sb + K::off_a;
      constexpr uint32_t id64 = mma_idesc(128, 64, 0, 0), idc = mma_idesc(128, C, 0, 0);
      auto layer = [&](uint32_t col, uint32_t b_base, uint32_t b_term, uint32_t row_bytes, uint64_t layout, int ksteps,
                       uint32_t idesc) {
#pragma unroll
        for (int p = 0; p < 6; ++p)
          for (int k = 0; k < ksteps; ++k)
            mma_bf16(tmem + col, smem_desc(s_a + kPairA[p] * K::a_term + 32u * k, 16, 8 * row_bytes, layout),
                     smem_desc(b_base + kPairW[p] * b_term + 32u * k, 16, 8 * row_bytes, layout), idesc,
                     (p > 0 || k > 0) ? 1u : 0u);
      };
      for (int i = 0; i < n_mine; ++i) {
        const uint32_t ph = i & 1;
        if (!mlp_wait(&bars[kBwA0], ph, s_abort, a.err)) break;
        tc_fence_after();
        layer(kColD1, sb + K::off_b1, K::b1_term, 64, kLayout64B, 2, id64);
        mma_commit(&bars[kBwD1]);
        if (!mlp_wait(&bars[kBwA2], ph, s_abort, a.err)) break;
        tc_fence_after();
        layer(kColD2, sb + K::off_b2, K::b2_term, 128, kLayout128B, 4, id64);
        mma_commit(&bars[kBwD2]);
        if (!mlp_wait(&bars[kBwA3], ph, s_abort, a.err)) break;
        tc_fence_after();
        layer(kColD3, sb + K::off_b3, K::b3_term, 128, kLayout128B, 4, idc);
        mma_commit(&bars[kBwD3]);
      }
      mma_commit(&bars[kBwDrain]);
      if (!mbar_wait(&bars[kBwDrain], 0)) set_err(a.err, kErrTimeout);
    }
  } else {
    // ---------------- epilogue: one Gaussian per thread ----------------
    const int r = warp * 32 + lane;
    const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
    unsigned char* s_a = sm + K::off_a;
    // A masked 64-wide layer output as the three terms of the next input.
    auto masked = [&](uint32_t col, uint64_t mask) {
      uint32_t v[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        tmem_ld32(t_row + col + 32 * half, v);
        tmem_wait_ld(v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int o = 32 * half + 8 * c + j;
            x[j] = ((mask >> o) & 1ull) ? __uint_as_float(v[8 * c + j]) : 0.0f;
          }
          store_split8(s_a, K::a_term, chunk_off(r, 4 * half + c, 128), x);
        }
      }
    };
    // This row's dd (zero for an inactive Gaussian or a row past P) and unit
    // masks of tile i, loaded one tile ahead so that their latency overlaps
    // the previous tile's layers.
    float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0, n2 = n0;
    uint4 nmk = make_uint4(0u, 0u, 0u, 0u);
    auto load_in = [&](int i) {
      const int64_t g = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kMlpBM + r;
      n0 = n1 = n2 = make_float4(0.f, 0.f, 0.f, 0.f);
      nmk = make_uint4(0u, 0u, 0u, 0u);
      if (g < a.P) {
        const float4* dd4 = reinterpret_cast<const float4*>(a.ddstate + g * 12);
        n0 = dd4[0]; n1 = dd4[1]; n2 = dd4[2];
        nmk = reinterpret_cast<const uint4*>(a.dstate + g * kDStride)[3];
      }
    };
    if (n_mine > 0) load_in(0);
    bool ok = true;
    for (int i = 0; ok && i < n_mine; ++i) {
      const uint32_t ph = i & 1;
      const int64_t g = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kMlpBM + r;
      const float4 q0 = n0, q1 = n1, q2 = n2;
      const uint4 mk = nmk;
      if (i + 1 < n_mine) load_in(i + 1);
      // dd as the first layer's input (the previous tile's products are
      // complete: its D3 was waited for), the masks for the later layers.
      float x[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) x[k] = 0.0f;
      uint64_t m1 = 0, m2 = 0;
      if (q2.w != 0.0f) {
        x[0] = q0.x; x[1] = q0.y; x[2] = q0.z; x[3] = q0.w; x[4] = q1.x; x[5] = q1.y;
        x[6] = q1.z; x[7] = q1.w; x[8] = q2.x; x[9] = q2.y; x[10] = q2.z;
        m1 = (uint64_t)mk.x | ((uint64_t)mk.y << 32);
        m2 = (uint64_t)mk.z | ((uint64_t)mk.w << 32);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) store_split8(s_a, K::a_term, chunk_off(r, c, 64), x + 8 * c);
      fence_proxy_async();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBwA0]);
      if (!mlp_wait(&bars[kBwD1], ph, s_abort, a.err)) break;
      tc_fence_after();
      masked(kColD1, m2);  // g2
      fence_proxy_async();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBwA2]);
      if (!mlp_wait(&bars[kBwD2], ph, s_abort, a.err)) break;
      tc_fence_after();
      masked(kColD2, m1);  // d1
      fence_proxy_async();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBwA3]);
      if (!mlp_wait(&bars[kBwD3], ph, s_abort, a.err)) break;
      tc_fence_after();
#pragma unroll
      for (int part = 0; part < C / 32; ++part) {
        uint32_t v[32];
        tmem_ld32(t_row + kColD3 + 32 * part, v);
        tmem_wait_ld(v);
        if (g < a.P) {
          float4* o = reinterpret_cast<float4*>(a.df + g * C + 32 * part);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                               __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
        }
      }
      tc_fence_before();
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == kMlpEpiWarps) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpTmemCols) : "memory");
  }
}

template <int C>
cudaError_t launch_mlp_bwd_t(const GaussArgs& g, const GaussBwdArgs& b, float* df, cudaStream_t st) {
  using K = MlpBwdCfg<C>;
  MlpBwdArgs a{};
  a.P = g.P;
  a.ntiles = (g.P + kMlpBM - 1) / kMlpBM;
  a.w1 = g.w1; a.w2 = g.w2; a.wh = g.wh;
  a.ddstate = b.ddstate;
  a.dstate = g.dstate;
  a.df = df;
  a.err = g.err;
  const int sms = num_sms();
  int grid = 2 * (sms > 0 ? sms : 1);
  if (grid > a.ntiles) grid = a.ntiles;
  auto k = deform_mlp_bwd_kernel<C>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::launch_bytes);
  if (e != cudaSuccess) return e;
  k<<<grid, kMlpBwdThreads, K::launch_bytes, st>>>(a);
  return cudaGetLastError();
}

template <int C>
cudaError_t launch_mlp_t(const GaussArgs& g, cudaStream_t st) {
  using K = MlpCfg<C>;
  const size_t term = (size_t)g.P * C;  // bf16 elements of one term array
  CUtensorMap m[3];
  const CUtensorMapSwizzle swz = C == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  // At least one whole tile of rows (the region has 128 rows of slack): the
  // rows past P that a small P's tile reads are never stored.
  const uint64_t rows = g.P > kMlpBM ? (uint64_t)g.P : (uint64_t)kMlpBM;
  for (int t = 0; t < 3; ++t)
    if (!make_map(&m[t], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.fsplit + t * term, C, rows, C, kMlpBM, swz))
      return cudaErrorInvalidValue;
  MlpArgs a{};
  a.P = g.P;
  a.ntiles = (g.P + kMlpBM - 1) / kMlpBM;
  a.w1 = g.w1; a.b1 = g.b1; a.w2 = g.w2; a.b2 = g.b2; a.wh = g.wh; a.bh = g.bh;
  a.dstate = g.dstate;
  a.err = g.err;
  const int sms = num_sms();
  int grid = 2 * (sms > 0 ? sms : 1);
  if (grid > a.ntiles) grid = a.ntiles;
  auto k = deform_mlp_kernel<C>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::launch_bytes);
  if (e != cudaSuccess) return e;
  k<<<grid, kMlpThreads, K::launch_bytes, st>>>(m[0], m[1], m[2], a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_deform_mlp_bwd(const GaussArgs& g, const GaussBwdArgs& b, float* df, cudaStream_t st) {
  if (g.P <= 0 || !g.has_deform) return cudaSuccess;
  if (!df || !g.dstate || !b.ddstate) return cudaErrorInvalidValue;
  if (g.C == 32) return launch_mlp_bwd_t<32>(g, b, df, st);
  if (g.C == 64) return launch_mlp_bwd_t<64>(g, b, df, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_deform_mlp(const GaussArgs& g, cudaStream_t st) {
  if (g.P <= 0 || !g.has_deform) return cudaSuccess;
  if (!g.fsplit || !g.dstate) return cudaErrorInvalidValue;
  if (g.C == 32) return launch_mlp_t<32>(g, st);
  if (g.C == 64) return launch_mlp_t<64>(g, st);
  return cudaErrorInvalidValue;
}

}  // namespace fe
