// Semantic decoder of the rendered feature map (Sec. 3.3, Eq. 9-10): a 1x1
// convolution from D to 256 channels, out[p][c] = sum_d F[p][d] W[c][d] + b[c],
// on the 5th-generation tensor cores (tcgen05, BF16 operands, FP32
// accumulators in tensor memory), optionally fused with the L1 feature loss
// of Eq. 10 and its reverse pass.
//
// One persistent CTA per SM walks 128-pixel tiles.  Warp roles:
//   warps 0-3  epilogue: tensor memory -> registers (one pixel row per
//              thread), bias, L1 against the staged target, sign -> S tile
//   warp 4     producer: TMA tile loads of W (once), F tiles and targets
//   warp 5     tensor-core issue (one thread) and tensor-memory allocation
// Per tile the MMAs are
//   acc[p][c]  = sum_d F[p][d] W[c][d]                   (K = D)
//   dF[p][d]   = sum_c S[p][c] W[c][d]                   (K = 256)
//   dW[c][d]  += sum_p S[p][c] F[p][d]                   (K = 128, two M halves)
//   db[c]     += sum_p S[p][c]                           (B = all-ones operand)
// with S = sign(out - target) in {-1, 0, 1} (exact in BF16).  The scale
// (1/HW for Eq. 10) is applied in FP32 afterwards.  dW and db stay in tensor
// memory for the whole CTA and are summed over CTAs in a fixed order by a
// second kernel: no floating-point atomics.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"

namespace fe {

namespace {

constexpr int kDecN = 256;        // output channels
constexpr int kDecBM = 128;       // pixels per tile (MMA M)
constexpr int kDecThreads = 192;  // 4 epilogue warps, producer warp, MMA warp
constexpr int kTStages = 4;       // target ring depth
constexpr uint32_t kBoxBytes = 16384;  // one target box: 128 rows x 128 bytes
constexpr uint32_t kPanel = 16384;     // one S panel: 128 rows x 64 bf16 channels
constexpr uint32_t kTmemCols = 512;
// Tensor-memory columns of the accumulators.
constexpr uint32_t kColAcc = 0, kColDF = 256, kColDW = 320, kColDB = 448;

enum DecMode : int { kDecForward = 0, kDecL1Bf16 = 1, kDecL1F32 = 2 };

// Shared-memory descriptor layouts (bits 61-63).
constexpr uint64_t kLayoutNone = 0, kLayout128B = 2, kLayout64B = 4;

template <int D>
struct DecCfg {
  static constexpr uint32_t row_bytes = D * 2;  // one F / W row in bf16
  static constexpr uint64_t layout = D == 64 ? kLayout128B : kLayout64B;
  static constexpr uint32_t sbo = 8 * row_bytes;  // stride of 8-row groups
  static constexpr uint32_t w_bytes = kDecN * row_bytes;
  static constexpr uint32_t f_bytes = kDecBM * row_bytes;
  static constexpr uint32_t off_w = 0;
  static constexpr uint32_t off_f = off_w + w_bytes;      // 2 stages
  static constexpr uint32_t off_s = off_f + 2 * f_bytes;  // 4 panels
  static constexpr uint32_t off_t = off_s + 4 * kPanel;   // target ring
  static constexpr uint32_t off_ones = off_t + kTStages * kBoxBytes;
  static constexpr uint32_t off_bias = off_ones + 4096;
  static constexpr uint32_t off_bar = off_bias + kDecN * 4;
  static constexpr uint32_t bytes = off_bar + 256;
  static constexpr size_t launch_bytes = bytes + 1024;  // slack for 1024-byte alignment
  static_assert(D == 32 || D == 64, "decoder feature width");
  static_assert(off_f % 1024 == 0 && off_s % 1024 == 0 && off_t % 1024 == 0 && off_ones % 1024 == 0,
                "swizzled operands need 1024-byte aligned buffers");
};

struct DecArgs {
  int64_t HW;
  int ntiles;
  const float* bias;
  float* out;        // forward: [HW, 256]
  float scale;       // L1: loss and gradient scale
  float* d_feat;     // [HW, D]
  float* part_loss;  // [ncta]
  float* part_dw;    // [ncta][256][D]
  float* part_db;    // [ncta][256]
  uint32_t* err;
};

// Barrier slots (8 bytes each) after off_bar.
enum : int {
  kBarW = 0, kBarFFull = 1, kBarFEmpty = 3, kBarTFull = 5, kBarTEmpty = 9, kBarAccFull = 13, kBarAccEmpty = 14,
  kBarSFull = 15, kBarBwd = 16, kBarDrain = 17, kNumBars = 18
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint64_t layout) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (layout << 61);
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 accumulator.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every tensor-core operation issued so far completes.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes; register i of
// lane l holds column col + i of row (lane base + l).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld1(uint32_t taddr, uint32_t& v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ bool dec_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint32_t* err) {
  if (*abort) return false;
  if (mbar_wait(bar, parity)) return true;
  *abort = 1;
  set_err(err, kErrTimeout);
  return false;
}

template <int D, int MODE>
__global__ void __launch_bounds__(kDecThreads, 1)
    decoder_kernel(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_w,
                   const __grid_constant__ CUtensorMap tm_t, const DecArgs a) {
  using C = DecCfg<D>;
  constexpr bool kL1 = MODE != kDecForward;
  constexpr int kBoxCh = MODE == kDecL1F32 ? 32 : 64;  // target channels per box
  constexpr int kNumBoxes = kDecN / kBoxCh;
  extern __shared__ unsigned char dsmem_raw[];
  // Swizzled operands are addressed by shared-memory address bits: align the
  // working base to 1024 bytes.
  const uint32_t raw_addr = smem_addr(dsmem_raw);
  unsigned char* sm = dsmem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sb = smem_addr(sm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::off_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + C::off_bar + kNumBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + C::off_bar + kNumBars * 8 + 4);
  float* s_red = reinterpret_cast<float*>(sm + C::off_bar + kNumBars * 8 + 8);  // [4]
  float* s_bias = reinterpret_cast<float*>(sm + C::off_bias);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(&bars[kBarW], 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bars[kBarFFull + s], 1);
      mbar_init(&bars[kBarFEmpty + s], 1);
    }
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(&bars[kBarTFull + s], 1);
      mbar_init(&bars[kBarTEmpty + s], 4);
    }
    mbar_init(&bars[kBarAccFull], 1);
    mbar_init(&bars[kBarAccEmpty], 4);
    mbar_init(&bars[kBarSFull], 4);
    mbar_init(&bars[kBarBwd], 1);
    mbar_init(&bars[kBarDrain], 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  if (warp < 4) {
    // All-ones B operand of the bias-gradient product, and the bias.
    uint4* ones = reinterpret_cast<uint4*>(sm + C::off_ones);
    for (int i = tid; i < 4096 / 16; i += 128) ones[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    for (int i = tid; i < kDecN; i += 128) s_bias[i] = a.bias[i];
    fence_proxy_async();
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 4) {
    // ---------------- producer ----------------
    if (lane == 0) {
      uint32_t f_uses = 0, t_uses = 0;
      mbar_arrive_expect_tx(&bars[kBarW], C::w_bytes);
      tma_2d(sm + C::off_w, &tm_w, 0, 0, &bars[kBarW]);
      uint32_t i = 0;
      for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
        const int f = i & 1;
        if (!dec_wait(&bars[kBarFEmpty + f], ((i >> 1) & 1) ^ 1, s_abort, a.err)) break;
        mbar_arrive_expect_tx(&bars[kBarFFull + f], C::f_bytes);
        tma_2d(sm + C::off_f + f * C::f_bytes, &tm_f, 0, tile * kDecBM, &bars[kBarFFull + f]);
        ++f_uses;
        if (kL1) {
          bool ok = true;
          for (int b = 0; b < kNumBoxes; ++b, ++t_uses) {
            const uint32_t r = t_uses % kTStages;
            if (!dec_wait(&bars[kBarTEmpty + r], ((t_uses / kTStages) & 1) ^ 1, s_abort, a.err)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&bars[kBarTFull + r], kBoxBytes);
            tma_2d(sm + C::off_t + r * kBoxBytes, &tm_t, b * kBoxCh, tile * kDecBM, &bars[kBarTFull + r]);
          }
          if (!ok) break;
        }
      }
      // Every copy issued must have landed before the block leaves.
      for (uint32_t u = f_uses > 2 ? f_uses - 2 : 0; u < f_uses; ++u)
        if (!mbar_wait(&bars[kBarFFull + (u & 1)], (u >> 1) & 1)) set_err(a.err, kErrTimeout);
      for (uint32_t u = t_uses > kTStages ? t_uses - kTStages : 0; u < t_uses; ++u)
        if (!mbar_wait(&bars[kBarTFull + u % kTStages], (u / kTStages) & 1)) set_err(a.err, kErrTimeout);
      if (!mbar_wait(&bars[kBarW], 0)) set_err(a.err, kErrTimeout);
    }
  } else if (warp == 5) {
    // ---------------- tensor-core issue ----------------
    if (lane == 0) {
      const uint32_t s_w = sb + C::off_w, s_s = sb + C::off_s, s_ones = sb + C::off_ones;
      constexpr uint32_t id_fwd = mma_idesc(128, kDecN, 0, 0);
      constexpr uint32_t id_df = mma_idesc(128, D, 0, 1);
      constexpr uint32_t id_dw = mma_idesc(128, D, 1, 1);
      constexpr uint32_t id_db = mma_idesc(128, 16, 1, 1);
      bool ok = dec_wait(&bars[kBarW], 0, s_abort, a.err);
      uint32_t i = 0;
      for (int tile = blockIdx.x; ok && tile < a.ntiles; tile += gridDim.x, ++i) {
        const int f = i & 1;
        const uint32_t s_f = sb + C::off_f + f * C::f_bytes;
        if (!dec_wait(&bars[kBarFFull + f], (i >> 1) & 1, s_abort, a.err)) break;
        if (i > 0 && !dec_wait(&bars[kBarAccEmpty], (i - 1) & 1, s_abort, a.err)) break;
        tc_fence_after();
        // acc = F W^T: A = F (K-major), B = W (K-major); 16 channels of K
        // are 32 bytes along each swizzled row.
#pragma unroll
        for (int k = 0; k < D / 16; ++k)
          mma_bf16(tmem + kColAcc, smem_desc(s_f + 32 * k, 16, C::sbo, C::layout),
                   smem_desc(s_w + 32 * k, 16, C::sbo, C::layout), id_fwd, k > 0);
        mma_commit(&bars[kBarAccFull]);
        if (!kL1) {
          mma_commit(&bars[kBarFEmpty + f]);
          continue;
        }
        if (!dec_wait(&bars[kBarSFull], i & 1, s_abort, a.err)) break;
        tc_fence_after();
        // dF = S W: A = S (K-major, 128B swizzle, 64-channel panels),
        // B = W read MN-major (K = channel rows, N = D along each row).
#pragma unroll
        for (int k = 0; k < kDecN / 16; ++k)
          mma_bf16(tmem + kColDF, smem_desc(s_s + (k >> 2) * kPanel + (k & 3) * 32, 16, 1024, kLayout128B),
                   smem_desc(s_w + k * 16 * C::row_bytes, 16, C::sbo, C::layout), id_df, k > 0);
        // dW += S^T F and db += S^T 1: A = S read MN-major (M = channels,
        // two 64-channel panels per half), B = F read MN-major / all ones.
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int k = 0; k < kDecBM / 16; ++k) {
            const uint64_t ad = smem_desc(s_s + h * 2 * kPanel + k * 2048, kPanel, 1024, kLayout128B);
            const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
            mma_bf16(tmem + kColDW + 64 * h, ad, smem_desc(s_f + k * 16 * C::row_bytes, 16, C::sbo, C::layout),
                     id_dw, acc);
            mma_bf16(tmem + kColDB + 16 * h, ad, smem_desc(s_ones + k * 512, 256, 128, kLayoutNone), id_db, acc);
          }
        }
        mma_commit(&bars[kBarBwd]);
        mma_commit(&bars[kBarFEmpty + f]);
      }
      // Drain: every issued tensor-core operation completes before the
      // accumulators are read or freed.
      mma_commit(&bars[kBarDrain]);
      if (!mbar_wait(&bars[kBarDrain], 0)) set_err(a.err, kErrTimeout);
    }
  } else {
    // ---------------- epilogue: warps 0-3, one pixel row per thread ----------------
    const int r = tid;  // tile row = tensor-memory lane
    const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
    float loss = 0.0f;
    uint32_t t_uses = 0;
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
      if (!dec_wait(&bars[kBarAccFull], i & 1, s_abort, a.err)) break;
      tc_fence_after();
      const int64_t p = (int64_t)tile * kDecBM + r;
      const bool valid = p < a.HW;
      bool ok = true;
#pragma unroll 1
      for (int ch = 0; ch < kDecN / 32; ++ch) {
        uint32_t v[32];
        tmem_ld32(t_row + kColAcc + 32 * ch, v);
        tmem_wait_ld();
        if (!kL1) {
          if (valid) {
            float4* o = reinterpret_cast<float4*>(a.out + p * kDecN + 32 * ch);
#pragma unroll
            for (int q = 0; q < 8; ++q)
              o[q] = make_float4(__uint_as_float(v[4 * q]) + s_bias[32 * ch + 4 * q],
                                 __uint_as_float(v[4 * q + 1]) + s_bias[32 * ch + 4 * q + 1],
                                 __uint_as_float(v[4 * q + 2]) + s_bias[32 * ch + 4 * q + 2],
                                 __uint_as_float(v[4 * q + 3]) + s_bias[32 * ch + 4 * q + 3]);
          }
          continue;
        }
        const bool first = MODE == kDecL1F32 || (ch & 1) == 0;
        const bool last = MODE == kDecL1F32 || (ch & 1) == 1;
        const uint32_t slot = t_uses % kTStages;
        if (first && !dec_wait(&bars[kBarTFull + slot], (t_uses / kTStages) & 1, s_abort, a.err)) {
          ok = false;
          break;
        }
        // Target row r of the staged box (128-byte rows, 16-byte chunks
        // permuted by row & 7).
        const unsigned char* trow = sm + C::off_t + slot * kBoxBytes + r * 128;
        float t[32];
        if (MODE == kDecL1F32) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 x = *reinterpret_cast<const float4*>(trow + ((q ^ (r & 7)) << 4));
            t[4 * q] = x.x; t[4 * q + 1] = x.y; t[4 * q + 2] = x.z; t[4 * q + 3] = x.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 x = *reinterpret_cast<const uint4*>(trow + (((4 * (ch & 1) + q) ^ (r & 7)) << 4));
            const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              t[8 * q + 2 * e] = __uint_as_float(w4[e] << 16);
              t[8 * q + 2 * e + 1] = __uint_as_float(w4[e] & 0xFFFF0000u);
            }
          }
        }
        uint32_t sg[16];
        float part = 0.0f;
#pragma unroll
        for (int c2 = 0; c2 < 16; ++c2) {
          uint32_t h2 = 0;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int c = 2 * c2 + e;
            const float d = __uint_as_float(v[c]) + s_bias[32 * ch + c] - t[c];
            part += fabsf(d);
            // sign(d) in bf16: +-1.0 (0x3F80 | sign bit), 0 for d == 0.
            const uint32_t s16 = d != 0.0f ? (((__float_as_uint(d) >> 16) & 0x8000u) | 0x3F80u) : 0u;
            h2 |= (valid ? s16 : 0u) << (16 * e);
          }
          sg[c2] = h2;
        }
        if (valid) loss += part;
        // S row r, channels 32ch .. 32ch+31: panel ch/2, logical chunks
        // 4 (ch & 1) .. +3 of the 128-byte row, permuted by row & 7.
        unsigned char* srow = sm + C::off_s + (ch >> 1) * kPanel + r * 128;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(srow + (((4 * (ch & 1) + q) ^ (r & 7)) << 4)) =
              make_uint4(sg[4 * q], sg[4 * q + 1], sg[4 * q + 2], sg[4 * q + 3]);
        if (last) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars[kBarTEmpty + slot]);
          ++t_uses;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBarAccEmpty]);
      if (!ok) break;
      if (!kL1) continue;
      fence_proxy_async();  // S stores -> tensor-core reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBarSFull]);
      if (!dec_wait(&bars[kBarBwd], i & 1, s_abort, a.err)) break;
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < D / 32; ++h) {
        uint32_t v[32];
        tmem_ld32(t_row + kColDF + 32 * h, v);
        tmem_wait_ld();
        if (valid) {
          float4* o = reinterpret_cast<float4*>(a.d_feat + p * D + 32 * h);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            o[q] = make_float4(a.scale * __uint_as_float(v[4 * q]), a.scale * __uint_as_float(v[4 * q + 1]),
                               a.scale * __uint_as_float(v[4 * q + 2]), a.scale * __uint_as_float(v[4 * q + 3]));
        }
      }
    }
    if (kL1) {
      // Per-CTA partials: dW rows and db of the channels of this lane, the
      // loss of this CTA (fixed-order sums).
      asm volatile("bar.sync 1, 128;" ::: "memory");  // epilogue warps only
      if (!*s_abort) {
        // The last backward barrier the epilogue waited on covers every
        // product of this CTA.
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = h * 128 + r;
#pragma unroll
          for (int q = 0; q < D / 32; ++q) {
            uint32_t v[32];
            tmem_ld32(t_row + kColDW + 64 * h + 32 * q, v);
            tmem_wait_ld();
            float4* o = reinterpret_cast<float4*>(a.part_dw + ((size_t)blockIdx.x * kDecN + c) * D + 32 * q);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                 __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
          }
          uint32_t vb;
          tmem_ld1(t_row + kColDB + 16 * h, vb);
          tmem_wait_ld();
          a.part_db[(size_t)blockIdx.x * kDecN + c] = __uint_as_float(vb);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
      if (lane == 0) s_red[warp] = loss;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid == 0) a.part_loss[blockIdx.x] = (s_red[0] + s_red[1]) + (s_red[2] + s_red[3]);
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Fixed-order sums of the per-CTA partials, scaled.
__global__ void decoder_reduce_kernel(int ncta, int D, float scale, const float* part_loss, const float* part_dw,
                                      const float* part_db, float* loss, float* d_weight, float* d_bias) {
  const int n_dw = kDecN * D;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_dw) {
    float s = 0.0f;
    for (int c = 0; c < ncta; ++c) s += part_dw[(size_t)c * n_dw + i];
    d_weight[i] = scale * s;
  } else if (i < n_dw + kDecN) {
    const int j = i - n_dw;
    float s = 0.0f;
    for (int c = 0; c < ncta; ++c) s += part_db[(size_t)c * kDecN + j];
    d_bias[j] = scale * s;
  } else if (i == n_dw + kDecN) {
    float s = 0.0f;
    for (int c = 0; c < ncta; ++c) s += part_loss[c];
    *loss = scale * s;
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 2-D row-major tensor map: `rows` rows of `cols` elements, box of
// box_cols x box_rows elements.
bool make_map(CUtensorMap* m, CUtensorMapDataType dt, int esize, const void* base, uint64_t cols, uint64_t rows,
              uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * (uint64_t)esize};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return n;
}

template <int D, int MODE>
cudaError_t launch_dec(const CUtensorMap& mf, const CUtensorMap& mw, const CUtensorMap& mt, const DecArgs& a, int grid,
                       cudaStream_t st) {
  auto k = decoder_kernel<D, MODE>;
  const size_t smem = DecCfg<D>::launch_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kDecThreads, smem, st>>>(mf, mw, mt, a);
  return cudaGetLastError();
}

// Workspace: 256-byte header (error bits), then per-CTA partial loss, dW, db.
struct DecLayout {
  int ncta;
  size_t loss, dw, db, total;
};

DecLayout dec_layout(int64_t HW, int D) {
  DecLayout L{};
  const int64_t ntiles = (HW + kDecBM - 1) / kDecBM;
  const int sms = num_sms();
  L.ncta = (int)(ntiles < sms ? ntiles : sms);
  if (L.ncta < 1) L.ncta = 1;
  L.loss = 256;
  L.dw = align_up(L.loss + (size_t)L.ncta * 4, 256);
  L.db = align_up(L.dw + (size_t)L.ncta * kDecN * D * 4, 256);
  L.total = align_up(L.db + (size_t)L.ncta * kDecN * 4, 256);
  return L;
}

bool aligned16p(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fe_status dec_check(const fe_decoder_args* a) {
  if (!a || a->HW < 0 || a->HW > (int64_t)kDecBM * ((1ll << 31) / kDecBM - 1)) return FE_ERR_INVALID_ARG;
  if (a->D != 32 && a->D != 64) return FE_ERR_UNSUPPORTED;
  if (!a->weight || !a->bias || !aligned16p(a->weight)) return FE_ERR_INVALID_ARG;
  if (a->HW > 0 && (!a->feat || !aligned16p(a->feat))) return FE_ERR_INVALID_ARG;
  return FE_OK;
}

template <int MODE>
cudaError_t dispatch(int D, const CUtensorMap& mf, const CUtensorMap& mw, const CUtensorMap& mt, const DecArgs& a,
                     int grid, cudaStream_t st) {
  return D == 32 ? launch_dec<32, MODE>(mf, mw, mt, a, grid, st) : launch_dec<64, MODE>(mf, mw, mt, a, grid, st);
}

}  // namespace

}  // namespace fe

using namespace fe;

extern "C" {

size_t fe_decoder_workspace_size(int64_t HW, int D) {
  if (HW < 0 || (D != 32 && D != 64)) return 0;
  return dec_layout(HW, D).total;
}

fe_status fe_decode_forward(const fe_decoder_args* a, float* out, void* workspace, size_t workspace_bytes,
                            void* stream) {
  fe_status s = dec_check(a);
  if (s != FE_OK) return s;
  if (!workspace || !out || !aligned16p(out)) return FE_ERR_INVALID_ARG;
  const DecLayout L = dec_layout(a->HW, a->D);
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(workspace, 0, 256, st) != cudaSuccess) return FE_ERR_CUDA;
  if (a->HW == 0) return FE_OK;
  CUtensorMap mf, mw;
  const CUtensorMapSwizzle swz = a->D == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (!make_map(&mf, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a->feat, a->D, a->HW, a->D, kDecBM, swz) ||
      !make_map(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a->weight, a->D, kDecN, a->D, kDecN, swz))
    return FE_ERR_CUDA;
  DecArgs d{};
  d.HW = a->HW;
  d.ntiles = (int)((a->HW + kDecBM - 1) / kDecBM);
  d.bias = a->bias;
  d.out = out;
  d.err = static_cast<uint32_t*>(workspace);
  return dispatch<kDecForward>(a->D, mf, mw, mw, d, L.ncta, st) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

fe_status fe_decode_l1(const fe_decoder_args* a, const void* target, int target_bf16, float scale, float* loss,
                       float* d_feat, float* d_weight, float* d_bias, void* workspace, size_t workspace_bytes,
                       void* stream) {
  fe_status s = dec_check(a);
  if (s != FE_OK) return s;
  if (!workspace || !loss || !d_weight || !d_bias) return FE_ERR_INVALID_ARG;
  if (a->HW > 0 && (!target || !aligned16p(target) || !d_feat || !aligned16p(d_feat))) return FE_ERR_INVALID_ARG;
  const DecLayout L = dec_layout(a->HW, a->D);
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (cudaMemsetAsync(workspace, 0, 256, st) != cudaSuccess) return FE_ERR_CUDA;
  if (a->HW == 0) {
    if (cudaMemsetAsync(loss, 0, 4, st) != cudaSuccess ||
        cudaMemsetAsync(d_weight, 0, (size_t)kDecN * a->D * 4, st) != cudaSuccess ||
        cudaMemsetAsync(d_bias, 0, (size_t)kDecN * 4, st) != cudaSuccess)
      return FE_ERR_CUDA;
    return FE_OK;
  }
  CUtensorMap mf, mw, mt;
  const CUtensorMapSwizzle swz = a->D == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  const bool tb = target_bf16 != 0;
  if (!make_map(&mf, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a->feat, a->D, a->HW, a->D, kDecBM, swz) ||
      !make_map(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a->weight, a->D, kDecN, a->D, kDecN, swz) ||
      !make_map(&mt, tb ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, tb ? 2 : 4, target,
                kDecN, a->HW, tb ? 64 : 32, kDecBM, CU_TENSOR_MAP_SWIZZLE_128B))
    return FE_ERR_CUDA;
  DecArgs d{};
  d.HW = a->HW;
  d.ntiles = (int)((a->HW + kDecBM - 1) / kDecBM);
  d.bias = a->bias;
  d.scale = scale;
  d.d_feat = d_feat;
  d.part_loss = reinterpret_cast<float*>(ws + L.loss);
  d.part_dw = reinterpret_cast<float*>(ws + L.dw);
  d.part_db = reinterpret_cast<float*>(ws + L.db);
  d.err = static_cast<uint32_t*>(workspace);
  const cudaError_t e = tb ? dispatch<kDecL1Bf16>(a->D, mf, mw, mt, d, L.ncta, st)
                           : dispatch<kDecL1F32>(a->D, mf, mw, mt, d, L.ncta, st);
  if (e != cudaSuccess) return FE_ERR_CUDA;
  const int n = kDecN * a->D + kDecN + 1;
  decoder_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(L.ncta, a->D, scale, d.part_loss, d.part_dw, d.part_db, loss,
                                                         d_weight, d_bias);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

fe_status fe_decoder_read_errors(const void* workspace, uint32_t* err, void* stream) {
  if (!workspace || !err) return FE_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(err, workspace, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FE_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

}  // extern "C"
