// Semantic decoder of the rendered feature map (Sec. 3.3): a 1x1
// convolution from D to 256 channels, out[p][c] = sum_d F[p][d] W[c][d] + b[c],
// on the 5th-generation tensor cores (tcgen05, BF16 operands, FP32
// accumulators in tensor memory), optionally fused with the L1 feature loss
// of Eq. 10 and its reverse pass.
//
// One persistent CTA per SM walks 128-pixel tiles.  Warp roles:
//   warps 0-7  epilogue: tensor memory -> registers (one pixel row per
//              thread; warps w and w+4 share the rows of lane quarter w and
//              take channels 0-127 and 128-255), bias, L1 against the staged
//              target, sign -> S tile written over the target it replaces
//   warp 8     tensor-core issue (one thread) and tensor-memory allocation
//   warp 9     TMA loads of W (once) and the F tiles
//   warps 10-11  TMA loads of the targets of channels 0-127 / 128-255
//              (separate warps, so that no producer waits behind another's
//              barrier)
// The staged target box of 64 bf16 channels x 128 rows has exactly the
// layout of a 64-channel S panel (128-byte rows, 128B swizzle), so each
// epilogue thread overwrites its row of targets with its row of signs and
// the reverse products read S from the target buffer.  Two tile buffers
// alternate: the epilogue fills tile i+1 while the tensor cores run the
// reverse products of tile i, and the first product of tile i+1 is issued
// ahead of the reverse products of tile i.
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
#include "tc.cuh"

namespace fe {

namespace {

using namespace tc;
using namespace tc_host;

constexpr int kDecN = 256;        // output channels
constexpr int kDecBM = 128;       // pixels per tile (MMA M)
constexpr int kEpiWarps = 8;
constexpr int kWarpMma = kEpiWarps, kWarpF = kEpiWarps + 1, kWarpT0 = kEpiWarps + 2;
constexpr int kDecThreads = 32 * (kEpiWarps + 4);
constexpr uint32_t kBoxBytes = 16384;   // one target box: 128 rows x 128 bytes
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColAcc = 0;

enum DecMode : int { kDecForward = 0, kDecL1Bf16 = 1, kDecL1F32 = 2 };

template <int D>
struct DecCfg {
  // Output channels per launch: 256, or (D = 128) 128 -- the D = 128 decoder
  // runs as two launches over output-channel halves, because the sign of
  // each output channel depends on that channel alone and the tensor memory
  // of one CTA holds the accumulators of only half the channels at D = 128.
  static constexpr int NO = D == 128 ? 128 : kDecN;
  // F tiles in flight (D = 64, 128: two, their larger tiles fill shared memory).
  static constexpr int kFStages = D == 32 ? 3 : 2;
  static_assert(kFStages <= 3, "barrier slots for three F stages");
  // Tile buffers of bf16 targets (and S).  (A third buffer at D = 32, in
  // place of the third F stage and the merged db product, measured slower:
  // the epilogue, not the target loads, sets the tile period.)
  static constexpr int kTBufs = 2;
  static constexpr uint32_t row_bytes = D * 2;              // one F / W row in bf16
  static constexpr int KP = D <= 64 ? 1 : D / 64;           // 128-byte K panels of a row (128B swizzle)
  static constexpr uint32_t prow = D <= 64 ? row_bytes : 128u;  // bytes of a row within one panel
  static constexpr uint64_t layout = D >= 64 ? kLayout128B : kLayout64B;
  static constexpr uint32_t sbo = 8 * prow;  // stride of 8-row groups
  static constexpr uint32_t w_bytes = NO * row_bytes;
  static constexpr uint32_t w_panel = NO * prow;
  static constexpr uint32_t f_bytes = kDecBM * row_bytes;
  static constexpr uint32_t f_panel = kDecBM * prow;
  // D = 32, 128: each F stage is followed by an all-ones panel of one
  // panel's shape, so one product (N = D + 16) yields dW and, in its extra
  // columns, db.  D = 64 has no room in shared memory for it.
  static constexpr bool merged = D == 32 || D == 128;
  // D = 32: dF double-buffered in tensor memory (no room at D = 64, 128).
  static constexpr bool dfdb = D == 32;
  static constexpr uint32_t f_stride = merged ? f_bytes + f_panel : f_bytes;
  // Tensor-memory columns: accumulators of the NO outputs, dF, dW (+ db).
  static constexpr uint32_t col_df = NO;
  static constexpr uint32_t col_dw = D == 128 ? 256u : 320u;  // per M half h: + 64 h (NO = 256)
  static constexpr uint32_t col_db = 448;                     // not merged: per M half + 16 h
  static_assert(D != 128 || col_dw + D + 16 <= kTmemCols, "tensor-memory columns");
  // Target boxes staged: kTBufs tiles of bf16 (64-channel boxes) or 1 tile
  // of fp32 (32-channel boxes).
  static constexpr int kTSlots = kTBufs * NO / 64 > NO / 32 ? kTBufs * NO / 64 : NO / 32;
  static_assert(kTSlots <= 12, "barrier slots for twelve target boxes");
  static constexpr uint32_t kTBufBytes = (NO / 64) * kBoxBytes;  // one tile buffer of bf16 targets
  static constexpr uint32_t off_w = 0;
  static constexpr uint32_t off_f = off_w + w_bytes;                  // kFStages stages
  static constexpr uint32_t off_t = off_f + kFStages * f_stride;      // target boxes / S panels
  // D <= 64: each epilogue warp stages its 32 rows x D/2 columns of dF in
  // a swizzled box of its own (64-byte rows at D = 32, 128-byte at D = 64)
  // and one tensor store writes it: 4 (8) whole-line writes of each row
  // instead of one 16-byte piece of 32 rows per store instruction.  D = 128
  // (no room) stores from registers.
  static constexpr bool tma_df = D <= 64;
  static constexpr uint32_t stage_warp = tma_df ? 32u * (D / 2) * 4u : 0u;
  static constexpr uint32_t off_stage = off_t + kTSlots * kBoxBytes;
  static constexpr uint32_t off_ones = off_stage + 8 * stage_warp;
  static constexpr uint32_t off_bias = off_ones + 512;  // one 16 x 16 all-ones operand
  static constexpr uint32_t off_bar = off_bias + kDecN * 4;
  static constexpr uint32_t bytes = off_bar + 320;
  static constexpr size_t launch_bytes = bytes + 1024;  // slack for 1024-byte alignment
  static_assert(D == 32 || D == 64 || D == 128, "decoder feature width");
  static_assert(off_f % 1024 == 0 && off_t % 1024 == 0 && f_stride % 1024 == 0 && w_panel % 1024 == 0,
                "swizzled operands need 1024-byte aligned buffers");
  static_assert(launch_bytes <= 232448, "shared memory per block");
};

// Byte offset of the k-th 16-channel K step within a row-major operand of
// D channels (K-major, 32 bytes per step; at D = 128 the second 64 channels
// are the second 128-byte panel).
template <int D>
__device__ __forceinline__ uint32_t kstep(int k, uint32_t panel) {
  return D <= 64 ? 32u * k : (uint32_t)(k >> 2) * panel + 32u * (k & 3);
}

struct DecArgs {
  int64_t HW;
  int ntiles;
  int c0;            // first output channel of this launch (D = 128: 0 or 128)
  int df_add;        // 1: add dF to d_feat (the second launch at D = 128)
  int d_real;        // channels of feat / d_feat / d_weight (<= D: D = 16 runs the D = 32 kernel on tiles
                     // the tensor maps zero-fill past channel 16; the padded columns are not stored)
  const float* bias;
  float* out;        // forward: [HW, 256]
  float scale;       // L1: loss and gradient scale
  float* d_feat;     // [HW, D]
  float* part_loss;  // [ncta] (this launch's)
  float* part_dw;    // [ncta][256][D]
  float* part_db;    // [ncta][256]
  uint32_t* err;
};

// Barrier slots (8 bytes each) after off_bar.
enum : int {
  kBarW = 0, kBarFFull = 1, kBarFEmpty = kBarFFull + 3, kBarTFull = kBarFEmpty + 3,  // up to 3 F stages
  kBarTEmpty = kBarTFull + 12,  // up to 12 target slots
  kBarAccFull = kBarTEmpty + 3, kBarAccEmpty,  // up to 3 tile buffers
  kBarSFull,                // [2] and
  kBarBwd = kBarSFull + 2,  // [2]: tiles alternate, so no wait can see its barrier two phases on
  kBarDrain = kBarBwd + 2, kNumBars
};
static_assert(kNumBars * 8 + 40 <= 320, "barrier area: barriers, tensor-memory base, abort flag, 8 warp sums");

// Packed bf16 signs of two differences: +-1.0 (0x3F80 | sign bit) per half,
// 0 where the difference is 0 or the row is masked.
__device__ __forceinline__ uint32_t sign_pair_bf16(float2 d, bool valid) {
  const uint32_t hi = __byte_perm(__float_as_uint(d.x), __float_as_uint(d.y), 0x7632);
  const uint32_t s = (hi & 0x80008000u) | 0x3F803F80u;
  const uint32_t keep = (d.x != 0.0f ? 0x0000FFFFu : 0u) | (d.y != 0.0f ? 0xFFFF0000u : 0u);
  return valid ? (s & keep) : 0u;
}

__device__ __forceinline__ bool dec_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint32_t* err) {
  if (*abort) return false;
  if (mbar_wait(bar, parity)) return true;
  *abort = 1;
  set_err(err, kErrTimeout);
  return false;
}

template <bool kSpin>
__device__ __forceinline__ bool dec_spin(uint64_t* bar, uint32_t parity, volatile int* abort, uint32_t* err) {
  if (!kSpin) return dec_wait(bar, parity, abort, err);
  if (*abort) return false;
  for (int i = 0; i < (1 << 26); ++i)
    if (mbar_test(bar, parity)) return true;
  *abort = 1;
  set_err(err, kErrTimeout);
  return false;
}


template <int D, int MODE>
__global__ void __launch_bounds__(kDecThreads, 1)
    decoder_kernel(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_w,
                   const __grid_constant__ CUtensorMap tm_t, const __grid_constant__ CUtensorMap tm_d,
                   const DecArgs a) {
  using C = DecCfg<D>;
  constexpr bool kL1 = MODE != kDecForward;
  constexpr bool kTF32 = MODE == kDecL1F32;
  constexpr int NO = C::NO;
  constexpr int kBoxCh = kTF32 ? 32 : 64;         // target channels per box
  constexpr int kNumBoxes = NO / kBoxCh;          // boxes per tile
  constexpr int CPH = NO / 64;                    // 32-channel chunks per epilogue half
  constexpr uint32_t kTBufBytes = C::kTBufBytes;
  constexpr int kBufs = kTF32 ? 1 : C::kTBufs;    // tile buffers
  constexpr uint32_t kPanel = kTF32 ? 2 * kBoxBytes : kBoxBytes;  // S panel stride
  extern __shared__ unsigned char dsmem_raw[];
  // Swizzled operands are addressed by shared-memory address bits: align the
  // working base to 1024 bytes.
  const uint32_t raw_addr = smem_addr(dsmem_raw);
  unsigned char* sm = dsmem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sb = smem_addr(sm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::off_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + C::off_bar + kNumBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + C::off_bar + kNumBars * 8 + 4);
  float* s_red = reinterpret_cast<float*>(sm + C::off_bar + kNumBars * 8 + 8);  // [8]
  float* s_bias = reinterpret_cast<float*>(sm + C::off_bias);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Tiles of this CTA: blockIdx.x + i * gridDim.x for i < n_mine.
  const int n_mine = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    mbar_init(&bars[kBarW], 1);
    for (int s = 0; s < C::kFStages; ++s) {
      mbar_init(&bars[kBarFFull + s], 1);
      mbar_init(&bars[kBarFEmpty + s], 1);
    }
    for (int s = 0; s < kBufs; ++s) mbar_init(&bars[kBarTEmpty + s], 1);  // commit after the reverse products
    for (int s = 0; s < C::kTSlots; ++s) mbar_init(&bars[kBarTFull + s], 1);
    mbar_init(&bars[kBarAccFull], 1);
    mbar_init(&bars[kBarAccEmpty], kEpiWarps);
    mbar_init(&bars[kBarSFull], kEpiWarps);
    mbar_init(&bars[kBarSFull + 1], kEpiWarps);
    mbar_init(&bars[kBarBwd], 1);
    mbar_init(&bars[kBarBwd + 1], 1);
    mbar_init(&bars[kBarDrain], 1);
    *s_abort = 0;
    mbar_init_fence();
  }
  if (warp < kEpiWarps) {
    // All-ones B operand of the bias-gradient product, and the bias.
    uint4* ones = reinterpret_cast<uint4*>(sm + C::off_ones);
    for (int i = tid; i < 512 / 16; i += 32 * kEpiWarps)
      ones[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    if (C::merged)
      for (int s = 0; s < C::kFStages; ++s) {
        uint4* op = reinterpret_cast<uint4*>(sm + C::off_f + s * C::f_stride + C::f_bytes);
        for (int i = tid; i < (int)(C::f_panel / 16); i += 32 * kEpiWarps)
          op[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
      }
    fence_proxy_async();
  }
  if (warp == kWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  // Set-up above touches no global memory; everything below may read what
  // the previous kernel of the stream wrote.
  grid_dep_wait();
  grid_dep_launch();

  if (warp == kWarpF) {
    // ---------------- W (once) and F tiles ----------------
    if (lane == 0) {
      uint32_t f_uses = 0;
      mbar_arrive_expect_tx(&bars[kBarW], C::w_bytes);
      for (int pnl = 0; pnl < C::KP; ++pnl) tma_2d(sm + C::off_w + pnl * C::w_panel, &tm_w, 64 * pnl, a.c0, &bars[kBarW]);
      for (int i = 0; i < n_mine; ++i) {
        const int f = i % C::kFStages;
        if (!dec_wait(&bars[kBarFEmpty + f], ((i / C::kFStages) & 1) ^ 1, s_abort, a.err)) break;
        mbar_arrive_expect_tx(&bars[kBarFFull + f], C::f_bytes);
        for (int pnl = 0; pnl < C::KP; ++pnl)
          tma_2d(sm + C::off_f + f * C::f_stride + pnl * C::f_panel, &tm_f, 64 * pnl,
                 ((int)blockIdx.x + i * (int)gridDim.x) * kDecBM, &bars[kBarFFull + f]);
        ++f_uses;
      }
      // Every copy issued must have landed before the block leaves.
      for (uint32_t u = f_uses > C::kFStages ? f_uses - C::kFStages : 0; u < f_uses; ++u)
        if (!mbar_wait(&bars[kBarFFull + u % C::kFStages], (u / C::kFStages) & 1)) set_err(a.err, kErrTimeout);
      if (!mbar_wait(&bars[kBarW], 0)) set_err(a.err, kErrTimeout);
    }
  } else if (warp >= kWarpT0) {
    // ---------------- targets of one channel half ----------------
    if (kL1 && lane == 0) {
      const int h = warp - kWarpT0;
      int issued = 0;
      for (int i = 0; i < n_mine; ++i) {
        const int buf = i % kBufs;
        const int use = i / kBufs;  // uses of this buffer so far
        if (!dec_wait(&bars[kBarTEmpty + buf], (use & 1) ^ 1, s_abort, a.err)) break;
        for (int b = h * (kNumBoxes / 2); b < (h + 1) * (kNumBoxes / 2); ++b) {
          const int slot = buf * kNumBoxes + b;
          mbar_arrive_expect_tx(&bars[kBarTFull + slot], kBoxBytes);
          tma_2d(sm + C::off_t + slot * kBoxBytes, &tm_t, a.c0 + b * kBoxCh,
                 ((int)blockIdx.x + i * (int)gridDim.x) * kDecBM, &bars[kBarTFull + slot]);
        }
        issued = i + 1;
      }
      // Every copy issued must have landed before the block leaves.
      for (int i = issued > kBufs ? issued - kBufs : 0; i < issued; ++i)
        for (int b = h * (kNumBoxes / 2); b < (h + 1) * (kNumBoxes / 2); ++b)
          if (!mbar_wait(&bars[kBarTFull + (i % kBufs) * kNumBoxes + b], (i / kBufs) & 1))
            set_err(a.err, kErrTimeout);
    }
  } else if (warp == kWarpMma) {
    // ---------------- tensor-core issue ----------------
    if (lane == 0) {
      const uint32_t s_w = sb + C::off_w, s_t = sb + C::off_t, s_ones = sb + C::off_ones;
      constexpr uint32_t id_fwd = mma_idesc(128, NO, 0, 0);
      constexpr uint32_t id_df = mma_idesc(128, D, 0, 1);
      constexpr uint32_t id_dw = mma_idesc(128, C::merged ? D + 16 : D, 1, 1);
      constexpr uint32_t id_db = mma_idesc(128, 16, 1, 1);
      // acc = F W^T: A = F (K-major), B = W (K-major); 16 channels of K are
      // 32 bytes along each swizzled row.
      auto forward = [&](int i) -> bool {
        const int f = i % C::kFStages;
        if (!dec_spin<C::dfdb>(&bars[kBarFFull + f], (i / C::kFStages) & 1, s_abort, a.err)) return false;
        if (i > 0 && !dec_spin<C::dfdb>(&bars[kBarAccEmpty], (i - 1) & 1, s_abort, a.err)) return false;
        tc_fence_after();
        const uint32_t s_f = sb + C::off_f + f * C::f_stride;
#pragma unroll
        for (int k = 0; k < D / 16; ++k)
          mma_bf16(tmem + kColAcc, smem_desc(s_f + kstep<D>(k, C::f_panel), 16, C::sbo, C::layout),
                   smem_desc(s_w + kstep<D>(k, C::w_panel), 16, C::sbo, C::layout), id_fwd, k > 0);
        mma_commit(&bars[kBarAccFull]);
        return true;
      };
      bool ok = dec_wait(&bars[kBarW], 0, s_abort, a.err) && (n_mine == 0 || forward(0));
      for (int i = 0; ok && i < n_mine; ++i) {
        const int f = i % C::kFStages;
        if (!kL1) {
          mma_commit(&bars[kBarFEmpty + f]);
          if (i + 1 < n_mine && !forward(i + 1)) break;
          continue;
        }
        // The next tile's forward product goes ahead of this tile's reverse.
        if (i + 1 < n_mine && !forward(i + 1)) break;
        if (!dec_spin<C::dfdb>(&bars[kBarSFull + (i & 1)], (i >> 1) & 1, s_abort, a.err)) break;
        tc_fence_after();
        const uint32_t s_s = s_t + (i % kBufs) * kTBufBytes;  // S panels of this tile
        const uint32_t s_f = sb + C::off_f + f * C::f_stride;
        const uint32_t col_df = C::col_df + (C::dfdb ? (i & 1) * D : 0);  // dF buffer of this tile
        // dW += S^T F and db += S^T 1: A = S read MN-major (M = channels,
        // two 64-channel panels per half), B = F read MN-major / all ones.
        // Issued first: F's stage is released once they complete.
#pragma unroll
        for (int h = 0; h < NO / 128; ++h) {
#pragma unroll
          for (int k = 0; k < kDecBM / 16; ++k) {
            const uint64_t ad = smem_desc(s_s + h * 2 * kPanel + k * 2048, kPanel, 1024, kLayout128B);
            const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
            // Merged: B = [F | ones] along N (the ones panel one panel on).
            mma_bf16(tmem + C::col_dw + 64 * h, ad,
                     smem_desc(s_f + k * 16 * C::prow, (C::merged || C::KP > 1) ? C::f_panel : 16, C::sbo, C::layout),
                     id_dw, acc);
            if (!C::merged)
              mma_bf16(tmem + C::col_db + 16 * h, ad, smem_desc(s_ones, 256, 128, kLayoutNone), id_db, acc);
          }
        }
        mma_commit(&bars[kBarFEmpty + f]);
        // dF = S W: A = S (K-major, 128B swizzle, 64-channel panels),
        // B = W read MN-major (K = channel rows, N = D along each row; at
        // D = 128 the row's second 64 channels are the next panel: LBO).
#pragma unroll
        for (int k = 0; k < NO / 16; ++k)
          mma_bf16(tmem + col_df, smem_desc(s_s + (k >> 2) * kPanel + (k & 3) * 32, 16, 1024, kLayout128B),
                   smem_desc(s_w + k * 16 * C::prow, C::KP > 1 ? C::w_panel : 16, C::sbo, C::layout), id_df, k > 0);
        mma_commit(&bars[kBarBwd + (i & 1)]);
        mma_commit(&bars[kBarTEmpty + (i % kBufs)]);
      }
      // Drain: every issued tensor-core operation completes before the
      // accumulators are read or freed.
      mma_commit(&bars[kBarDrain]);
      if (!mbar_wait(&bars[kBarDrain], 0)) set_err(a.err, kErrTimeout);
    }
  } else {
    // ---------------- epilogue: warps 0-7, one pixel row per thread ----------------
    for (int i = tid; i < NO; i += 32 * kEpiWarps) s_bias[i] = a.bias[a.c0 + i];
    asm volatile("bar.sync 1, 256;" ::: "memory");  // epilogue warps only: the bias is in place
    const int q = warp & 3, h = warp >> 2;  // lane quarter, channel half
    const int r = q * 32 + lane;            // tile row = tensor-memory lane
    const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16);
    float loss = 0.0f;
    // This half's D/2 columns of dF for the rows of tile j, scaled, to d_feat.
    auto store_df = [&](int j) {
      const int64_t pj = ((int64_t)blockIdx.x + (int64_t)j * gridDim.x) * kDecBM + r;
      const uint32_t col = C::col_df + (C::dfdb ? (j & 1) * D : 0);  // dF buffer of tile j
      if constexpr (C::tma_df) {
        uint32_t v[32];
        const int c_lo = (D / 2) * h;  // first column of this half
        if (D == 32) tmem_ld16(t_row + col + c_lo, v);
        else tmem_ld32(t_row + col + c_lo, v);
        tmem_wait_ld(v);
        const int64_t row0 = pj - lane;                 // first row of this warp's box
        if (row0 < a.HW && c_lo < a.d_real) {  // else the box lies outside d_feat (warp-uniform)
          unsigned char* stg = sm + C::off_stage + warp * C::stage_warp;
          // This warp's previous tensor store has read the staging box.
          if (lane == 0) bulk_wait_read();
          __syncwarp();
          // Row `lane` of the box, its 16-byte chunks placed as the tensor
          // map's swizzle reads them: chunk e at e ^ ((lane / 2) mod 4) in
          // 64-byte rows, at e ^ (lane mod 8) in 128-byte rows.
          constexpr int NE = D / 8;
          const int sw = D == 32 ? (lane >> 1) & 3 : lane & 7;
#pragma unroll
          for (int e = 0; e < NE; ++e)
            *reinterpret_cast<float4*>(stg + lane * (NE * 16) + ((e ^ sw) << 4)) =
                make_float4(a.scale * __uint_as_float(v[4 * e]), a.scale * __uint_as_float(v[4 * e + 1]),
                            a.scale * __uint_as_float(v[4 * e + 2]), a.scale * __uint_as_float(v[4 * e + 3]));
          fence_proxy_async();  // staging stores -> the tensor store's reads
          __syncwarp();
          // Rows past HW are clipped by the tensor map.
          if (lane == 0) tma_store_2d(&tm_d, stg, c_lo, (int)row0);
        }
      } else {
        // This half's D/2 columns, 32 at a time, from registers (the second
        // launch adds to the first's dF).
#pragma unroll
        for (int part = 0; part < D / 64; ++part) {
          uint32_t v[32];
          const int c_lo = (D / 2) * h + 32 * part;  // first column of this part
          tmem_ld32(t_row + col + c_lo, v);
          tmem_wait_ld(v);
          if (pj < a.HW && c_lo < a.d_real) {
            float4* o = reinterpret_cast<float4*>(a.d_feat + pj * a.d_real + c_lo);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              float4 x = make_float4(a.scale * __uint_as_float(v[4 * e]), a.scale * __uint_as_float(v[4 * e + 1]),
                                     a.scale * __uint_as_float(v[4 * e + 2]), a.scale * __uint_as_float(v[4 * e + 3]));
              if (a.df_add) {
                const float4 y = o[e];
                x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
              }
              o[e] = x;
            }
          }
        }
      }
    };
    int i = 0;
    bool ok = true;
    for (; i < n_mine; ++i) {
      if (!dec_wait(&bars[kBarAccFull], i & 1, s_abort, a.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int64_t p = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kDecBM + r;
      const bool valid = p < a.HW;
      unsigned char* tbuf = sm + C::off_t + (i % kBufs) * kTBufBytes;
      // CPH 32-channel chunks; the load of chunk c+1 is in flight while
      // chunk c is processed.  Once the last chunk is in registers the
      // accumulator is released, so the next tile's forward product runs
      // while that chunk is processed.
      uint32_t va[32], vb[32];
      tmem_ld32(t_row + kColAcc + 32 * (CPH * h), va);
      tmem_wait_ld(va);
#pragma unroll
      for (int c = 0; c < CPH; ++c) {
        uint32_t(&cur)[32] = (c & 1) ? vb : va;
        uint32_t(&nxt)[32] = (c & 1) ? va : vb;
        if (c > 0) tmem_wait_ld(cur);
        if (c < CPH - 1) tmem_ld32(t_row + kColAcc + 32 * (CPH * h + c + 1), nxt);
        if (c == CPH - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars[kBarAccEmpty]);
        }
        const int ch = CPH * h + c;
        const float2* bias2 = reinterpret_cast<const float2*>(s_bias + 32 * ch);
        if (!kL1) {
          if (valid) {
            float4* o = reinterpret_cast<float4*>(a.out + p * kDecN + a.c0 + 32 * ch);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float2 lo = __fadd2_rn(make_float2(__uint_as_float(cur[4 * e]), __uint_as_float(cur[4 * e + 1])),
                                           bias2[2 * e]);
              const float2 hi = __fadd2_rn(
                  make_float2(__uint_as_float(cur[4 * e + 2]), __uint_as_float(cur[4 * e + 3])), bias2[2 * e + 1]);
              o[e] = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
          }
          continue;
        }
        // Target box of this chunk and its row r (128-byte rows, 16-byte
        // chunks permuted by row & 7).
        const int box = kTF32 ? ch : ch >> 1;
        if ((kTF32 || (c & 1) == 0) &&
            !dec_wait(&bars[kBarTFull + (i % kBufs) * kNumBoxes + box], (i / kBufs) & 1, s_abort, a.err))
          ok = false;
        const unsigned char* trow = tbuf + box * kBoxBytes + r * 128;
        float2 t2[16];
        if (kTF32) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float4 x = *reinterpret_cast<const float4*>(trow + ((e ^ (r & 7)) << 4));
            t2[2 * e] = make_float2(x.x, x.y);
            t2[2 * e + 1] = make_float2(x.z, x.w);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint4 x = *reinterpret_cast<const uint4*>(trow + (((4 * (c & 1) + e) ^ (r & 7)) << 4));
            const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
              t2[4 * e + k] = make_float2(__uint_as_float(w4[k] << 16), __uint_as_float(w4[k] & 0xFFFF0000u));
          }
        }
        uint32_t sg[16];
        // |o - t| of even and odd channels in two chains (then one sum).
        float part_e = 0.0f, part_o = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float2 o =
              __fadd2_rn(make_float2(__uint_as_float(cur[2 * k]), __uint_as_float(cur[2 * k + 1])), bias2[k]);
          const float2 d = __ffma2_rn(t2[k], make_float2(-1.0f, -1.0f), o);  // o - t, one rounding
          part_e += fabsf(d.x);
          part_o += fabsf(d.y);
          sg[k] = sign_pair_bf16(d, valid);
        }
        if (valid) loss += part_e + part_o;
        // S row r, channels 32ch .. 32ch+31: panel ch/2 of this tile buffer,
        // logical chunks 4 (ch & 1) .. +3 -- over targets already consumed.
        unsigned char* srow = tbuf + (ch >> 1) * kPanel + r * 128;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          *reinterpret_cast<uint4*>(srow + (((4 * (ch & 1) + e) ^ (r & 7)) << 4)) =
              make_uint4(sg[4 * e], sg[4 * e + 1], sg[4 * e + 2], sg[4 * e + 3]);
      }
      if (!ok) break;
      if (!kL1) continue;
      if (C::dfdb) {
        // dF is double-buffered: release this tile's S at once, then store
        // the previous tile's dF (its reverse products ran meanwhile).
        fence_proxy_async();  // S stores -> tensor-core reads
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[kBarSFull + (i & 1)]);
        if (i > 0) {
          if (!dec_wait(&bars[kBarBwd + ((i - 1) & 1)], ((i - 1) >> 1) & 1, s_abort, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          store_df(i - 1);
          tc_fence_before();
        }
        continue;
      }
      // dF of the previous tile (its reverse products ran while this tile
      // was processed), before this tile's products may overwrite it.
      if (i > 0) {
        if (!dec_wait(&bars[kBarBwd + ((i - 1) & 1)], ((i - 1) >> 1) & 1, s_abort, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        store_df(i - 1);
        tc_fence_before();
      }
      fence_proxy_async();  // S stores -> tensor-core reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[kBarSFull + (i & 1)]);
    }
    if (kL1) {
      if (ok && n_mine > 0 &&
          dec_wait(&bars[kBarBwd + ((n_mine - 1) & 1)], ((n_mine - 1) >> 1) & 1, s_abort, a.err)) {
        tc_fence_after();
        store_df(n_mine - 1);
      }
      // Per-CTA partials: the dW rows and db of this half's channels, the
      // loss of this CTA (fixed-order sums).
      asm volatile("bar.sync 1, 256;" ::: "memory");  // epilogue warps only
      if (!*s_abort && n_mine > 0) {
        // The last backward barrier covers every product of this CTA.
        // NO = 256: M half h = channels 128 h + r, its D columns; NO = 128
        // (D = 128): one M tile of channels c0 + r, its columns split between
        // the two warps of each lane quarter (h: columns 64 h .. 64 h + 63).
        tc_fence_after();
        const int c = a.c0 + (NO == 256 ? h * 128 : 0) + r;
        constexpr int KW = NO == 256 ? D / 32 : D / 64;  // 32-column loads per warp
#pragma unroll
        for (int k = 0; k < KW; ++k) {
          const int c_lo = NO == 256 ? 32 * k : 64 * h + 32 * k;
          uint32_t v[32];
          tmem_ld32(t_row + C::col_dw + (NO == 256 ? 64 * h : 0) + c_lo, v);
          tmem_wait_ld(v);
          float4* o = reinterpret_cast<float4*>(a.part_dw + ((size_t)blockIdx.x * kDecN + c) * D + c_lo);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                               __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
        }
        uint32_t vb1;
        // db: a column of its own, or (merged) column D of the dW product.
        tmem_ld1(t_row + (C::merged ? C::col_dw + (NO == 256 ? 64 * h : 0) + D : C::col_db + 16 * h), vb1);
        tmem_wait_ld1(vb1);
        if (NO == 256 || h == 0) a.part_db[(size_t)blockIdx.x * kDecN + c] = __uint_as_float(vb1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
      if (lane == 0) s_red[warp] = loss;
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (tid == 0) {
        float sum = 0.0f;
        for (int w = 0; w < kEpiWarps; ++w) sum += s_red[w];
        a.part_loss[blockIdx.x] = sum;
      }
    }
    // Tensor stores of dF complete before the block leaves.
    if (C::tma_df && kL1 && lane == 0) bulk_wait_all();
    tc_fence_before();
  }
  __syncthreads();
  if (warp == kWarpMma) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Fixed-order sums of the per-CTA partials, scaled (partials of D columns,
// the first d_real of them stored; nloss loss partials).  A block sums 32
// outputs (one per lane): warp w adds the partials c = w, w + 8, ... in
// order, then the eight warp sums are added in warp order.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(32 * kRedWarps) decoder_reduce_kernel(int ncta, int nloss, int D, int d_real,
                                                                        float scale, const float* part_loss,
                                                                        const float* part_dw, const float* part_db,
                                                                        float* loss, float* d_weight, float* d_bias) {
  __shared__ float s_part[kRedWarps][33];
  grid_dep_wait();  // the decoder launches that wrote the partials
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_dw = kDecN * d_real;
  const int i = blockIdx.x * 32 + lane;
  const float* src = nullptr;
  size_t stride = 0;
  int count = 0;
  float* dst = nullptr;
  if (i < n_dw) {
    src = part_dw + (size_t)(i / d_real) * D + i % d_real;
    stride = (size_t)kDecN * D;
    count = ncta;
    dst = d_weight + i;
  } else if (i < n_dw + kDecN) {
    src = part_db + (i - n_dw);
    stride = kDecN;
    count = ncta;
    dst = d_bias + (i - n_dw);
  } else if (i == n_dw + kDecN) {
    src = part_loss;
    stride = 1;
    count = nloss;
    dst = loss;
  }
  float s = 0.0f;
#pragma unroll 4
  for (int c = warp; c < count; c += kRedWarps) s += src[(size_t)c * stride];
  s_part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && dst) {
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < kRedWarps; ++w) t += s_part[w][lane];
    *dst = scale * t;
  }
}

template <int D, int MODE>
cudaError_t launch_dec(const CUtensorMap& mf, const CUtensorMap& mw, const CUtensorMap& mt, const CUtensorMap& md,
                       const DecArgs& a, int grid, cudaStream_t st) {
  auto k = decoder_kernel<D, MODE>;
  const size_t smem = DecCfg<D>::launch_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k, grid, kDecThreads, smem, st, mf, mw, mt, md, a);
}

// Workspace: 256-byte header (error bits), then per-CTA partial loss, dW, db.
struct DecLayout {
  int ncta;
  size_t loss, dw, db, total;
};

// Launches of one decoder call: D = 128 runs over two output-channel halves.
int dec_passes(int DW) { return DW == 128 ? 2 : 1; }

DecLayout dec_layout(int64_t HW, int D) {
  DecLayout L{};
  const int64_t ntiles = (HW + kDecBM - 1) / kDecBM;
  const int sms = num_sms();
  L.ncta = (int)(ntiles < sms ? ntiles : sms);
  if (L.ncta < 1) L.ncta = 1;
  L.loss = 256;
  L.dw = align_up(L.loss + (size_t)dec_passes(D) * L.ncta * 4, 256);
  L.db = align_up(L.dw + (size_t)L.ncta * kDecN * D * 4, 256);
  L.total = align_up(L.db + (size_t)L.ncta * kDecN * 4, 256);
  return L;
}

bool aligned16p(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The kernel width for D channels (16 runs as 32 on zero-filled tiles).
int dec_width(int D) { return D == 16 ? 32 : D; }

fe_status dec_check(const fe_decoder_args* a) {
  if (!a || a->HW < 0 || a->HW > (int64_t)kDecBM * ((1ll << 31) / kDecBM - 1)) return FE_ERR_INVALID_ARG;
  if (a->D != 16 && a->D != 32 && a->D != 64 && a->D != 128) return FE_ERR_UNSUPPORTED;
  if (!a->weight || !a->bias || !aligned16p(a->weight)) return FE_ERR_INVALID_ARG;
  if (a->HW > 0 && (!a->feat || !aligned16p(a->feat))) return FE_ERR_INVALID_ARG;
  return FE_OK;
}

template <int MODE>
cudaError_t dispatch(int D, const CUtensorMap& mf, const CUtensorMap& mw, const CUtensorMap& mt, const CUtensorMap& md,
                     const DecArgs& a, int grid, cudaStream_t st) {
  switch (D) {
    case 32: return launch_dec<32, MODE>(mf, mw, mt, md, a, grid, st);
    case 64: return launch_dec<64, MODE>(mf, mw, mt, md, a, grid, st);
    case 128: return launch_dec<128, MODE>(mf, mw, mt, md, a, grid, st);
  }
  return cudaErrorInvalidValue;
}

// Tensor maps of the feature map and the weights: rows of D channels, boxes
// of DW channels (zero-filled past D) or, at D = 128, of one 64-channel
// panel; weight boxes of the rows one launch reads.
bool dec_maps(const fe_decoder_args* a, int DW, CUtensorMap* mf, CUtensorMap* mw) {
  const CUtensorMapSwizzle swz = DW >= 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  const uint32_t box = DW <= 64 ? (uint32_t)DW : 64u;
  const uint32_t wrows = DW == 128 ? 128u : (uint32_t)kDecN;
  return make_map(mf, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a->feat, a->D, a->HW, box, kDecBM, swz) &&
         make_map(mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a->weight, a->D, kDecN, box, wrows, swz);
}

}  // namespace

}  // namespace fe

using namespace fe;

extern "C" {

size_t fe_decoder_workspace_size(int64_t HW, int D) {
  if (HW < 0 || (D != 16 && D != 32 && D != 64 && D != 128)) return 0;
  return dec_layout(HW, dec_width(D)).total;
}

fe_status fe_decode_forward(const fe_decoder_args* a, float* out, void* workspace, size_t workspace_bytes,
                            void* stream) {
  fe_status s = dec_check(a);
  if (s != FE_OK) return s;
  if (!workspace || !out || !aligned16p(out)) return FE_ERR_INVALID_ARG;
  const int DW = dec_width(a->D);
  const DecLayout L = dec_layout(a->HW, DW);
  if (workspace_bytes < L.total) return FE_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(workspace, 0, 256, st) != cudaSuccess) return FE_ERR_CUDA;
  if (a->HW == 0) return FE_OK;
  CUtensorMap mf, mw;
  if (!dec_maps(a, DW, &mf, &mw)) return FE_ERR_CUDA;
  DecArgs d{};
  d.HW = a->HW;
  d.ntiles = (int)((a->HW + kDecBM - 1) / kDecBM);
  d.d_real = a->D;
  d.bias = a->bias;
  d.out = out;
  d.err = static_cast<uint32_t*>(workspace);
  for (int pass = 0; pass < dec_passes(DW); ++pass) {
    d.c0 = 128 * pass;
    if (dispatch<kDecForward>(DW, mf, mw, mw, mw, d, L.ncta, st) != cudaSuccess) return FE_ERR_CUDA;
  }
  return FE_OK;
}

fe_status fe_decode_l1(const fe_decoder_args* a, const void* target, int target_bf16, float scale, float* loss,
                       float* d_feat, float* d_weight, float* d_bias, void* workspace, size_t workspace_bytes,
                       void* stream) {
  fe_status s = dec_check(a);
  if (s != FE_OK) return s;
  if (!workspace || !loss || !d_weight || !d_bias) return FE_ERR_INVALID_ARG;
  if (a->HW > 0 && (!target || !aligned16p(target) || !d_feat || !aligned16p(d_feat))) return FE_ERR_INVALID_ARG;
  const int DW = dec_width(a->D);
  const DecLayout L = dec_layout(a->HW, DW);
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
  CUtensorMap mf, mw, mt, md;
  const bool tb = target_bf16 != 0;
  if (!dec_maps(a, DW, &mf, &mw) ||
      !make_map(&mt, tb ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, tb ? 2 : 4, target,
                kDecN, a->HW, tb ? 64 : 32, kDecBM, CU_TENSOR_MAP_SWIZZLE_128B))
    return FE_ERR_CUDA;
  // d_feat in boxes of 32 rows x DW/2 channels: the dF a warp stages at
  // D <= 64 (D = 128 stores from registers and reads no map).
  md = mw;
  if (DW <= 64 && !make_map(&md, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d_feat, a->D, a->HW, DW / 2, 32,
                            DW == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B))
    return FE_ERR_CUDA;
  DecArgs d{};
  d.HW = a->HW;
  d.ntiles = (int)((a->HW + kDecBM - 1) / kDecBM);
  d.d_real = a->D;
  d.bias = a->bias;
  d.scale = scale;
  d.d_feat = d_feat;
  d.part_loss = reinterpret_cast<float*>(ws + L.loss);
  d.part_dw = reinterpret_cast<float*>(ws + L.dw);
  d.part_db = reinterpret_cast<float*>(ws + L.db);
  d.err = static_cast<uint32_t*>(workspace);
  // D = 128: the second launch (channels 128-255) adds its dF to the
  // first's (same stream: a fixed order) and has loss partials of its own.
  const int npass = dec_passes(DW);
  for (int pass = 0; pass < npass; ++pass) {
    DecArgs dp = d;
    dp.c0 = 128 * pass;
    dp.df_add = pass > 0 ? 1 : 0;
    dp.part_loss = d.part_loss + (size_t)pass * L.ncta;
    const cudaError_t e = tb ? dispatch<kDecL1Bf16>(DW, mf, mw, mt, md, dp, L.ncta, st)
                             : dispatch<kDecL1F32>(DW, mf, mw, mt, md, dp, L.ncta, st);
    if (e != cudaSuccess) return FE_ERR_CUDA;
  }
  const int n = kDecN * a->D + kDecN + 1;
  const cudaError_t e = launch_pdl(decoder_reduce_kernel, (n + 31) / 32, 32 * kRedWarps, 0, st, L.ncta, npass * L.ncta,
                                   DW, a->D, scale, (const float*)d.part_loss, (const float*)d.part_dw,
                                   (const float*)d.part_db, loss, d_weight, d_bias);
  return e == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

fe_status fe_decoder_read_errors(const void* workspace, uint32_t* err, void* stream) {
  if (!workspace || !err) return FE_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(err, workspace, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FE_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

}  // extern "C"
