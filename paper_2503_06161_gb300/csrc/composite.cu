// Per-tile front-to-back compositing of colour, semantic feature and depth
// (Sec. 3.3, Eq. 7-8) and its reverse pass.
//
// Forward: one 256-thread block per tile, one pixel per thread.  Batches of
// the tile's sorted list are staged in shared memory; each pixel walks them
// in order, accumulating w = alpha*T into rgb, depth and the D feature
// channels, and stops before a Gaussian that would take T below 1e-4.  The
// block leaves as soon as every pixel is done (__syncthreads_count).
//
// Reverse: the same block walks the list backwards from the largest
// n_contrib of the tile, replaying T_i = T_{i+1} / (1 - alpha_i) from
// T_final (no per-pixel lists are stored).  Per batch, the per-(pixel,
// Gaussian) terms go to shared memory and are summed over the tile's pixels
// in a fixed order, one partial row per (tile, Gaussian) entry: no
// floating-point atomics, bitwise deterministic.
#include "common.cuh"
#include "kernels.h"

namespace fe {

namespace {

// Gaussians per staged batch of the forward; two batches are in flight.
template <int D>
constexpr int fwd_batch() { return D <= 32 ? 128 : (D <= 64 ? 64 : 32); }

// Bytes of one staged batch: B render records (48 bytes each), then B
// feature rows in their stored format (fp32 or bf16).
__host__ __device__ constexpr uint32_t stage_bytes(int B, int D, int bf16) {
  return (uint32_t)B * (uint32_t)(kRec * 4 + D * (bf16 ? 2 : 4));
}

// Bulk copies of one batch into a staging buffer, completing on `bar`:
// thread 0 arms the barrier with the batch's byte count, thread t < nb copies
// the record and the feature row of its Gaussian g.  Sources start at
// 48 g and g * row bytes of 16-byte aligned arrays, destinations at
// multiples of 16 bytes, and every size is a multiple of 16 bytes.
template <int D>
__device__ __forceinline__ void stage_issue(const CompositeArgs& a, unsigned char* buf, int B, int nb, uint32_t g,
                                            uint64_t* bar) {
  const int tid = threadIdx.x;
  const uint32_t rowb = (uint32_t)D * (a.feat_bf16 ? 2u : 4u);
  if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)nb * ((uint32_t)kRec * 4u + rowb));
  if (tid < nb) {
    fence_proxy_async();  // earlier generic reads of this buffer come first
    tma_load_1d(buf + (size_t)tid * kRec * 4, a.rec + 3 * (size_t)g, (uint32_t)kRec * 4u, bar);
    tma_load_1d(buf + (size_t)B * kRec * 4 + (size_t)tid * rowb,
                static_cast<const unsigned char*>(a.feat) + (size_t)g * a.feat_row_bytes, rowb, bar);
  }
}

// bf16 feature rows of a landed batch -> fp32 rows (whole block).
template <int D>
__device__ __forceinline__ void widen_bf16(const unsigned char* raw, float* dst, int nb) {
  const uint4* src = reinterpret_cast<const uint4*>(raw);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < nb * (D / 8); i += kThreads) {
    const uint4 q = src[i];
    d4[2 * i] = make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xFFFF0000u),
                            __uint_as_float(q.y << 16), __uint_as_float(q.y & 0xFFFF0000u));
    d4[2 * i + 1] = make_float4(__uint_as_float(q.z << 16), __uint_as_float(q.z & 0xFFFF0000u),
                                __uint_as_float(q.w << 16), __uint_as_float(q.w & 0xFFFF0000u));
  }
}

// Shared memory of the forward with B-Gaussian batches: two staging
// buffers, then (bf16 features) one fp32 copy of the current batch's rows.
__host__ __device__ constexpr size_t fwd_smem_bytes(int B, int D, int bf16) {
  return 2 * (size_t)stage_bytes(B, D, bf16) + (bf16 ? (size_t)B * D * 4 : 0);
}

// Staging state a block carries from tile to tile: how many times each of
// its two staging buffers has been armed.  Arming is block-uniform, so
// every thread derives the same wait parity from it: batch j of a tile sits
// in buffer j & 1 and completes that buffer's (arms[b] + j / 2)-th phase.
struct StageState {
  uint32_t arms[2];
  bool dead;  // a drain gave up: shared memory may still receive a copy
};

__device__ __forceinline__ uint32_t stage_parity(const StageState& st, uint32_t j) {
  return (st.arms[j & 1] + (j >> 1)) & 1u;
}

// A tile is done with its staging buffers: the last two batches it issued
// (any earlier one completed before its buffer was re-armed) must land
// before shared memory is reused, whether the tile finished, left early or
// gave up on a wait.  The drain has its own, long bound; if even that runs
// out the block stops taking tiles.
__device__ __forceinline__ void stage_drain(StageState& st, uint64_t* s_bar, uint32_t issued, uint32_t* err) {
  bool ok = true;
  for (uint32_t j = issued > 2 ? issued - 2 : 0; j < issued; ++j)
    ok &= mbar_wait(&s_bar[j & 1], stage_parity(st, j), kDrainPolls);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) set_err(err, kErrTimeout);
    st.dead = true;
  }
  st.arms[0] += (issued + 1) / 2;
  st.arms[1] += issued / 2;
}

// True when no pixel centre of the rectangle [x0, x1] x [y0, y1] can blend
// record `rec` (so a warp covering it may skip the entry without changing
// anything): either the 3-sigma square misses the rectangle -- the per-pixel
// test, at the rectangle's nearest centres, with the same subtractions -- or
// the record's blend box (word 11) does.
__device__ __forceinline__ bool block_misses(const float* rec, float x0, float x1, float y0, float y1) {
  const float2 uv = *reinterpret_cast<const float2*>(rec);
  const float2 rb = *reinterpret_cast<const float2*>(rec + 10);  // radius, packed box
  const float u = uv.x, v = uv.y, r = rb.x;
  if (__fsub_rn(x0, u) > r || __fsub_rn(u, x1) > r || __fsub_rn(y0, v) > r || __fsub_rn(v, y1) > r) return true;
  const uint32_t hb = __float_as_uint(rb.y);
  const __half2 h = *reinterpret_cast<const __half2*>(&hb);
  const float hx = __low2float(h), hy = __high2float(h);
  return hx < 0.0f || x0 - u > hx || u - x1 > hx || y0 - v > hy || v - y1 > hy;
}

// Forward compositing of one tile by the whole block (see the file comment).
template <int D, int B, bool kCount>
__device__ __forceinline__ void fwd_tile(const CompositeArgs& a, const int tile, unsigned char* smem, uint64_t* s_bar,
                                         int* s_abort, StageState& stg) {
  const int tid = threadIdx.x;
  const bool bf16 = a.feat_bf16 != 0;
  const uint32_t sbytes = stage_bytes(B, D, a.feat_bf16);
  float* s_wide = reinterpret_cast<float*>(smem + 2 * (size_t)sbytes);
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  int lx, ly;
  tile_pixel(tid, a.tw, lx, ly);
  const int px = tx * a.tw + lx, py = ty * a.th + ly;
  const bool inside = px < a.W && py < a.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const uint2 rg = a.ranges[tile];
  const uint32_t n = rg.y - rg.x;
  const uint32_t nbatch = (n + B - 1) / B;
  // Gaussian of this thread's slot in batch k (prefetched a batch ahead).
  auto slot_gid = [&](uint32_t k) -> uint32_t {
    const uint32_t p = k * B + (uint32_t)tid;
    return (k < nbatch && tid < B && p < n) ? __ldg(&a.sorted[rg.x + p].y) : 0u;
  };
  auto batch_len = [&](uint32_t k) -> int { return (int)min((uint32_t)B, n - k * B); };
  uint32_t issued = 0;
  if (nbatch > 0) {
    stage_issue<D>(a, smem, B, batch_len(0), slot_gid(0), &s_bar[0]);
    issued = 1;
  }
  uint32_t g_next = slot_gid(1);
  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Z = 0.f;
  float2 F[D / 2];  // feature channels in pairs (packed FP32 FMA)
#pragma unroll
  for (int d = 0; d < D / 2; ++d) F[d] = make_float2(0.0f, 0.0f);
  uint32_t last = 0;
  uint32_t visits = 0, contribs = 0;  // only used by the counting variant
  bool done = !inside;
  // Entries of the current batch this pixel blended, per 32-entry group
  // (up to four groups: B <= 128).
  constexpr int NG = B / 32;
  static_assert(NG >= 1 && NG <= 4, "blend masks cover at most four groups");
  uint32_t cm0 = 0u, cm1 = 0u, cm2 = 0u, cm3 = 0u;
  const bool track = !kCount && a.cmask != nullptr && a.aux;
  const size_t cslot0 = (size_t)(rg.x >> 5) + (size_t)tile;
  const int lane = tid & 31, warp = tid >> 5;
  // Pixel centres of this warp's 8 x 4 block.
  const float bx0 = (float)(tx * a.tw + ((warp % (a.tw >> 3)) << 3)) + 0.5f;
  const float by0 = (float)(ty * a.th + ((warp / (a.tw >> 3)) << 2)) + 0.5f;
  for (uint32_t k = 0; k < nbatch; ++k) {
    // Every thread is past batch k-1 here, so its buffer may be refilled.
    // A wait on batch k-1 that gave up (s_abort[(k-1) & 1], written before
    // this barrier; a failure in this iteration writes the other slot, so
    // no thread can see it change) ends the tile for the whole block before
    // anything is re-armed.
    if (__syncthreads_count(done) == kThreads || (k > 0 && ((volatile int*)s_abort)[(k - 1) & 1])) break;
    if (k + 1 < nbatch) {
      stage_issue<D>(a, smem + ((k + 1) & 1) * (size_t)sbytes, B, batch_len(k + 1), g_next, &s_bar[(k + 1) & 1]);
      issued = k + 2;
      g_next = slot_gid(k + 2);
    }
    const unsigned char* buf = smem + (k & 1) * (size_t)sbytes;
    const bool landed = mbar_wait(&s_bar[k & 1], stage_parity(stg, k), a.polls);
    if (!landed) {
      ((volatile int*)s_abort)[k & 1] = 1;
      set_err(a.err, kErrTimeout);
      done = true;
    }
    const int nb = batch_len(k);
    const float* s_rec = reinterpret_cast<const float*>(buf);
    const float* s_feat = reinterpret_cast<const float*>(buf + (size_t)B * kRec * 4);
    if (bf16) {
      // Every thread widens its share of the rows (also threads whose pixel
      // is outside the image or done), unless its wait gave up.
      if (landed) widen_bf16<D>(buf + (size_t)B * kRec * 4, s_wide, nb);
      __syncthreads();
      s_feat = s_wide;
    }
    uint32_t cur = 0u;  // blended entries of the current 32-entry group
    // Entries of each 32-entry group that some pixel of this warp's block
    // may blend (the others leave every pixel of the block unchanged).
    uint32_t em0 = 0u, em1 = 0u, em2 = 0u, em3 = 0u;
    if (!kCount && __any_sync(0xFFFFFFFFu, !done)) {
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const int j = 32 * g + lane;
        const bool ev = j < nb && !block_misses(s_rec + j * kRec, bx0, bx0 + 7.0f, by0, by0 + 3.0f);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, ev);
        if (g == 0) em0 = m;
        if (g == 1) em1 = m;
        if (g == 2) em2 = m;
        if (g == 3) em3 = m;
      }
    }
    // Blend entry j (pe: its evaluation); true once the pixel is done.
    auto blend = [&](int j, const PairEval& pe) -> bool {
      const float* rec = s_rec + j * kRec;
      const float Tn = __fmul_rn(T, __fsub_rn(1.0f, pe.alpha));
      if (Tn < kTMin) {
        done = true;
        return true;
      }
      if (kCount) ++contribs;
      const float w = pe.alpha * T;
      C0 = fmaf(w, rec[7], C0);
      C1 = fmaf(w, rec[8], C1);
      C2 = fmaf(w, rec[9], C2);
      Z = fmaf(w, rec[6], Z);
      const float4* f4 = reinterpret_cast<const float4*>(s_feat + j * D);
      const float2 w2 = make_float2(w, w);
#pragma unroll
      for (int d4 = 0; d4 < D / 4; ++d4) {
        const float4 f = f4[d4];
        F[2 * d4] = __ffma2_rn(w2, make_float2(f.x, f.y), F[2 * d4]);
        F[2 * d4 + 1] = __ffma2_rn(w2, make_float2(f.z, f.w), F[2 * d4 + 1]);
      }
      T = Tn;
      last = k * B + (uint32_t)j + 1u;
      cur |= 1u << (j & 31);
      return false;
    };
    if (!done) {
      if (kCount) {
        // Counting form: every listed pair up to termination.
        for (int j = 0; j < nb; ++j) {
          PairEval pe;
          ++visits;
          if (eval_pair(s_rec + j * kRec, pxc, pyc, pe) && blend(j, pe)) break;
        }
      } else {
        // Groups of 32 entries; the entries the warp's block may blend are
        // taken in order, two at a time: both evaluated ahead of their
        // (ordered) blending -- the two evaluations are independent, only
        // the blend carries T.
        for (int g = 0; g < NG && !done; ++g) {
          uint32_t t = g == 0 ? em0 : g == 1 ? em1 : g == 2 ? em2 : em3;
          cur = 0u;
          while (t) {
            const int ja = 32 * g + __ffs(t) - 1;
            t &= t - 1u;
            PairEval p0, p1;
            // Evaluations without early exits, so that they interleave
            // (identical arithmetic and decisions to eval_pair).
            const bool h0 = eval_pair_flat(s_rec + ja * kRec, pxc, pyc, p0);
            if (t) {
              const int jb = 32 * g + __ffs(t) - 1;
              t &= t - 1u;
              const bool h1 = eval_pair_flat(s_rec + jb * kRec, pxc, pyc, p1);
              if (h0 && blend(ja, p0)) break;
              if (h1 && blend(jb, p1)) break;
            } else if (h0 && blend(ja, p0)) {
              break;
            }
          }
          cm0 |= g == 0 ? cur : 0u;
          if (NG > 1) cm1 |= g == 1 ? cur : 0u;
          if (NG > 2) cm2 |= g == 2 ? cur : 0u;
          if (NG > 3) cm3 |= g == 3 ? cur : 0u;
        }
      }
    }
    if (track) {
      // The warp's blended entries of each group of this batch.
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const uint32_t m = __reduce_or_sync(0xFFFFFFFFu, g == 0 ? cm0 : g == 1 ? cm1 : g == 2 ? cm2 : cm3);
        if (lane == 0 && k * B + 32u * g < n) a.cmask[(cslot0 + (k * B) / 32 + g) * 8 + warp] = m;
      }
      cm0 = cm1 = cm2 = cm3 = 0u;
    }
  }
  stage_drain(stg, s_bar, issued, a.err);
  if (kCount) {
    // Block sums of the pair counts, one 64-bit atomic per warp.
    unsigned long long v = visits, c = contribs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(a.counts), v);
      atomicAdd(reinterpret_cast<unsigned long long*>(a.counts) + 1, c);
    }
    return;
  }
  if (inside) {
    const size_t HW = (size_t)a.W * a.H, p = (size_t)py * a.W + px;
    if (a.aux) {
      a.out_rgb[p] = C0 + T * a.bg[0];
      a.out_rgb[HW + p] = C1 + T * a.bg[1];
      a.out_rgb[2 * HW + p] = C2 + T * a.bg[2];
      a.out_depth[p] = Z;
      a.out_alpha[p] = 1.0f - T;
      a.t_final[p] = T;
      a.n_contrib[p] = last;
    }
    float4* fo = reinterpret_cast<float4*>(a.out_feat + p * a.out_ld);
#pragma unroll
    for (int d4 = 0; d4 < D / 4; ++d4) fo[d4] = make_float4(F[2 * d4].x, F[2 * d4].y, F[2 * d4 + 1].x, F[2 * d4 + 1].y);
    if (a.out_feat_bf16) {
      uint4* fb = reinterpret_cast<uint4*>(a.out_feat_bf16 + p * a.out_ld);
#pragma unroll
      for (int q = 0; q < D / 8; ++q) {
        uint32_t w4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(F[4 * q + e].x, F[4 * q + e].y);
          w4[e] = *reinterpret_cast<const uint32_t*>(&h);
        }
        fb[q] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
    }
  }
}

// Barriers and the abort flag of a compositing block, initialised once.
__device__ __forceinline__ void stage_init(uint64_t* s_bar) {
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
}

// One block per tile.
template <int D, int B, bool kCount>
__global__ void __launch_bounds__(kThreads, D <= 32 ? 3 : (D <= 64 ? 2 : 1)) composite_fwd_kernel(const CompositeArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_abort[2];
  stage_init(s_bar);
  if (threadIdx.x == 0) s_abort[0] = s_abort[1] = 0;
  __syncthreads();
  StageState stg{{0u, 0u}, false};
  fwd_tile<D, B, kCount>(a, blockIdx.x, smem, s_bar, s_abort, stg);
}

// (view, tile) work item `item` of a batch: the view whose item range holds it.
__device__ __forceinline__ int batch_view(const BatchCompositeArgs& ba, int item) {
  int v = 0;
  while (v + 1 < ba.V && item >= ba.item_start[v + 1]) ++v;
  return v;
}

// Persistent form over a batch of views: each block takes (view, tile)
// items from a device counter until the batch is exhausted (no block waits
// for another: items are independent).
template <int D, int B>
__global__ void __launch_bounds__(kThreads, D <= 32 ? 3 : (D <= 64 ? 2 : 1))
    composite_fwd_batch_kernel(const __grid_constant__ BatchCompositeArgs ba) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_abort[2], s_item;
  stage_init(s_bar);
  StageState stg{{0u, 0u}, false};
  for (;;) {
    // Every thread is past the previous tile (its drain ended in a barrier).
    if (threadIdx.x == 0) {
      s_item = (int)atomicAdd(ba.queue, 1u);
      s_abort[0] = s_abort[1] = 0;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= ba.nitems || stg.dead) break;
    const int v = batch_view(ba, item);
    fwd_tile<D, B, false>(ba.view[v], item - ba.item_start[v], smem, s_bar, s_abort, stg);
  }
}

// ---------------------------------------------------------------------------
// Reverse pass.  Per batch of B list entries (walked backwards), each pixel
// thread replays its recurrence and forms, per (pixel, entry): the blend
// weight w and six geometric terms (du, dv, dA, dB, dCc, dopacity).  Then:
//  * geometric terms: a shuffle reduce-scatter over the warp's 32 pixels,
//    only for entries where some lane of the warp contributed;
//  * linear terms sum_p w_p G_p with G_p = (g_rgb, g_depth, g_feat): a
//    register-blocked (entries x channels) product over the warp's pixels;
//  * a fixed-order sum of the 8 warp partials per entry.
template <int D>
struct BwdCfg {
  static constexpr int NC = 4 + D;                  // linear channels
  static constexpr int B = D <= 64 ? 32 : 16;       // entries per batch
  static constexpr int JG = 16, CG = 2;             // lane grid of the per-warp product
  static constexpr int JPL = B / JG;                // entries per lane
  static constexpr int CPL = NC / CG;               // channels per lane (even: packed FMA)
  static constexpr bool GREG = D <= 64;             // upstream gradients kept in registers
  static constexpr int GS = NC + 2;                 // per-pixel gradient row stride (8-byte rows)
  static constexpr int WS = B + 2;                  // w row stride (8-byte rows; 2-way bank conflicts on the w writes)
  static constexpr int SLICE = (32 * WS > B * NC) ? 32 * WS : B * NC;
  // Scalar row of a warp's entry: du dv dA dB dCc dopacity | r g b | depth | 0 0
  // (the layout of the partial row's scalar columns); B + 1 rows per warp,
  // the last one a sink for the sums of no entry.
  static constexpr int GR = 12;
  static_assert(B % JG == 0 && CPL % 2 == 0 && JPL <= 2, "lane grid of the per-warp product");
  // Byte offsets in dynamic shared memory: per-pixel gradient rows, warp
  // slices, geometric warp partials, two staging buffers, the fp32 copy of
  // bf16 feature rows, list entries of the two staged batches.
  static constexpr size_t off_G = 0;
  static constexpr size_t off_slice = off_G + (size_t)kThreads * GS * 4;
  static constexpr size_t off_geo = off_slice + (size_t)8 * SLICE * 4;
  static constexpr size_t off_stage = (off_geo + (size_t)8 * (B + 1) * GR * 4 + 127) / 128 * 128;
  __host__ __device__ static constexpr size_t off_wide(int bf16) { return off_stage + 2 * (size_t)stage_bytes(B, D, bf16); }
  __host__ __device__ static constexpr size_t off_e(int bf16) {
    return off_wide(bf16) + (bf16 ? (size_t)B * D * 4 : 0);
  }
  __host__ __device__ static constexpr size_t smem_bytes(int bf16) { return off_e(bf16) + (size_t)(2 * B + 8 + 4) * 4; }
};

static_assert(BwdCfg<16>::smem_bytes(1) <= 232448 && BwdCfg<32>::smem_bytes(1) <= 232448 &&
                  BwdCfg<64>::smem_bytes(1) <= 232448 && BwdCfg<128>::smem_bytes(1) <= 232448 &&
                  BwdCfg<128>::smem_bytes(0) <= 232448,
              "reverse compositing shared memory per block");
static_assert(2 * (BwdCfg<32>::smem_bytes(1) + 1024) <= 233472, "two reverse blocks per SM at D <= 32");

// Reverse compositing of one tile by the whole block.
template <int D>
__device__ __forceinline__ void bwd_tile(const CompositeArgs& a, const int tile, unsigned char* smem, uint64_t* s_bar,
                                         int* s_abort, StageState& stg) {
  using K = BwdCfg<D>;
  constexpr int B = K::B, NC = K::NC, GS = K::GS, WS = K::WS;
  const bool bf16 = a.feat_bf16 != 0;
  const uint32_t sbytes = stage_bytes(B, D, a.feat_bf16);
  float* s_G = reinterpret_cast<float*>(smem + K::off_G);          // [256][GS]
  float* s_slice = reinterpret_cast<float*>(smem + K::off_slice);  // [8][SLICE]: w[p][j], then P[j][c]
  float* s_geo = reinterpret_cast<float*>(smem + K::off_geo);      // [8][B + 1][GR]
  unsigned char* s_stage = smem + K::off_stage;                     // [2][sbytes]
  float* s_wide = reinterpret_cast<float*>(smem + K::off_wide(a.feat_bf16));
  uint32_t* s_e = reinterpret_cast<uint32_t*>(smem + K::off_e(a.feat_bf16));  // [2][B]
  uint32_t* s_jact = s_e + 2 * B;
  uint32_t* s_maxn = s_jact + 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  int lx, ly;
  tile_pixel(tid, a.tw, lx, ly);
  const int px = tx * a.tw + lx, py = ty * a.th + ly;
  const bool inside = px < a.W && py < a.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const size_t HW = (size_t)a.W * a.H, pix = inside ? (size_t)py * a.W + px : 0;
  const uint2 rg = a.ranges[tile];
  float* grow = s_G + tid * GS;
  float ga = 0.f;
  {
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, gz = 0.f;
    if (inside) {
      if (a.g_rgb) { g0 = a.g_rgb[pix]; g1 = a.g_rgb[HW + pix]; g2 = a.g_rgb[2 * HW + pix]; }
      if (a.g_depth) gz = a.g_depth[pix];
      if (a.g_alpha) ga = a.g_alpha[pix];
    }
    grow[0] = g0; grow[1] = g1; grow[2] = g2; grow[3] = gz;
    if (inside && a.g_feat) {
      const float4* src = reinterpret_cast<const float4*>(a.g_feat + pix * a.out_ld);
#pragma unroll
      for (int d4 = 0; d4 < D / 4; ++d4) {
        const float4 v = __ldg(src + d4);
        grow[4 + 4 * d4] = v.x; grow[5 + 4 * d4] = v.y; grow[6 + 4 * d4] = v.z; grow[7 + 4 * d4] = v.w;
      }
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d) grow[4 + d] = 0.0f;
    }
  }
  for (int i = tid; i < 8 * (B + 1); i += kThreads) {
    s_geo[i * K::GR + 10] = 0.0f;
    s_geo[i * K::GR + 11] = 0.0f;
  }
  float2 G[K::GREG ? NC / 2 : 1];
  if (K::GREG) {
#pragma unroll
    for (int c = 0; c < NC / 2; ++c) G[c] = make_float2(grow[2 * c], grow[2 * c + 1]);
  }
  const float Tf = inside ? a.t_final[pix] : 1.0f;
  const uint32_t nc = inside ? a.n_contrib[pix] : 0u;
  float T = Tf;
  float Q = (grow[0] * a.bg[0] + grow[1] * a.bg[1] + grow[2] * a.bg[2]) * Tf;
  const uint32_t wmax = __reduce_max_sync(0xFFFFFFFFu, nc);
  if (tid == 0) *s_maxn = 0u;
  __syncthreads();
  if (lane == 0 && wmax) atomicMax(s_maxn, wmax);
  __syncthreads();
  // Batches walk [rg.x, rg.x + maxn) backwards: batch k covers
  // [max(rg.x, hi_k - B), hi_k) with hi_k = rg.x + maxn - k B.
  const uint32_t n = *s_maxn;
  const uint32_t nbatch = (n + B - 1) / B;
  // Batches aligned to multiples of B from the tile start (the first one
  // processed, the last in list order, may be short).
  auto batch_lo = [&](uint32_t k) -> uint32_t { return (nbatch - 1 - k) * (uint32_t)B; };
  auto batch_len = [&](uint32_t k) -> int { return (int)min((uint32_t)B, n - batch_lo(k)); };
  // The forward's masks say which entries of each 32-entry group blended in
  // some pixel of this warp; the others are skipped (a 16-entry batch takes
  // its half of the group's word).
  const bool masked = a.cmask != nullptr;
  const size_t cslot0 = (size_t)(rg.x >> 5) + (size_t)tile;
  // List entry and Gaussian of this thread's slot in batch k.
  auto slot = [&](uint32_t k, uint32_t& e, uint32_t& g) {
    e = 0u;
    g = 0u;
    if (k < nbatch && tid < batch_len(k)) {
      const uint32_t p = rg.x + batch_lo(k) + (uint32_t)tid;
      const uint2 eg = __ldg(a.sorted + p);
      e = eg.x;
      g = eg.y;
    }
  };
  // The forward's blend-mask word of this warp for batch k (read a batch
  // ahead, so its global latency overlaps the previous batch).
  auto mask_word = [&](uint32_t k) -> uint32_t {
    return (masked && k < nbatch && batch_lo(k) < wmax)
               ? __ldg(a.cmask + (cslot0 + batch_lo(k) / 32) * 8 + warp) >> (batch_lo(k) & 31u)
               : 0xFFFFFFFFu;
  };
  uint32_t mask_next = mask_word(0);
  uint32_t e_next, g_next;
  slot(0, e_next, g_next);
  uint32_t issued = 0;
  if (nbatch > 0) {
    stage_issue<D>(a, s_stage, B, batch_len(0), g_next, &s_bar[0]);
    if (tid < B) s_e[tid] = e_next;
    issued = 1;
  }
  slot(1, e_next, g_next);
  float* slice = s_slice + warp * K::SLICE;
  for (uint32_t k = 0; k < nbatch; ++k) {
    // Every thread is past batch k-1 (and its combine) here.  A wait on
    // batch k-1 that gave up ends the tile for the whole block (the flag
    // slots alternate by batch, as in the forward).
    __syncthreads();
    if (k > 0 && ((volatile int*)s_abort)[(k - 1) & 1]) break;
    if (k + 1 < nbatch) {
      stage_issue<D>(a, s_stage + ((k + 1) & 1) * (size_t)sbytes, B, batch_len(k + 1), g_next, &s_bar[(k + 1) & 1]);
      if (tid < B) s_e[((k + 1) & 1) * B + tid] = e_next;
      issued = k + 2;
      slot(k + 2, e_next, g_next);
    }
    bool live = true;
    if (!mbar_wait(&s_bar[k & 1], stage_parity(stg, k), a.polls)) {
      ((volatile int*)s_abort)[k & 1] = 1;
      set_err(a.err, kErrTimeout);
      live = false;
    }
    const unsigned char* buf = s_stage + (k & 1) * (size_t)sbytes;
    const float* s_rec = reinterpret_cast<const float*>(buf);
    const float* s_feat = reinterpret_cast<const float*>(buf + (size_t)B * kRec * 4);
    const int nb = batch_len(k);
    if (bf16) {
      if (live) widen_bf16<D>(buf + (size_t)B * kRec * 4, s_wide, nb);
      __syncthreads();
      s_feat = s_wide;
    }
    const uint32_t rel0 = batch_lo(k);
    const uint32_t mask_k = mask_next;
    mask_next = mask_word(k + 1);
    uint32_t jact = 0;
    if (rel0 < wmax) {
      const uint32_t lenmask = nb >= 32 ? 0xFFFFFFFFu : ((1u << nb) - 1u);
      uint32_t todo = mask_k & lenmask;
      // Every lane writes w (0 where it did not blend) for every entry the
      // warp visits; rows of entries it does not visit may hold stale values:
      // the products of those columns are never combined.
      // Entry j given its evaluation (hit: the pixel includes it): the T
      // replay and the gradient terms v (six geometric values, then two
      // zeros), and the blend weight written to the warp's w slice.
      auto entry = [&](int j, bool hit, const PairEval& pe, float (&v)[8]) {
        // Without branches, so that the two entries of a pair interleave:
        // a lane that did not blend takes alpha = 0, which leaves T and Q
        // exactly as they were (1 / (1 - 0) = 1, w = 0), and zero terms.
        const float* rec = s_rec + j * kRec;
        const float al = hit ? pe.alpha : 0.0f;
        const float one_m = 1.0f - al;
        const float inv = __fdividef(1.0f, one_m);  // one_m >= 0.01
        T = T * inv;  // transmittance before this Gaussian
        const float w = al * T;
        // s = g . (rgb, depth, feature) of this Gaussian, in four
        // independent chains of channel pairs (pair i in chain i mod 4).
        const float4 r0 = *reinterpret_cast<const float4*>(rec);      // ., ., A, B
        const float4 r4 = *reinterpret_cast<const float4*>(rec + 4);  // Cc, ., depth, r
        const float4 r8 = *reinterpret_cast<const float4*>(rec + 8);  // g, b, ., .
        const float4* f4 = reinterpret_cast<const float4*>(s_feat + j * D);
        const float2* g2 = reinterpret_cast<const float2*>(grow);
        float2 sc[4];
        sc[0] = __fmul2_rn(K::GREG ? G[0] : g2[0], make_float2(r4.w, r8.x));
        sc[1] = __fmul2_rn(K::GREG ? G[1] : g2[1], make_float2(r8.y, r4.z));
        sc[2] = make_float2(0.0f, 0.0f);
        sc[3] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int d4 = 0; d4 < D / 4; ++d4) {
          const float4 xv = f4[d4];
          const int c0 = 2 + 2 * d4;  // channel pair of xv.x, xv.y
          sc[c0 & 3] = __ffma2_rn(K::GREG ? G[c0] : g2[c0], make_float2(xv.x, xv.y), sc[c0 & 3]);
          sc[(c0 + 1) & 3] = __ffma2_rn(K::GREG ? G[c0 + 1] : g2[c0 + 1], make_float2(xv.z, xv.w), sc[(c0 + 1) & 3]);
        }
        const float2 s01 = __fadd2_rn(sc[0], sc[1]), s23 = __fadd2_rn(sc[2], sc[3]);
        const float2 s2 = __fadd2_rn(s01, s23);
        const float s = s2.x + s2.y;
        const float dalpha = T * s - (Q - ga * Tf) * inv;
        Q = fmaf(w, s, Q);
        // Geometric terms: zero where the pixel did not blend, and all but
        // the opacity term zero where alpha was clamped.
        const bool geo = hit && !pe.clamped;
        const float dp2 = geo ? dalpha * pe.alpha * kLn2 : 0.0f;
        v[0] = -dp2 * (2.0f * r0.z * pe.dx + r0.w * pe.dy);
        v[1] = -dp2 * (2.0f * r4.x * pe.dy + r0.w * pe.dx);
        v[2] = dp2 * pe.dx * pe.dx;
        v[3] = dp2 * pe.dx * pe.dy;
        v[4] = dp2 * pe.dy * pe.dy;
        v[5] = hit ? dalpha * pe.G : 0.0f;
        v[6] = 0.0f;
        v[7] = 0.0f;
        slice[lane * WS + j] = w;
      };
      const int b16 = (lane >> 4) & 1, b8 = (lane >> 3) & 1, b4 = (lane >> 2) & 1, b2 = (lane >> 1) & 1;
      // Warp sums of one entry's v[0..7] (reduce-scatter: lane 4m ends with
      // the sum of index m).
      auto scatter1 = [&](int j, float (&v)[8]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float send = b16 ? v[i] : v[i + 4];
          const float keep = b16 ? v[i + 4] : v[i];
          v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float send = b8 ? v[i] : v[i + 2];
          const float keep = b8 ? v[i + 2] : v[i];
          v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
        }
        {
          const float send = b4 ? v[0] : v[1];
          const float keep = b4 ? v[1] : v[0];
          v[0] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
        }
        v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], 2);
        v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], 1);
        const int m = lane >> 2;
        if ((lane & 3) == 0 && m < 6) s_geo[(warp * (B + 1) + j) * K::GR + m] = v[0];
      };
      // Both entries' sums at once: u = (va, vb), lane 2m ends with the sum
      // of index m (16 shuffles instead of 18, and no warp-wide exchange
      // between the two entries' arithmetic).
      auto scatter2 = [&](int ja, int jb, const float (&va)[8], const float (&vb)[8]) {
        float u[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float send = b16 ? va[i] : vb[i];
          const float keep = b16 ? vb[i] : va[i];
          u[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float send = b8 ? u[i] : u[i + 4];
          const float keep = b8 ? u[i + 4] : u[i];
          u[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float send = b4 ? u[i] : u[i + 2];
          const float keep = b4 ? u[i + 2] : u[i];
          u[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
        }
        {
          const float send = b2 ? u[0] : u[1];
          const float keep = b2 ? u[1] : u[0];
          u[0] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 2);
        }
        u[0] += __shfl_xor_sync(0xFFFFFFFFu, u[0], 1);
        // lane 2m holds index m = 8 b16 + 4 b8 + 2 b4 + b2 of u = (va, vb).
        const int m = lane >> 1, e = m & 7;
        if ((lane & 1) == 0 && e < 6) s_geo[(warp * (B + 1) + (m < 8 ? ja : jb)) * K::GR + e] = u[0];
      };
      auto evaluate = [&](int j, PairEval& pe) -> bool {
        const bool h = eval_pair_flat(s_rec + j * kRec, pxc, pyc, pe);
        return h && live && rel0 + (uint32_t)j < nc;
      };
      // The entries to visit, back to front: with an odd count the first
      // (the latest in list order) alone, then pairs -- both evaluated, then
      // replayed in order (the T chain).  A pair's warp sums are formed
      // after the next pair's arithmetic (the first time, zeros go to the
      // sink row), so the shuffles overlap independent work.
      const int cnt = __popc(todo);
      if (cnt & 1) {
        const int ja = 31 - __clz(todo);
        todo &= ~(1u << ja);
        PairEval pa;
        float va[8];
        const bool ha = evaluate(ja, pa);
        entry(ja, ha, pa, va);
        if (__any_sync(0xFFFFFFFFu, ha)) {
          jact |= 1u << ja;
          scatter1(ja, va);
        }
      }
      float qa[8], qb[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) qa[i] = qb[i] = 0.0f;
      int qja = B, qjb = B;
      for (int n = 0; n < cnt / 2; ++n) {
        const int ja = 31 - __clz(todo);
        todo &= ~(1u << ja);
        const int jb = 31 - __clz(todo);
        todo &= ~(1u << jb);
        PairEval pa, pb;
        float va[8], vb[8];
        const bool ha = evaluate(ja, pa);
        const bool hb = evaluate(jb, pb);
        const bool aa = __any_sync(0xFFFFFFFFu, ha), ab = __any_sync(0xFFFFFFFFu, hb);
        // Neither entry blends in this warp (only without the forward's
        // masks): nothing changes, nothing to sum.
        if (!(aa || ab)) continue;
        entry(ja, ha, pa, va);
        entry(jb, hb, pb, vb);
        jact |= (aa ? 1u << ja : 0u) | (ab ? 1u << jb : 0u);
        scatter2(qja, qjb, qa, qb);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          qa[i] = va[i];
          qb[i] = vb[i];
        }
        qja = ja;
        qjb = jb;
      }
      if (cnt >= 2) scatter2(qja, qjb, qa, qb);
      __syncwarp();
      if (K::JPL == 2 && jact && __popc(jact) <= 16) {
        // At most 16 active entries: lane pair jg takes the jg-th active
        // entry, so one pass covers them all (P rows of inactive entries
        // are left unwritten: the combine reads only active ones).
        constexpr int CP2 = K::CPL / 2;
        const int jg = lane >> 1, cg = lane & 1;
        const bool has = jg < __popc(jact);
        const int jl = has ? (int)__fns(jact, 0, jg + 1) : 0;
        float2 acc[CP2];
#pragma unroll
        for (int c = 0; c < CP2; ++c) acc[c] = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int p = 0; p < 32; ++p) {
          const float wv = has ? slice[p * WS + jl] : 0.0f;
          const float2* gr = reinterpret_cast<const float2*>(s_G + (warp * 32 + p) * GS + cg * K::CPL);
#pragma unroll
          for (int c = 0; c < CP2; ++c) acc[c] = __ffma2_rn(make_float2(wv, wv), gr[c], acc[c]);
        }
        __syncwarp();
        if (has) {
#pragma unroll
          for (int c = 0; c < CP2; ++c) {
            // Colour and depth (the first two pairs) go to the scalar row.
            float* dst = (cg == 0 && c < 2) ? s_geo + (warp * (B + 1) + jl) * K::GR + 6 + 2 * c
                                            : slice + jl * NC + cg * K::CPL + 2 * c;
            *reinterpret_cast<float2*>(dst) = acc[c];
          }
        }
      } else if (jact) {
        // P[j][c] = sum over the warp's pixels of w[p][j] * G[p][c], channel
        // pairs in packed FMAs.
        constexpr int CP2 = K::CPL / 2;
        const int jg = lane >> 1, cg = lane & 1;
        float2 acc[K::JPL][CP2];
#pragma unroll
        for (int jj = 0; jj < K::JPL; ++jj)
#pragma unroll
          for (int c = 0; c < CP2; ++c) acc[jj][c] = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int p = 0; p < 32; ++p) {
          float wv[K::JPL];
          if (K::JPL == 2) {
            const float2 t2 = *reinterpret_cast<const float2*>(slice + p * WS + jg * 2);
            wv[0] = t2.x; wv[1] = t2.y;
          } else {
            wv[0] = slice[p * WS + jg];
          }
          const float2* gr = reinterpret_cast<const float2*>(s_G + (warp * 32 + p) * GS + cg * K::CPL);
#pragma unroll
          for (int c = 0; c < CP2; ++c) {
            const float2 gv = gr[c];
#pragma unroll
            for (int jj = 0; jj < K::JPL; ++jj) acc[jj][c] = __ffma2_rn(make_float2(wv[jj], wv[jj]), gv, acc[jj][c]);
          }
        }
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < K::JPL; ++jj)
#pragma unroll
          for (int c = 0; c < CP2; ++c)
          {
            const int jj2 = jg * K::JPL + jj;
            float* dst = (cg == 0 && c < 2) ? s_geo + (warp * (B + 1) + jj2) * K::GR + 6 + 2 * c
                                            : slice + jj2 * NC + cg * K::CPL + 2 * c;
            *reinterpret_cast<float2*>(dst) = acc[jj][c];
          }
      }
    }
    if (lane == 0) s_jact[warp] = jact;
    __syncthreads();
    // Fixed-order sum of the warp partials: one row per (tile, entry) that
    // some pixel of the tile blended (the other rows stay unwritten and
    // unflagged, i.e. zero).
    const uint32_t* se = s_e + (k & 1) * B;
    uint32_t jm[8], bm = 0;
#pragma unroll
    for (int w8 = 0; w8 < 8; ++w8) {
      jm[w8] = s_jact[w8];
      bm |= jm[w8];
    }
    // One item = four consecutive columns of an active entry's partial row
    // [features | du dv dA dB dCc dopacity | r g b | depth | 0 0]: the warp
    // partials (feature columns from the warp slices, the rest from the
    // warps' scalar rows, which have that layout) summed in warp order, one
    // 16-byte store.  A channel-split pass that is not the first adds its
    // geometric terms (du .. dopacity) to the row the first pass wrote and
    // leaves colour and depth alone.
    // Items over every entry slot (a compile-time count of column groups):
    // slots no pixel blended, and the last group outside the first pass,
    // are skipped.
    constexpr int NQ = D / 4 + 3;
    for (int item = tid; item < B * NQ; item += kThreads) {
      const int j = item / NQ, q4 = item - j * NQ;
      if (!((bm >> j) & 1u) || (!a.aux && q4 == NQ - 1)) continue;
      const bool fcol = q4 < D / 4;
      const float* src = fcol ? s_slice + j * NC + 4 + 4 * q4 : s_geo + j * K::GR + 4 * (q4 - D / 4);
      const int wstride = fcol ? K::SLICE : (B + 1) * K::GR;
      float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int w8 = 0; w8 < 8; ++w8) {
        if ((jm[w8] >> j) & 1u) {
          const float4 v = *reinterpret_cast<const float4*>(src + w8 * wstride);
          acc.x += v.x;
          acc.y += v.y;
          acc.z += v.z;
          acc.w += v.w;
        }
      }
      if ((int64_t)se[j] < a.cap) {
        float* row = a.partials + (size_t)se[j] * a.prow;
        float4* dst = reinterpret_cast<float4*>(q4 < D / 4 ? row + a.pcol0 + 4 * q4 : row + a.pscal + 4 * (q4 - D / 4));
        if (!a.aux && q4 >= D / 4) {
          const float4 prev = *dst;
          acc.x += prev.x;
          acc.y += prev.y;
          if (q4 == D / 4) {
            acc.z += prev.z;
            acc.w += prev.w;
          } else {
            acc.z = prev.z;  // colour: the first pass's
            acc.w = prev.w;
          }
        }
        *dst = acc;
      }
    }
    if (tid < nb && ((bm >> tid) & 1u) && (int64_t)se[tid] < a.cap)
      atomicOr(a.pflags + (se[tid] >> 5), 1u << (se[tid] & 31u));
  }
  stage_drain(stg, s_bar, issued, a.err);
}

// One block per tile.
template <int D>
__global__ void __launch_bounds__(kThreads, D <= 32 ? 2 : 1) composite_bwd_kernel(const CompositeArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_abort[2];
  stage_init(s_bar);
  if (threadIdx.x == 0) s_abort[0] = s_abort[1] = 0;
  __syncthreads();
  StageState stg{{0u, 0u}, false};
  bwd_tile<D>(a, blockIdx.x, smem, s_bar, s_abort, stg);
}

// Persistent form over a batch of views, as the forward's.
template <int D>
__global__ void __launch_bounds__(kThreads, D <= 32 ? 2 : 1)
    composite_bwd_batch_kernel(const __grid_constant__ BatchCompositeArgs ba) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_abort[2], s_item;
  stage_init(s_bar);
  StageState stg{{0u, 0u}, false};
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (int)atomicAdd(ba.queue, 1u);
      s_abort[0] = s_abort[1] = 0;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= ba.nitems || stg.dead) break;
    const int v = batch_view(ba, item);
    bwd_tile<D>(ba.view[v], item - ba.item_start[v], smem, s_bar, s_abort, stg);
  }
}

template <int D, int B, bool kCount>
cudaError_t launch_fwd_t(const CompositeArgs& a, cudaStream_t st) {
  const size_t smem = fwd_smem_bytes(B, D, a.feat_bf16);
  auto k = composite_fwd_kernel<D, B, kCount>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<a.ntiles, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// Batch sizes: 32, 64, 128 Gaussians (128 only up to D = 64); the counting
// form runs with the default batch only.
template <int D>
cudaError_t launch_fwd_d(const CompositeArgs& a, int B, cudaStream_t st) {
  if (B == 0) B = fwd_batch<D>();
  if (a.counts) return B == fwd_batch<D>() ? launch_fwd_t<D, fwd_batch<D>(), true>(a, st) : cudaErrorInvalidValue;
  switch (B) {
    case 32: return launch_fwd_t<D, 32, false>(a, st);
    case 64: return launch_fwd_t<D, 64, false>(a, st);
    case 128:
      if constexpr (D <= 64) return launch_fwd_t<D, 128, false>(a, st);
      break;
  }
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t launch_bwd_t(const CompositeArgs& a, cudaStream_t st) {
  const size_t smem = BwdCfg<D>::smem_bytes(a.feat_bf16);
  auto k = composite_bwd_kernel<D>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<a.ntiles, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// Grid of a persistent launch: as many blocks as fit on the GPU at once
// (occupancy x SMs), never more than there are work items.
template <typename Kern>
cudaError_t persistent_grid(Kern k, size_t smem, int nitems, int& grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess) return e;
  grid = per_sm * sms;
  if (grid > nitems) grid = nitems;
  if (grid < 1) grid = 1;
  return cudaSuccess;
}

template <int D, int B>
cudaError_t launch_fwd_batch_t(const BatchCompositeArgs& b, int bf16, cudaStream_t st) {
  const size_t smem = fwd_smem_bytes(B, D, bf16);
  auto k = composite_fwd_batch_kernel<D, B>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int grid = 1;
  if (e == cudaSuccess) e = persistent_grid(k, smem, b.nitems, grid);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(b);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_fwd_batch_d(const BatchCompositeArgs& b, int bf16, int B, cudaStream_t st) {
  if (B == 0) B = fwd_batch<D>();
  switch (B) {
    case 32: return launch_fwd_batch_t<D, 32>(b, bf16, st);
    case 64: return launch_fwd_batch_t<D, 64>(b, bf16, st);
    case 128:
      if constexpr (D <= 64) return launch_fwd_batch_t<D, 128>(b, bf16, st);
      break;
  }
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t launch_bwd_batch_t(const BatchCompositeArgs& b, int bf16, cudaStream_t st) {
  const size_t smem = BwdCfg<D>::smem_bytes(bf16);
  auto k = composite_bwd_batch_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int grid = 1;
  if (e == cudaSuccess) e = persistent_grid(k, smem, b.nitems, grid);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(b);
  return cudaGetLastError();
}

// D = 256 runs as two passes over 128-channel halves (h = 0, 1): the same
// list, the same per-pixel decisions, each pass staging and accumulating
// its half of every feature row.  Pass 0 owns colour, depth, alpha, T_final,
// n_contrib, the blend masks and (reverse) the colour / depth / alpha /
// background terms; the reverse's geometric terms are linear in the dot
// products g . x, so pass 1 adds the share of its channels to the rows pass
// 0 wrote (same stream, pass 0 first: a fixed order).
CompositeArgs channel_half(const CompositeArgs& a, int h) {
  CompositeArgs c = a;
  const size_t elem = a.feat_bf16 ? 2 : 4;
  c.D = 128;
  c.feat = static_cast<const unsigned char*>(a.feat) + (size_t)h * 128 * elem;
  if (a.out_feat) c.out_feat = a.out_feat + h * 128;
  if (a.out_feat_bf16) c.out_feat_bf16 = a.out_feat_bf16 + h * 128;
  if (a.g_feat) c.g_feat = a.g_feat + h * 128;
  c.pcol0 = a.pcol0 + h * 128;
  if (h > 0) {
    c.aux = 0;
    c.g_rgb = c.g_depth = c.g_alpha = nullptr;
  }
  return c;
}

}  // namespace

bool fwd_batch_supported(int B) { return B == 0 || B == 32 || B == 64 || B == 128; }

cudaError_t launch_composite_fwd(const CompositeArgs& a, int fwd_batch, cudaStream_t st) {
  if (a.ntiles <= 0) return cudaSuccess;
  switch (a.D) {
    case 16: return launch_fwd_d<16>(a, fwd_batch, st);
    case 32: return launch_fwd_d<32>(a, fwd_batch, st);
    case 64: return launch_fwd_d<64>(a, fwd_batch, st);
    case 128: return launch_fwd_d<128>(a, fwd_batch, st);
    case 256: {
      if (a.counts) return launch_fwd_d<128>(channel_half(a, 0), fwd_batch, st);
      const cudaError_t e = launch_fwd_d<128>(channel_half(a, 0), fwd_batch, st);
      return e != cudaSuccess ? e : launch_fwd_d<128>(channel_half(a, 1), fwd_batch, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_composite_bwd(const CompositeArgs& a, cudaStream_t st) {
  if (a.ntiles <= 0) return cudaSuccess;
  switch (a.D) {
    case 16: return launch_bwd_t<16>(a, st);
    case 32: return launch_bwd_t<32>(a, st);
    case 64: return launch_bwd_t<64>(a, st);
    case 128: return launch_bwd_t<128>(a, st);
    case 256: {
      const cudaError_t e = launch_bwd_t<128>(channel_half(a, 0), st);
      return e != cudaSuccess ? e : launch_bwd_t<128>(channel_half(a, 1), st);
    }
  }
  return cudaErrorInvalidValue;
}

// The batch's per-view arguments for channel half h, its own work counter.
static BatchCompositeArgs batch_half(const BatchCompositeArgs& b, int h) {
  BatchCompositeArgs c = b;
  for (int v = 0; v < b.V; ++v) c.view[v] = channel_half(b.view[v], h);
  c.queue = b.queue + 2 * h;
  return c;
}

cudaError_t launch_composite_fwd_batch(const BatchCompositeArgs& b, int D, int feat_bf16, int fwd_batch,
                                       cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
  switch (D) {
    case 16: return launch_fwd_batch_d<16>(b, feat_bf16, fwd_batch, st);
    case 32: return launch_fwd_batch_d<32>(b, feat_bf16, fwd_batch, st);
    case 64: return launch_fwd_batch_d<64>(b, feat_bf16, fwd_batch, st);
    case 128: return launch_fwd_batch_d<128>(b, feat_bf16, fwd_batch, st);
    case 256: {
      const cudaError_t e = launch_fwd_batch_d<128>(batch_half(b, 0), feat_bf16, fwd_batch, st);
      return e != cudaSuccess ? e : launch_fwd_batch_d<128>(batch_half(b, 1), feat_bf16, fwd_batch, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_composite_bwd_batch(const BatchCompositeArgs& b, int D, int feat_bf16, cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
  switch (D) {
    case 16: return launch_bwd_batch_t<16>(b, feat_bf16, st);
    case 32: return launch_bwd_batch_t<32>(b, feat_bf16, st);
    case 64: return launch_bwd_batch_t<64>(b, feat_bf16, st);
    case 128: return launch_bwd_batch_t<128>(b, feat_bf16, st);
    case 256: {
      const cudaError_t e = launch_bwd_batch_t<128>(batch_half(b, 0), feat_bf16, st);
      return e != cudaSuccess ? e : launch_bwd_batch_t<128>(batch_half(b, 1), feat_bf16, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace fe
