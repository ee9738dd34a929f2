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

template <int D>
constexpr int fwd_batch() { return D <= 32 ? 256 : (D <= 64 ? 128 : 64); }

template <int D>
__device__ __forceinline__ void load_feat_row(const void* feat, int bf16, uint32_t g, float* dst) {
  if (bf16) {
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(feat) + (size_t)g * D);
#pragma unroll
    for (int i = 0; i < D / 8; ++i) {
      const uint4 q = __ldg(src + i);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        dst[8 * i + 2 * j] = __uint_as_float(w[j] << 16);
        dst[8 * i + 2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
      }
    }
  } else {
    const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(feat) + (size_t)g * D);
#pragma unroll
    for (int i = 0; i < D / 4; ++i) reinterpret_cast<float4*>(dst)[i] = __ldg(src + i);
  }
}

template <int D, bool kCount>
__global__ void __launch_bounds__(kThreads) composite_fwd_kernel(const CompositeArgs a) {
  constexpr int B = fwd_batch<D>();
  extern __shared__ __align__(16) float smem[];
  float* s_rec = smem;                 // [B][12]
  float* s_feat = smem + B * kRec;     // [B][D]
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int px = tx * a.tw + tid % a.tw, py = ty * a.th + tid / a.tw;
  const bool inside = px < a.W && py < a.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const uint2 rg = a.ranges[tile];
  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Z = 0.f;
  float F[D];
#pragma unroll
  for (int d = 0; d < D; ++d) F[d] = 0.0f;
  uint32_t last = 0;
  uint32_t visits = 0, contribs = 0;  // only used by the counting variant
  bool done = !inside;
  for (uint32_t bs = rg.x; bs < rg.y; bs += B) {
    if (__syncthreads_count(done) == kThreads) break;
    if (tid < B && bs + tid < rg.y) {
      const uint32_t e = a.sorted_e[bs + tid];
      const uint32_t g = a.gid_of_emit[e];
      const float4* r = a.rec + 3 * (size_t)g;
      float4* d = reinterpret_cast<float4*>(s_rec + tid * kRec);
      d[0] = __ldg(r);
      d[1] = __ldg(r + 1);
      d[2] = __ldg(r + 2);
      load_feat_row<D>(a.feat, a.feat_bf16, g, s_feat + tid * D);
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)B, rg.y - bs);
    if (!done) {
      for (int j = 0; j < nb; ++j) {
        const float* rec = s_rec + j * kRec;
        PairEval pe;
        if (kCount) ++visits;
        if (!eval_pair(rec, pxc, pyc, pe)) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, pe.alpha));
        if (Tn < kTMin) {
          done = true;
          break;
        }
        if (kCount) ++contribs;
        const float w = pe.alpha * T;
        C0 = fmaf(w, rec[7], C0);
        C1 = fmaf(w, rec[8], C1);
        C2 = fmaf(w, rec[9], C2);
        Z = fmaf(w, rec[6], Z);
        const float4* f4 = reinterpret_cast<const float4*>(s_feat + j * D);
#pragma unroll
        for (int d4 = 0; d4 < D / 4; ++d4) {
          const float4 f = f4[d4];
          F[4 * d4] = fmaf(w, f.x, F[4 * d4]);
          F[4 * d4 + 1] = fmaf(w, f.y, F[4 * d4 + 1]);
          F[4 * d4 + 2] = fmaf(w, f.z, F[4 * d4 + 2]);
          F[4 * d4 + 3] = fmaf(w, f.w, F[4 * d4 + 3]);
        }
        T = Tn;
        last = bs - rg.x + (uint32_t)j + 1u;
      }
    }
  }
  if (kCount) {
    // Block sums of the pair counts, one 64-bit atomic per block.
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
    a.out_rgb[p] = C0 + T * a.bg[0];
    a.out_rgb[HW + p] = C1 + T * a.bg[1];
    a.out_rgb[2 * HW + p] = C2 + T * a.bg[2];
    a.out_depth[p] = Z;
    a.out_alpha[p] = 1.0f - T;
    float4* fo = reinterpret_cast<float4*>(a.out_feat + p * D);
#pragma unroll
    for (int d4 = 0; d4 < D / 4; ++d4) fo[d4] = make_float4(F[4 * d4], F[4 * d4 + 1], F[4 * d4 + 2], F[4 * d4 + 3]);
    a.t_final[p] = T;
    a.n_contrib[p] = last;
  }
}

// ---------------------------------------------------------------------------
constexpr int kBwdBatch = 8;
constexpr int kPairStride = kThreads + 1;  // padded row of per-pixel terms

template <int D>
constexpr size_t bwd_smem_floats() {
  return (size_t)kBwdBatch * kRec + (size_t)kBwdBatch * D + (size_t)kThreads * (4 + D + 1) +
         (size_t)7 * kBwdBatch * kPairStride + kBwdBatch + 4;
}

template <int D>
__global__ void __launch_bounds__(kThreads) composite_bwd_kernel(const CompositeArgs a) {
  constexpr int B = kBwdBatch;
  constexpr int GS = 4 + D + 1;  // row stride of the per-pixel upstream gradients
  constexpr int NP = kPartialScalars + D;
  extern __shared__ __align__(16) float smem[];
  float* s_rec = smem;
  float* s_feat = s_rec + B * kRec;
  float* s_G = s_feat + B * D;
  float* s_pair = s_G + kThreads * GS;
  uint32_t* s_e = reinterpret_cast<uint32_t*>(s_pair + 7 * B * kPairStride);
  uint32_t* s_maxn = s_e + B;
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int px = tx * a.tw + tid % a.tw, py = ty * a.th + tid / a.tw;
  const bool inside = px < a.W && py < a.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const size_t HW = (size_t)a.W * a.H, pix = inside ? (size_t)py * a.W + px : 0;
  const uint2 rg = a.ranges[tile];
  float gr0 = 0.f, gr1 = 0.f, gr2 = 0.f, gz = 0.f, ga = 0.f;
  float* gF = s_G + tid * GS + 4;
  if (inside) {
    if (a.g_rgb) { gr0 = a.g_rgb[pix]; gr1 = a.g_rgb[HW + pix]; gr2 = a.g_rgb[2 * HW + pix]; }
    if (a.g_depth) gz = a.g_depth[pix];
    if (a.g_alpha) ga = a.g_alpha[pix];
  }
  s_G[tid * GS + 0] = gr0;
  s_G[tid * GS + 1] = gr1;
  s_G[tid * GS + 2] = gr2;
  s_G[tid * GS + 3] = gz;
  if (inside && a.g_feat) {
    const float4* src = reinterpret_cast<const float4*>(a.g_feat + pix * D);
#pragma unroll
    for (int d4 = 0; d4 < D / 4; ++d4) {
      const float4 v = __ldg(src + d4);
      gF[4 * d4] = v.x; gF[4 * d4 + 1] = v.y; gF[4 * d4 + 2] = v.z; gF[4 * d4 + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) gF[d] = 0.0f;
  }
  const float Tf = inside ? a.t_final[pix] : 1.0f;
  const uint32_t nc = inside ? a.n_contrib[pix] : 0u;
  float T = Tf;
  float Q = (gr0 * a.bg[0] + gr1 * a.bg[1] + gr2 * a.bg[2]) * Tf;
  if (tid == 0) *s_maxn = 0u;
  __syncthreads();
  if (nc) atomicMax(s_maxn, nc);
  __syncthreads();
  const uint32_t end = rg.x + *s_maxn;
  for (uint32_t be = end; be > rg.x;) {
    const uint32_t bs = be - rg.x > (uint32_t)B ? be - B : rg.x;
    const int nb = (int)(be - bs);
    __syncthreads();
    if (tid < nb) {
      const uint32_t e = a.sorted_e[bs + tid];
      const uint32_t g = a.gid_of_emit[e];
      s_e[tid] = e;
      const float4* r = a.rec + 3 * (size_t)g;
      float4* d = reinterpret_cast<float4*>(s_rec + tid * kRec);
      d[0] = __ldg(r);
      d[1] = __ldg(r + 1);
      d[2] = __ldg(r + 2);
      load_feat_row<D>(a.feat, a.feat_bf16, g, s_feat + tid * D);
    }
    __syncthreads();
    for (int j = nb - 1; j >= 0; --j) {
      const uint32_t rel = bs - rg.x + (uint32_t)j;
      float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f, w = 0.f;
      if (rel < nc) {
        const float* rec = s_rec + j * kRec;
        PairEval pe;
        if (eval_pair(rec, pxc, pyc, pe)) {
          const float one_m = 1.0f - pe.alpha;
          T = T / one_m;  // transmittance before this Gaussian
          w = pe.alpha * T;
          const float* fj = s_feat + j * D;
          float s = gr0 * rec[7] + gr1 * rec[8] + gr2 * rec[9] + gz * rec[6];
#pragma unroll
          for (int d = 0; d < D; ++d) s = fmaf(gF[d], fj[d], s);
          const float dalpha = T * s - (Q - ga * Tf) / one_m;
          Q = fmaf(w, s, Q);
          if (!pe.clamped) {
            const float dp2 = dalpha * pe.alpha * kLn2;
            du = -dp2 * (2.0f * rec[2] * pe.dx + rec[3] * pe.dy);
            dv = -dp2 * (2.0f * rec[4] * pe.dy + rec[3] * pe.dx);
            dA = dp2 * pe.dx * pe.dx;
            dB = dp2 * pe.dx * pe.dy;
            dC = dp2 * pe.dy * pe.dy;
            dop = dalpha * pe.G;
          }
        }
      }
      float* sp = s_pair + j * kPairStride + tid;
      sp[0 * B * kPairStride] = du;
      sp[1 * B * kPairStride] = dv;
      sp[2 * B * kPairStride] = dA;
      sp[3 * B * kPairStride] = dB;
      sp[4 * B * kPairStride] = dC;
      sp[5 * B * kPairStride] = dop;
      sp[6 * B * kPairStride] = w;
    }
    __syncthreads();
    // Fixed-order sums over the tile's 256 pixels.
    for (int item = tid; item < nb * NP; item += kThreads) {
      const int j = item / NP, k = item - j * NP;
      float acc = 0.0f;
      if (k < 6) {
        const float* row = s_pair + (k * B + j) * kPairStride;
#pragma unroll 8
        for (int p = 0; p < kThreads; ++p) acc += row[p];
      } else {
        const float* wr = s_pair + (6 * B + j) * kPairStride;
        const float* gc = s_G + (k - 6);
#pragma unroll 8
        for (int p = 0; p < kThreads; ++p) acc = fmaf(wr[p], gc[p * GS], acc);
      }
      a.partials[(size_t)s_e[j] * NP + k] = acc;
    }
    if (tid < nb) a.pflags[s_e[tid]] = 1;
    be = bs;
  }
}

template <int D>
cudaError_t launch_fwd_t(const CompositeArgs& a, cudaStream_t st) {
  constexpr int B = fwd_batch<D>();
  const size_t smem = (size_t)B * (kRec + D) * sizeof(float);
  auto k = a.counts ? composite_fwd_kernel<D, true> : composite_fwd_kernel<D, false>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<a.ntiles, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_bwd_t(const CompositeArgs& a, cudaStream_t st) {
  const size_t smem = bwd_smem_floats<D>() * sizeof(float);
  auto k = composite_bwd_kernel<D>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<a.ntiles, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_composite_fwd(const CompositeArgs& a, cudaStream_t st) {
  if (a.ntiles <= 0) return cudaSuccess;
  switch (a.D) {
    case 16: return launch_fwd_t<16>(a, st);
    case 32: return launch_fwd_t<32>(a, st);
    case 64: return launch_fwd_t<64>(a, st);
    case 128: return launch_fwd_t<128>(a, st);
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
  }
  return cudaErrorInvalidValue;
}

}  // namespace fe
