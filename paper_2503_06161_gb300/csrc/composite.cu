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
      float4* d = reinterpret_cast<float4*>(s_rec + tid * kRec);
      if ((int64_t)e < a.cap) {
        const uint32_t g = a.gid_of_emit[e];
        const float4* r = a.rec + 3 * (size_t)g;
        d[0] = __ldg(r);
        d[1] = __ldg(r + 1);
        d[2] = __ldg(r + 2);
        load_feat_row<D>(a.feat, a.feat_bf16, g, s_feat + tid * D);
      } else {
        d[2] = make_float4(0.f, 0.f, -1.0f, 0.f);  // radius -1: never included
      }
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
  static constexpr int JG = 8, CG = 4;              // lane grid of the per-warp product
  static constexpr int JPL = B / JG;                // entries per lane
  static constexpr int CPL = NC / CG;               // channels per lane
  static constexpr bool GREG = D <= 32;             // upstream gradients kept in registers
  static constexpr int GS = NC + 1;                 // per-pixel gradient row stride (odd)
  static constexpr int WS = B + 4;                  // w row stride (16-byte rows)
  static constexpr int SLICE = (32 * WS > B * NC) ? 32 * WS : B * NC;
  static constexpr size_t smem_floats() {
    return (size_t)B * kRec + (size_t)B * NC + (size_t)kThreads * GS + (size_t)8 * SLICE + (size_t)8 * B * 8 + B +
           8 + 4;
  }
};

template <int D>
__global__ void __launch_bounds__(kThreads) composite_bwd_kernel(const CompositeArgs a) {
  using K = BwdCfg<D>;
  constexpr int B = K::B, NC = K::NC, GS = K::GS, WS = K::WS, NP = partial_stride(D);
  constexpr int NV = kPartialScalars + D;  // values per row
  extern __shared__ __align__(16) float smem[];
  float* s_rec = smem;                       // [B][12]
  float* s_x = s_rec + B * kRec;             // [B][NC]: rgb, depth, z
  float* s_G = s_x + B * NC;                 // [256][GS]
  float* s_slice = s_G + kThreads * GS;      // [8][SLICE]: w[p][j], then P[j][c]
  float* s_geo = s_slice + 8 * K::SLICE;     // [8][B][8]
  uint32_t* s_e = reinterpret_cast<uint32_t*>(s_geo + 8 * B * 8);
  uint32_t* s_jact = s_e + B;
  uint32_t* s_maxn = s_jact + 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int px = tx * a.tw + tid % a.tw, py = ty * a.th + tid / a.tw;
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
      const float4* src = reinterpret_cast<const float4*>(a.g_feat + pix * D);
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
  float G[K::GREG ? NC : 1];
  if (K::GREG) {
#pragma unroll
    for (int c = 0; c < NC; ++c) G[c] = grow[c];
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
  const uint32_t end = rg.x + *s_maxn;
  float* slice = s_slice + warp * K::SLICE;
  for (uint32_t be = end; be > rg.x;) {
    const uint32_t bs = be - rg.x > (uint32_t)B ? be - B : rg.x;
    const int nb = (int)(be - bs);
    __syncthreads();
    if (tid < nb) {
      const uint32_t e = a.sorted_e[bs + tid];
      float4* d = reinterpret_cast<float4*>(s_rec + tid * kRec);
      s_e[tid] = e;
      if ((int64_t)e < a.cap) {
        const uint32_t g = a.gid_of_emit[e];
        const float4* r = a.rec + 3 * (size_t)g;
        const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2);
        d[0] = r0; d[1] = r1; d[2] = r2;
        float* x = s_x + tid * NC;
        x[0] = r1.w; x[1] = r2.x; x[2] = r2.y; x[3] = r1.z;  // rgb, depth
        load_feat_row<D>(a.feat, a.feat_bf16, g, x + 4);
      } else {
        d[2] = make_float4(0.f, 0.f, -1.0f, 0.f);  // radius -1: never included
      }
    }
    __syncthreads();
    const uint32_t rel0 = bs - rg.x;
    uint32_t jact = 0;
    if (rel0 < wmax) {
      for (int j = nb - 1; j >= 0; --j) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0f;
        float w = 0.0f;
        bool contrib = false;
        if (rel0 + (uint32_t)j < nc) {
          const float* rec = s_rec + j * kRec;
          PairEval pe;
          if (eval_pair(rec, pxc, pyc, pe)) {
            contrib = true;
            const float one_m = 1.0f - pe.alpha;
            const float inv = __fdividef(1.0f, one_m);  // one_m >= 0.01
            T = T * inv;  // transmittance before this Gaussian
            w = pe.alpha * T;
            const float4* x4 = reinterpret_cast<const float4*>(s_x + j * NC);
            float s = 0.0f;
#pragma unroll
            for (int c4 = 0; c4 < NC / 4; ++c4) {
              const float4 xv = x4[c4];
              if (K::GREG) {
                s = fmaf(G[4 * c4], xv.x, s);
                s = fmaf(G[4 * c4 + 1], xv.y, s);
                s = fmaf(G[4 * c4 + 2], xv.z, s);
                s = fmaf(G[4 * c4 + 3], xv.w, s);
              } else {
                s = fmaf(grow[4 * c4], xv.x, s);
                s = fmaf(grow[4 * c4 + 1], xv.y, s);
                s = fmaf(grow[4 * c4 + 2], xv.z, s);
                s = fmaf(grow[4 * c4 + 3], xv.w, s);
              }
            }
            const float dalpha = T * s - (Q - ga * Tf) * inv;
            Q = fmaf(w, s, Q);
            if (!pe.clamped) {
              const float dp2 = dalpha * pe.alpha * kLn2;
              v[0] = -dp2 * (2.0f * rec[2] * pe.dx + rec[3] * pe.dy);
              v[1] = -dp2 * (2.0f * rec[4] * pe.dy + rec[3] * pe.dx);
              v[2] = dp2 * pe.dx * pe.dx;
              v[3] = dp2 * pe.dx * pe.dy;
              v[4] = dp2 * pe.dy * pe.dy;
              v[5] = dalpha * pe.G;
            }
          }
        }
        slice[lane * WS + j] = w;
        if (__ballot_sync(0xFFFFFFFFu, contrib)) {
          jact |= 1u << j;
          // Reduce-scatter of v[0..7] over the warp: lane 4m ends with index m.
          const int b16 = (lane >> 4) & 1, b8 = (lane >> 3) & 1, b4 = (lane >> 2) & 1;
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
          if ((lane & 3) == 0 && m < 6) s_geo[(warp * B + j) * 8 + m] = v[0];
        }
      }
      __syncwarp();
      if (jact) {
        // P[j][c] = sum over the warp's pixels of w[p][j] * G[p][c].
        const int jg = lane >> 2, cg = lane & 3;
        float acc[K::JPL][K::CPL];
#pragma unroll
        for (int jj = 0; jj < K::JPL; ++jj)
#pragma unroll
          for (int c = 0; c < K::CPL; ++c) acc[jj][c] = 0.0f;
#pragma unroll 4
        for (int p = 0; p < 32; ++p) {
          float wv[K::JPL];
          if (K::JPL == 4) {
            const float4 t4 = *reinterpret_cast<const float4*>(slice + p * WS + jg * 4);
            wv[0] = t4.x; wv[1] = t4.y; wv[2] = t4.z; wv[3] = t4.w;
          } else {
            const float2 t2 = *reinterpret_cast<const float2*>(slice + p * WS + jg * 2);
            wv[0] = t2.x; wv[1] = t2.y;
          }
          const float* gr = s_G + (warp * 32 + p) * GS + cg * K::CPL;
#pragma unroll
          for (int c = 0; c < K::CPL; ++c) {
            const float gv = gr[c];
#pragma unroll
            for (int jj = 0; jj < K::JPL; ++jj) acc[jj][c] = fmaf(wv[jj], gv, acc[jj][c]);
          }
        }
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < K::JPL; ++jj)
#pragma unroll
          for (int c = 0; c < K::CPL; ++c) slice[(jg * K::JPL + jj) * NC + cg * K::CPL + c] = acc[jj][c];
      }
    }
    if (lane == 0) s_jact[warp] = jact;
    __syncthreads();
    // Fixed-order sum of the warp partials: one row per (tile, entry).
    for (int item = tid; item < nb * NV; item += kThreads) {
      // k: 0..5 geometric terms, 6..9 rgb/depth, 10.. features; row index
      // puts the features first.
      const int j = item / NV, k = item - j * NV;
      float acc = 0.0f;
#pragma unroll
      for (int w8 = 0; w8 < 8; ++w8) {
        if ((s_jact[w8] >> j) & 1u)
          acc += k < 6 ? s_geo[(w8 * B + j) * 8 + k] : s_slice[w8 * K::SLICE + j * NC + (k - 6)];
      }
      const int col = k < kPartialScalars ? D + k : k - kPartialScalars;
      if ((int64_t)s_e[j] < a.cap) a.partials[(size_t)s_e[j] * NP + col] = acc;
    }
    if (tid < nb && (int64_t)s_e[tid] < a.cap) atomicOr(a.pflags + (s_e[tid] >> 5), 1u << (s_e[tid] & 31u));
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
  const size_t smem = BwdCfg<D>::smem_floats() * sizeof(float);
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
