// Adaptive density control (the 3D Gaussian splatting lineage's procedure,
// whose intervals and percent-dense fraction the paper's appendix
// hyperparameter table gives): screen-space gradient statistics, clone /
// split / prune with a deterministic output order, and the opacity reset.
//
// fe_densify runs three kernels: decide (one decision per Gaussian and
// per-block counts of survivors, clones and splits), scan (one block:
// exclusive offsets of every block, in block order) and scatter (one block
// per 256 Gaussians and attribute stream, writing each Gaussian's rows to
// their final places).  The output order is fixed by the scans, so the
// result does not depend on scheduling.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace fe {

namespace {

constexpr int kDT = 256;        // threads per block
constexpr int kMaxAttrs = 32;
constexpr int kSplitN = 2;

struct AttrDev {
  const void* src;
  void* dst;
  int width, elem_bytes, role;
  int unit;   // bytes moved per access: 16, 8, 4 or 2 (4 with float arithmetic for MEANS / LOG_SCALES)
  int wu;     // units per row
};

struct DensArgs {
  int P;
  const float *means, *log_scales, *quats, *logits, *accum;
  const int32_t* count;
  const float* normals;
  // Thresholds moved into the inputs' domains on the host (in double,
  // rounded once): sigmoid(x) < m <=> x < logit(m) and
  // max exp(ls) > s <=> max ls > log(s), so a decision needs one division
  // and three comparisons and no transcendental.
  float grad_thresh, logit_min, log_dense;
  AttrDev attrs[kMaxAttrs];
  int nattrs;
  int8_t* dec;      // [P] decision: -1 prune, 0 keep, 1 clone, 2 split
  int* blk;         // [nblk][3]: counts of survivors, clones, splits; then exclusive offsets
  int* tot;         // [3] totals
  int64_t* new_P;
};

__device__ __forceinline__ int decide(const DensArgs& a, int g) {
  if (a.logits[g] < a.logit_min) return -1;
  const int c = a.count[g];
  const float avg = c > 0 ? a.accum[g] / (float)c : 0.0f;
  if (!(avg >= a.grad_thresh)) return 0;
  const float* ls = a.log_scales + (size_t)g * 3;
  return fmaxf(fmaxf(ls[0], ls[1]), ls[2]) > a.log_dense ? 2 : 1;
}

// Inclusive block sum of v over kDT threads (fixed order); s: kDT/32 ints.
__device__ __forceinline__ int block_prefix(int v, int* s, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s[warp] = x;
  __syncthreads();
  int base = 0;
  total = 0;
  for (int w = 0; w < kDT / 32; ++w) {
    if (w < warp) base += s[w];
    total += s[w];
  }
  __syncthreads();
  return base + x;  // inclusive
}

__global__ void __launch_bounds__(kDT) densify_decide_kernel(const DensArgs a) {
  __shared__ int s[3][kDT / 32];
  const int g = blockIdx.x * kDT + threadIdx.x;
  int d = -1;
  if (g < a.P) {
    d = decide(a, g);
    a.dec[g] = (int8_t)d;
  }
  int tk, tc, ts;
  block_prefix(d == 0 || d == 1, s[0], tk);
  block_prefix(d == 1, s[1], tc);
  block_prefix(d == 2, s[2], ts);
  if (threadIdx.x == 0) {
    a.blk[blockIdx.x * 3] = tk;
    a.blk[blockIdx.x * 3 + 1] = tc;
    a.blk[blockIdx.x * 3 + 2] = ts;
  }
}

// One block: exclusive offsets of every block, in block order, per category.
__global__ void __launch_bounds__(1024) densify_scan_kernel(const DensArgs a, int nblk) {
  __shared__ int s_w[32];
  __shared__ int s_carry[3];
  if (threadIdx.x < 3) s_carry[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; ++k) {
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
      const int b = b0 + threadIdx.x;
      const int v = b < nblk ? a.blk[b * 3 + k] : 0;
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_w[warp] = x;
      __syncthreads();
      int base = s_carry[k];
      for (int w = 0; w < warp; ++w) base += s_w[w];
      if (b < nblk) a.blk[b * 3 + k] = base + x - v;  // exclusive
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 32; ++w) t += s_w[w];
        s_carry[k] += t;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    a.tot[0] = s_carry[0];
    a.tot[1] = s_carry[1];
    a.tot[2] = s_carry[2];
    *a.new_P = (int64_t)s_carry[0] + s_carry[1] + (int64_t)kSplitN * s_carry[2];
  }
}

// One block per (256 Gaussians, attribute): the rows of the block's
// Gaussians -- survivor row, clone row and first split child row -- and the
// decision are staged in shared memory by the thread that owns the Gaussian
// (with the split children's centre offsets R(q)(s * n_i) for the MEANS
// attribute); then the attribute is moved with the block's threads laid over
// (row, unit) pairs, units fastest, so that the reads of the block's
// contiguous source rows and the writes of consecutive destination rows are
// coalesced whatever the attribute's width.  A grid of (tiles x attributes)
// blocks runs many waves, so the last wave's tail is short.
struct ScatterSmem {
  uint32_t row[3][kDT];            // survivor, clone, first split child
  float off[kSplitN * 3][kDT];     // child centre offsets
  int8_t d[kDT];
};

// Moves one attribute's rows in units U (16, 8, 4 or 2 bytes); ARITH: the
// float MEANS / LOG_SCALES roles, whose split children are computed.  Each
// thread loads up to 64 bytes (rows j, j + R, ...; at most 8 units) before
// storing any, so that enough bytes are in flight to cover the latency.
template <typename U>
constexpr int unroll_of() { return 64 / (int)sizeof(U) > 8 ? 8 : 64 / (int)sizeof(U); }

template <typename U, bool ARITH>
__device__ __forceinline__ void store_rows(const AttrDev& at, const ScatterSmem& sm, U* dst, int j, int c, U v,
                                           float shrink) {
  const int d = sm.d[j];
  const size_t WU = (size_t)at.wu;
  const U z{};
  if (d <= 1) {
    dst[sm.row[0][j] * WU + c] = v;
    if (d == 1) dst[sm.row[1][j] * WU + c] = at.role == FE_ATTR_STATE ? z : v;
    return;
  }
#pragma unroll
  for (int i = 0; i < kSplitN; ++i) {
    U o = at.role == FE_ATTR_STATE ? z : v;
    if constexpr (ARITH) o = at.role == FE_ATTR_MEANS ? v + sm.off[i * 3 + c][j] : v + shrink;
    dst[(sm.row[2][j] + i) * WU + c] = o;
  }
}

template <typename U, bool ARITH>
__device__ __forceinline__ void move_attr(const AttrDev& at, const ScatterSmem& sm, int g0, int nrows, float shrink) {
  const int WU = at.wu;
  const U* src = reinterpret_cast<const U*>(static_cast<const char*>(at.src) + (size_t)g0 * at.width * at.elem_bytes);
  U* dst = static_cast<U*>(at.dst);
  if (WU <= kDT) {
    const int R = kDT / WU;  // rows per pass
    const int j0 = threadIdx.x / WU, c = threadIdx.x - j0 * WU;
    if (j0 >= R) return;
    constexpr int kUnroll = unroll_of<U>();
    for (int jb = j0; jb < nrows; jb += R * kUnroll) {
      U v[kUnroll];
      bool live[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int j = jb + u * R;
        live[u] = j < nrows && sm.d[j] >= 0;
        if (live[u]) v[u] = src[(size_t)j * WU + c];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (live[u]) store_rows<U, ARITH>(at, sm, dst, jb + u * R, c, v[u], shrink);
    }
  } else {
    for (int j = 0; j < nrows; ++j) {
      if (sm.d[j] < 0) continue;
      for (int c = threadIdx.x; c < WU; c += kDT) store_rows<U, ARITH>(at, sm, dst, j, c, src[(size_t)j * WU + c], shrink);
    }
  }
}

__global__ void __launch_bounds__(kDT) densify_scatter_kernel(const DensArgs a) {
  __shared__ int s[3][kDT / 32];
  __shared__ ScatterSmem sm;
  const int g0 = blockIdx.x * kDT;
  const int g = g0 + threadIdx.x;
  const int d = g < a.P ? (int)a.dec[g] : -1;
  int tk, tc, ts;
  const int ik = block_prefix(d == 0 || d == 1, s[0], tk) - (d == 0 || d == 1);
  const int ic = block_prefix(d == 1, s[1], tc) - (d == 1);
  const int is = block_prefix(d == 2, s[2], ts) - (d == 2);
  const uint32_t K = (uint32_t)a.tot[0], C = (uint32_t)a.tot[1];
  sm.d[threadIdx.x] = (int8_t)d;
  sm.row[0][threadIdx.x] = (uint32_t)(a.blk[blockIdx.x * 3] + ik);
  sm.row[1][threadIdx.x] = K + (uint32_t)(a.blk[blockIdx.x * 3 + 1] + ic);
  sm.row[2][threadIdx.x] = K + C + (uint32_t)kSplitN * (uint32_t)(a.blk[blockIdx.x * 3 + 2] + is);
  const AttrDev& at = a.attrs[blockIdx.y];
  if (d == 2 && at.role == FE_ATTR_MEANS) {
    // Rotation of the (normalised) quaternion applied to s * n_i.
    const float* q = a.quats + (size_t)g * 4;
    const float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] * n, x = q[1] * n, y = q[2] * n, z = q[3] * n;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = expf(a.log_scales[(size_t)g * 3 + k]);
#pragma unroll
    for (int i = 0; i < kSplitN; ++i) {
      const float* nv = a.normals + ((size_t)g * kSplitN + i) * 3;
      const float v0 = sc[0] * nv[0], v1 = sc[1] * nv[1], v2 = sc[2] * nv[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.off[i * 3 + k][threadIdx.x] = R[3 * k] * v0 + R[3 * k + 1] * v1 + R[3 * k + 2] * v2;
    }
  }
  __syncthreads();
  const int nrows = min(kDT, a.P - g0);
  const float shrink = logf(1.0f / (0.8f * (float)kSplitN));
  if (at.role == FE_ATTR_MEANS || at.role == FE_ATTR_LOG_SCALES) move_attr<float, true>(at, sm, g0, nrows, shrink);
  else if (at.unit == 16) move_attr<uint4, false>(at, sm, g0, nrows, shrink);
  else if (at.unit == 8) move_attr<uint2, false>(at, sm, g0, nrows, shrink);
  else if (at.unit == 4) move_attr<uint32_t, false>(at, sm, g0, nrows, shrink);
  else move_attr<uint16_t, false>(at, sm, g0, nrows, shrink);
}

__global__ void reset_opacity_kernel(float* logits, int64_t P, float cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    logits[i] = fminf(logits[i], cap);
}

// A Gaussian is in view when the projection wrote its record (radius > 0).
__global__ void screen_stats_kernel(const float4* __restrict__ rec, const float* __restrict__ psum, int P,
                                    float sx, float sy, float* accum, int32_t* count) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P || !(rec[3 * (size_t)g + 2].z > 0.0f)) return;
  const float du = psum[(size_t)g * 12] * sx, dv = psum[(size_t)g * 12 + 1] * sy;
  accum[g] += sqrtf(du * du + dv * dv);
  count[g] += 1;
}

int ceil_blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }
size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

cudaError_t launch_screen_stats(const float4* rec, const float* psum, int P, int W, int H, float* accum,
                                int32_t* count, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  screen_stats_kernel<<<ceil_blocks(P, 256), 256, 0, st>>>(rec, psum, P, 0.5f * (float)W, 0.5f * (float)H,
                                                           accum, count);
  return cudaGetLastError();
}

}  // namespace fe

using namespace fe;

extern "C" size_t fe_densify_workspace_size(int P) {
  if (P < 0) return 0;
  const int nblk = ceil_blocks(P, kDT) + 1;
  return al256((size_t)P) + al256((size_t)nblk * 3 * 4) + 256;
}

extern "C" fe_status fe_densify(const fe_densify_args* args, int64_t* new_P, void* workspace,
                                size_t workspace_bytes, void* stream) {
  if (!args || !new_P || args->P < 0 || args->nattrs < 1 || args->nattrs > kMaxAttrs || !args->attrs)
    return FE_ERR_INVALID_ARG;
  const int P = args->P;
  if (args->capacity < (int64_t)kSplitN * P) return FE_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < fe_densify_workspace_size(P)) return FE_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 16) return FE_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P == 0) return cudaMemsetAsync(new_P, 0, sizeof(int64_t), st) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
  if (!args->means || !args->log_scales || !args->quats || !args->opacity_logits || !args->accum || !args->count ||
      !args->normals)
    return FE_ERR_INVALID_ARG;
  for (const void* p : {(const void*)args->means, (const void*)args->log_scales, (const void*)args->quats,
                        (const void*)args->opacity_logits, (const void*)args->accum, (const void*)args->count,
                        (const void*)args->normals})
    if (reinterpret_cast<uintptr_t>(p) % 4) return FE_ERR_INVALID_ARG;
  DensArgs a{};
  a.P = P;
  a.means = args->means;
  a.log_scales = args->log_scales;
  a.quats = args->quats;
  a.logits = args->opacity_logits;
  a.accum = args->accum;
  a.count = args->count;
  a.normals = args->normals;
  if (std::isnan(args->grad_thresh) || std::isnan(args->dense_scale) || std::isnan(args->min_opacity))
    return FE_ERR_INVALID_ARG;
  a.grad_thresh = args->grad_thresh;
  const double m = args->min_opacity, ds = args->dense_scale;
  a.logit_min = m <= 0.0 ? -INFINITY : m >= 1.0 ? INFINITY : (float)std::log(m / (1.0 - m));
  a.log_dense = ds <= 0.0 ? -INFINITY : (float)std::log(ds);
  a.nattrs = args->nattrs;
  for (int t = 0; t < args->nattrs; ++t) {
    const fe_attr& at = args->attrs[t];
    if (!at.src || !at.dst || at.src == at.dst || at.width < 1 || (at.elem_bytes != 4 && at.elem_bytes != 2) ||
        at.role < FE_ATTR_COPY || at.role > FE_ATTR_STATE ||
        (reinterpret_cast<uintptr_t>(at.src) | reinterpret_cast<uintptr_t>(at.dst)) % at.elem_bytes)
      return FE_ERR_INVALID_ARG;
    if ((at.role == FE_ATTR_MEANS || at.role == FE_ATTR_LOG_SCALES) && (at.width != 3 || at.elem_bytes != 4))
      return FE_ERR_INVALID_ARG;
    // Widest access that every row start of src and dst allows.
    const size_t row = (size_t)at.width * at.elem_bytes;
    const uintptr_t base = reinterpret_cast<uintptr_t>(at.src) | reinterpret_cast<uintptr_t>(at.dst);
    int unit = at.elem_bytes;
    if (at.role == FE_ATTR_COPY || at.role == FE_ATTR_STATE)
      for (int u : {16, 8, 4})
        if (u > unit && row % u == 0 && base % u == 0) {
          unit = u;
          break;
        }
    a.attrs[t] = AttrDev{at.src, at.dst, at.width, at.elem_bytes, at.role, unit, (int)(row / unit)};
  }
  const int nblk = ceil_blocks(P, kDT);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  a.dec = reinterpret_cast<int8_t*>(ws);
  a.blk = reinterpret_cast<int*>(ws + al256((size_t)P));
  a.tot = reinterpret_cast<int*>(ws + al256((size_t)P) + al256((size_t)(nblk + 1) * 3 * 4));
  a.new_P = new_P;
  densify_decide_kernel<<<nblk, kDT, 0, st>>>(a);
  densify_scan_kernel<<<1, 1024, 0, st>>>(a, nblk);
  densify_scatter_kernel<<<dim3(nblk, a.nattrs), kDT, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" fe_status fe_reset_opacity(float* logits, int64_t P, float max_opacity, void* stream) {
  if (P < 0 || !(max_opacity > 0.0f && max_opacity < 1.0f) || (P > 0 && !logits)) return FE_ERR_INVALID_ARG;
  if (P == 0) return FE_OK;
  const float cap = (float)std::log((double)max_opacity / (1.0 - (double)max_opacity));
  const int64_t blocks = (P + 255) / 256;
  reset_opacity_kernel<<<(int)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      logits, P, cap);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
