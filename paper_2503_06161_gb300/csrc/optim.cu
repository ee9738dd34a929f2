// Adam update of the Gaussian parameters (Sec. 4.1 trains with Adam; the
// update is the standard one with bias correction):
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
//   p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
// on FP32 master copies, optionally refreshing a bf16 copy of p (the storage
// format the renderer reads for SH and features).  One launch covers every
// parameter group; each thread owns four consecutive elements of one group
// (16-byte loads and stores), so the pass streams each array once.
#include <cmath>

#include "common.cuh"

namespace fe {

namespace {

constexpr int kAdamMaxGroups = 8;

struct AdamGroupDev {
  float* p;
  const float* g;
  float* m;
  float* v;
  uint16_t* pb;  // optional bf16 copy
  int64_t n;
  float lr;
};

struct AdamBatch {
  AdamGroupDev grp[kAdamMaxGroups];
  int64_t chunk0[kAdamMaxGroups + 1];  // first 4-element chunk of each group
  int ngroups;
  float b1, b2, eps, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, const AdamBatch& b, float lr) {
  m = fmaf(b.b1, m, (1.0f - b.b1) * g);
  v = fmaf(b.b2, v, (1.0f - b.b2) * g * g);
  const float den = sqrtf(v * b.c2) + b.eps;
  p = p - lr * ((m * b.c1) / den);
}

__global__ void __launch_bounds__(256) adam_kernel(const AdamBatch b) {
  const int64_t total = b.chunk0[b.ngroups];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < b.ngroups && c >= b.chunk0[k + 1]) ++k;
    const AdamGroupDev& G = b.grp[k];
    const int64_t e = (c - b.chunk0[k]) * 4;
    const float lr = G.lr;
    if (e + 4 <= G.n) {
      float4 p = *reinterpret_cast<const float4*>(G.p + e);
      const float4 g = __ldg(reinterpret_cast<const float4*>(G.g + e));
      float4 m = *reinterpret_cast<const float4*>(G.m + e);
      float4 v = *reinterpret_cast<const float4*>(G.v + e);
      adam_one(p.x, g.x, m.x, v.x, b, lr);
      adam_one(p.y, g.y, m.y, v.y, b, lr);
      adam_one(p.z, g.z, m.z, v.z, b, lr);
      adam_one(p.w, g.w, m.w, v.w, b, lr);
      *reinterpret_cast<float4*>(G.p + e) = p;
      *reinterpret_cast<float4*>(G.m + e) = m;
      *reinterpret_cast<float4*>(G.v + e) = v;
      if (G.pb) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(p.x, p.y), hi = __floats2bfloat162_rn(p.z, p.w);
        *reinterpret_cast<uint2*>(G.pb + e) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
      }
    } else {
      for (int64_t j = e; j < G.n; ++j) {
        float p = G.p[j], m = G.m[j], v = G.v[j];
        adam_one(p, G.g[j], m, v, b, lr);
        G.p[j] = p;
        G.m[j] = m;
        G.v[j] = v;
        if (G.pb) {
          const __nv_bfloat16 h = __float2bfloat16_rn(p);
          G.pb[j] = *reinterpret_cast<const uint16_t*>(&h);
        }
      }
    }
  }
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

constexpr int kSumMaxSrc = 8;
struct SumArgs {
  const float* src[kSumMaxSrc];
  int nsrc;
};

// dst = ((src0 + src1) + src2) + ..., element by element, four at a time.
__global__ void __launch_bounds__(256) sum_kernel(float* __restrict__ dst, const SumArgs s, int64_t n) {
  const int64_t n4 = n / 4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 acc = __ldg(reinterpret_cast<const float4*>(s.src[0]) + i);
    for (int k = 1; k < s.nsrc; ++k) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(s.src[k]) + i);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    reinterpret_cast<float4*>(dst)[i] = acc;
  }
  if (blockIdx.x == 0 && threadIdx.x < (unsigned)(n - 4 * n4)) {
    const int64_t i = 4 * n4 + threadIdx.x;
    float acc = s.src[0][i];
    for (int k = 1; k < s.nsrc; ++k) acc += s.src[k][i];
    dst[i] = acc;
  }
}

// Unaligned arrays: one element per thread.
__global__ void __launch_bounds__(256) sum1_kernel(float* __restrict__ dst, const SumArgs s, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = s.src[0][i];
    for (int k = 1; k < s.nsrc; ++k) acc += s.src[k][i];
    dst[i] = acc;
  }
}

}  // namespace

cudaError_t launch_sum_f32(float* dst, const float* const* srcs, int nsrc, int64_t n, cudaStream_t st) {
  if (nsrc < 1 || nsrc > kSumMaxSrc) return cudaErrorInvalidValue;
  if (n <= 0) return cudaSuccess;
  SumArgs s{};
  s.nsrc = nsrc;
  bool vec = al16(dst);
  for (int k = 0; k < nsrc; ++k) {
    s.src[k] = srcs[k];
    vec = vec && al16(srcs[k]);
  }
  if (vec) {
    const int64_t blocks = (n / 4 + 255) / 256 + 1;
    sum_kernel<<<(int)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(dst, s, n);
  } else {
    const int64_t blocks = (n + 255) / 256;
    sum1_kernel<<<(int)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(dst, s, n);
  }
  return cudaGetLastError();
}

}  // namespace fe

using namespace fe;

extern "C" fe_status fe_sum_f32(float* dst, const float* const* srcs, int nsrc, int64_t n, void* stream) {
  if (!dst || !srcs || nsrc < 1 || nsrc > kSumMaxSrc || n < 0 || !al16(dst)) return FE_ERR_INVALID_ARG;
  SumArgs s{};
  s.nsrc = nsrc;
  for (int k = 0; k < nsrc; ++k) {
    if (!srcs[k] || !al16(srcs[k])) return FE_ERR_INVALID_ARG;
    s.src[k] = srcs[k];
  }
  if (n == 0) return FE_OK;
  const int64_t blocks = (n / 4 + 255) / 256 + 1;
  const int grid = (int)(blocks < 152 * 8 ? blocks : 152 * 8);
  sum_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(dst, s, n);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" fe_status fe_adam_step(const fe_adam_group* groups, int ngroups, int step, float beta1, float beta2,
                                  float eps, void* stream) {
  if (!groups || ngroups < 1 || ngroups > kAdamMaxGroups || step < 1) return FE_ERR_INVALID_ARG;
  if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f)) return FE_ERR_INVALID_ARG;
  AdamBatch b{};
  b.ngroups = ngroups;
  b.b1 = beta1;
  b.b2 = beta2;
  b.eps = eps;
  b.c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)step)));
  b.c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)step)));
  int64_t chunks = 0;
  for (int k = 0; k < ngroups; ++k) {
    const fe_adam_group& g = groups[k];
    if (g.n < 0) return FE_ERR_INVALID_ARG;
    if (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v || !al16(g.param) || !al16(g.grad) || !al16(g.m) ||
                    !al16(g.v) || (g.param_bf16 && (reinterpret_cast<uintptr_t>(g.param_bf16) & 7u))))
      return FE_ERR_INVALID_ARG;
    b.grp[k] = AdamGroupDev{g.param, g.grad, g.m, g.v, static_cast<uint16_t*>(g.param_bf16), g.n, g.lr};
    b.chunk0[k] = chunks;
    chunks += (g.n + 3) / 4;
  }
  b.chunk0[ngroups] = chunks;
  if (chunks == 0) return FE_OK;
  const int64_t blocks = (chunks + 255) / 256;
  const int grid = (int)(blocks < 152 * 8 ? blocks : 152 * 8);
  adam_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(b);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
