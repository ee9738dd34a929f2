// Per-pixel L1 loss and its gradient (Sec. 3.3, Eq. 10 form: mean over
// pixels of the L1 norm over channels), with a fixed-order two-level sum so
// the loss value is bitwise deterministic.
#include "common.cuh"
#include "kernels.h"

namespace fe {

namespace {

constexpr int kL1Blocks = 1024;

__device__ __forceinline__ float block_sum(float v, float* s_warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  float t = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_warp[w];
  return t;
}

// Grid-stride over float4 groups when aligned, scalars for the tail; each
// block writes one partial sum.
__global__ void __launch_bounds__(256) l1_grad_kernel(const float* __restrict__ pred, const float* __restrict__ target,
                                                       int64_t n, float inv_rows, float* __restrict__ grad,
                                                       float* __restrict__ partial) {
  __shared__ float s_warp[8];
  float acc = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(pred) | reinterpret_cast<uintptr_t>(target) |
                     reinterpret_cast<uintptr_t>(grad)) & 15u) == 0;
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    auto sg = [&](float d) { return d > 0.0f ? inv_rows : (d < 0.0f ? -inv_rows : 0.0f); };
    auto one = [&](const float4 p, const float4 t, int64_t i) {
      const float d0 = p.x - t.x, d1 = p.y - t.y, d2 = p.z - t.z, d3 = p.w - t.w;
      acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
      reinterpret_cast<float4*>(grad)[i] = make_float4(sg(d0), sg(d1), sg(d2), sg(d3));
    };
    // Four groups in flight per thread; the additions keep the same order
    // as one group at a time.
    int64_t i = i0;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      float4 p[4], t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        p[u] = __ldcs(reinterpret_cast<const float4*>(pred) + i + u * stride);
        t[u] = __ldcs(reinterpret_cast<const float4*>(target) + i + u * stride);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) one(p[u], t[u], i + u * stride);
    }
    for (; i < n4; i += stride)
      one(reinterpret_cast<const float4*>(pred)[i], reinterpret_cast<const float4*>(target)[i], i);
    done = n4 * 4;
  }
  for (int64_t i = done + i0; i < n; i += stride) {
    const float d = pred[i] - target[i];
    acc += fabsf(d);
    grad[i] = d > 0.0f ? inv_rows : (d < 0.0f ? -inv_rows : 0.0f);
  }
  const float b = block_sum(acc, s_warp);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

__global__ void __launch_bounds__(256) l1_finish_kernel(const float* __restrict__ partial, int nparts, float inv_rows,
                                                         float* loss) {
  __shared__ float s_warp[8];
  float acc = 0.0f;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[i];
  const float b = block_sum(acc, s_warp);
  if (threadIdx.x == 0) *loss = b * inv_rows;
}

}  // namespace

void l1_grad_launch(const float* pred, const float* target, int64_t n, float inv_rows, float* grad, float* partial,
                    int blocks, cudaStream_t st) {
  l1_grad_kernel<<<blocks, 256, 0, st>>>(pred, target, n, inv_rows, grad, partial);
}

void l1_finish_launch(const float* partial, int nparts, float inv_rows, float* loss, cudaStream_t st) {
  l1_finish_kernel<<<1, 256, 0, st>>>(partial, nparts, inv_rows, loss);
}

cudaError_t launch_l1(const float* pred, const float* target, int64_t n, int64_t rows, float* grad, float* loss,
                      float* scratch, cudaStream_t st) {
  const float inv = rows > 0 ? 1.0f / (float)rows : 0.0f;
  int blocks = (int)((n + 1023) / 1024);
  if (blocks > kL1Blocks) blocks = kL1Blocks;
  if (blocks < 1) blocks = 1;
  l1_grad_kernel<<<blocks, 256, 0, st>>>(pred, target, n, inv, grad, scratch);
  l1_finish_kernel<<<1, 256, 0, st>>>(scratch, blocks, inv, loss);
  return cudaGetLastError();
}

}  // namespace fe

// ---------------------------------------------------------------------------
// Allocation-free variant of the L1 loss: the per-block partial sums live in
// a file-scope device array instead of caller scratch.  One block per 2048
// elements, at most 16384 blocks (64 KiB, held by every GPU that loads the
// library until the process exits).
namespace {

constexpr int kNoAllocBlocks = 16384;
constexpr int64_t kNoAllocPerBlock = 2048;
__device__ __align__(256) float g_l1_noalloc_scratch[kNoAllocBlocks];

// Device address of g_l1_noalloc_scratch on the current device.  The
// host-side name of the array is only a stand-in, not a device address, so
// every call asks the runtime (a host-side lookup; nothing is cached, so a
// device reset or another thread cannot leave a stale address behind).  The
// first lookup on a device may load the module: make the first call before
// any stream capture.
cudaError_t noalloc_scratch(float** out) {
  float* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_l1_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" fe_status fe_l1_loss_grad_noalloc(const float* pred, const float* target, int64_t n, int64_t rows,
                                             float* grad, float* loss, void* stream) {
  if (n < 0 || rows <= 0 || (n > 0 && (!pred || !target || !grad)) || !loss) return FE_ERR_INVALID_ARG;
  if (n > (int64_t)kNoAllocBlocks * kNoAllocPerBlock) return FE_ERR_WORKSPACE;
  float* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess || !scratch) return FE_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float inv = 1.0f / (float)rows;
  int blocks = (int)((n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
  if (blocks < 1) blocks = 1;
  // Every block writes its own partial before the finishing kernel reads
  // it, so nothing in the shared array needs clearing between calls.
  fe::l1_grad_launch(pred, target, n, inv, grad, scratch, blocks, st);
  fe::l1_finish_launch(scratch, blocks, inv, loss, st);
  return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
