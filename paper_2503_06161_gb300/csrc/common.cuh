// Shared definitions of the sm_103a FE-4DGS kernels: constants of the
// compositing recurrence, the workspace layout and small device helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fe4dgs.h"

namespace fe {

constexpr int kHidden = 64;   // MLP width W (Appendix A)
constexpr int kHeads = 11;    // d_mu(3) d_q(4) d_s(3) d_o(1) (Eq. 4)
constexpr int kThreads = 256; // one pixel per thread in a 256-pixel tile

// Compositing thresholds (readings; the paper gives none): alpha clamp,
// skip below 1/255, stop before T would drop under 1e-4, EWA dilation.
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Packed per-Gaussian render record (48 bytes, 16-byte aligned):
//  [0] u  [1] v  [2] A  [3] B  [4] Cc  [5] opacity  [6] depth
//  [7] r  [8] g  [9] b  [10] radius (float)
//  [11] half-widths (x, y) of a box holding every pixel centre the Gaussian
//       may blend, two fp16 rounded up (negative: it blends nowhere;
//       infinite: no box, the radius alone bounds it)
// with power2 = A dx^2 + B dx dy + Cc dy^2 = log2(e) * power, i.e.
// A = -0.5 log2(e) a, B = -log2(e) b, Cc = -0.5 log2(e) c for the conic
// (a, b, c) = inverse of the dilated 2D covariance.
constexpr int kRec = 12;

// Record word 11 for the quadratic form q = qa dx^2 + qb dx dy + qc dy^2
// (power2 = -q) and opacity o: alpha = o 2^-q >= 1/255 needs
// q <= log2(255 o), an ellipse whose box has half-widths
// sqrt(L qc / det), sqrt(L qa / det), det = qa qc - qb^2 / 4.  Widened by 1%
// and half a pixel, with L raised by 0.01, the box leaves out only centres
// whose alpha is below 1/255 by a margin far above the rounding of the
// per-pixel evaluation.  Used only when det cancels less than a hundredfold.
__device__ __forceinline__ float blend_box(float qa, float qb, float qc, float o) {
  float hx, hy;
  const float ac = qa * qc, det = fmaf(-0.25f * qb, qb, ac);
  if (!(255.0f * o >= 0.99f)) {
    hx = hy = -1.0f;  // alpha <= o < 1/255 everywhere
  } else if (!(det > 0.01f * ac)) {
    hx = hy = __int_as_float(0x7f800000);
  } else {
    const float L = fmaxf(log2f(255.0f * o), 0.0f) + 0.01f;
    hx = fmaf(sqrtf(L * qc / det), 1.01f, 0.5f);
    hy = fmaf(sqrtf(L * qa / det), 1.01f, 0.5f);
  }
  const __half2 h = __halves2half2(__float2half_ru(hx), __float2half_ru(hy));
  return __uint_as_float(*reinterpret_cast<const uint32_t*>(&h));
}

// Device-side error bits, sticky within one call.
enum : uint32_t { kErrOverflow = 1u, kErrTimeout = 2u, kErrNonFinite = 4u };

// Partial-gradient row per (tile, Gaussian) entry, D + 12 floats (16-byte
// rows): [0, D) dfeat, then du dv dA dB dCc dopacity, drgb[3], ddepth, 2 pad.
// Written only for the entries the reverse pass reached, which set their
// bit in a bitmask over the emission index.
constexpr int kPartialScalars = 10;
__host__ __device__ constexpr int partial_stride(int D) { return D + 12; }

struct Header {           // first 256 bytes of every workspace
  uint32_t err;           // error bits
  uint32_t num_dups;      // K written by keygen (may exceed capacity)
  uint32_t num_visible;
  uint32_t has_forward;
  uint32_t ticket[24];    // per-kernel block tickets (decoupled look-back)
  uint32_t pad[36];
};
static_assert(sizeof(Header) == 256, "header is 256 bytes");

// Radix / scan chunking: 256 threads x 16 items over the K list entries,
// 256 threads x 4 items over the P Gaussians (so P-sized passes still fill
// all SMs).
constexpr int kSortItems = 16;
constexpr int kSortChunk = kThreads * kSortItems;
constexpr int kPItems = 8;
constexpr int kPChunk = kThreads * kPItems;
// Depth-ordered Gaussians per block of the tile count / scatter kernels
// (each of the 8 warps walks 64 of them in order).
constexpr int kBinItems = 2;
constexpr int kBinChunk = kThreads * kBinItems;

// Ticket slots in the header.
enum : int {
  kTicketDepth0 = 0,  // 4 depth passes
  kTicketScan = 4,    // tiles_touched scan + per-block tile counts
  kTicketTable = 5,   // scan of the (tile, block) count table
  kNumTickets = 8,
};

// Largest tile count of the counting scatter (its per-warp counters live in
// shared memory).
constexpr int kMaxTiles = 8192;

struct Layout {
  int P, D, W, H, tw, th, tiles_x, tiles_y, ntiles, pblocks, bblocks;
  int64_t cap;
  bool with_backward;
  size_t hdr, rec, rect, touched, dkey[2], dval[2], offs, offs_by_gid, sorted, table;
  size_t status, hist, ranges, tfinal, ncontrib, partials, pflags, cmask, dstate, fsplit, ddstate, psum;
  size_t status_words, table_blocks;
  size_t total;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Host-side layout of a workspace; every region 256-byte aligned.
inline Layout make_layout(int P, int D, int W, int H, int tw, int th, int64_t cap, bool with_backward) {
  Layout L{};
  L.P = P; L.D = D; L.W = W; L.H = H; L.tw = tw; L.th = th;
  L.tiles_x = (W + tw - 1) / tw;
  L.tiles_y = (H + th - 1) / th;
  L.ntiles = L.tiles_x * L.tiles_y;
  L.cap = cap;
  L.with_backward = with_backward;
  const size_t Pn = (size_t)(P > 0 ? P : 1);
  const size_t Kn = (size_t)(cap > 0 ? cap : 1);
  L.pblocks = ceil_div((int64_t)Pn, kPChunk);
  L.bblocks = ceil_div((int64_t)Pn, kBinChunk);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  L.hdr = take(sizeof(Header));
  L.rec = take(Pn * kRec * 4);
  L.rect = take(Pn * 8);
  L.touched = take(Pn * 4);
  for (int i = 0; i < 2; ++i) L.dkey[i] = take(Pn * 4);
  for (int i = 0; i < 2; ++i) L.dval[i] = take(Pn * 4);
  L.offs = take((Pn + 1) * 4);
  L.offs_by_gid = take(Pn * 4);
  L.sorted = take(Kn * 8);
  const size_t table_n = (size_t)L.ntiles * L.bblocks;
  L.table = take(table_n * 4);
  L.table_blocks = (size_t)ceil_div((int64_t)(table_n > 0 ? table_n : 1), kPChunk);
  // Look-back words: 4 depth passes (u32 per digit per block), then u64 per
  // block of the tiles_touched scan and of the table scan.
  L.status_words = (size_t)L.pblocks * 256 * 4 + 2 * (size_t)L.bblocks + 2 * L.table_blocks;
  L.status = take(L.status_words * 4);
  L.hist = take((4 + 3) * 256 * 4);
  L.ranges = take((size_t)L.ntiles * 8);
  L.tfinal = take((size_t)W * H * 4);
  L.ncontrib = take((size_t)W * H * 4);
  // Deformation state (offsets + MLP unit masks) and the HexPlane features
  // as three BF16 terms (up to 64 channels) for the tensor-core MLP, with
  // 128 rows of slack so a 128-row tile of any term stays in the region.
  L.dstate = take(Pn * 16 * 4);
  L.fsplit = take((Pn + 128) * 3 * 64 * 2);
  if (with_backward) {
    L.partials = take(Kn * (size_t)partial_stride(D) * 4);
    L.pflags = take((Kn + 31) / 32 * 4);
    // Per (tile, 32-entry group, warp): which entries blended in some pixel
    // of the warp; tile t's groups start at slot rg.x / 32 + t.
    L.cmask = take(((Kn + 31) / 32 + (size_t)L.ntiles + 1) * 8 * 4);
    L.ddstate = take(Pn * 12 * 4);
    L.psum = take(Pn * 12 * 4);
  }
  L.total = off;
  return L;
}

template <typename T>
__host__ __device__ inline T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float(((uint32_t)b) << 16); }

// Tile rect of the pixels whose centre lies in the square of half-side r
// around (u, v), in binary32 with one rounding per add (no contraction).
// Returns false when empty.
__host__ __device__ inline bool pixel_rect(float u, float v, int r, int W, int H, int& x0, int& y0, int& x1, int& y1) {
#ifdef __CUDA_ARCH__
  const float rf = (float)r;
  const float rp = __fadd_rn(rf, 0.5f), rm = __fsub_rn(rf, 0.5f);
  float fx0 = ceilf(__fsub_rn(u, rp)), fx1 = floorf(__fadd_rn(u, rm));
  float fy0 = ceilf(__fsub_rn(v, rp)), fy1 = floorf(__fadd_rn(v, rm));
#else
  const float rf = (float)r;
  const float rp = rf + 0.5f, rm = rf - 0.5f;
  float fx0 = ceilf(u - rp), fx1 = floorf(u + rm);
  float fy0 = ceilf(v - rp), fy1 = floorf(v + rm);
#endif
  fx0 = fmaxf(fx0, 0.0f);
  fy0 = fmaxf(fy0, 0.0f);
  fx1 = fminf(fx1, (float)(W - 1));
  fy1 = fminf(fy1, (float)(H - 1));
  if (!(fx0 <= fx1 && fy0 <= fy1)) return false;
  x0 = (int)fx0; x1 = (int)fx1; y0 = (int)fy0; y1 = (int)fy1;
  return true;
}

// Pixel of thread `tid` inside a tile of tw x th = 256 pixels: each warp
// covers an 8 x 4 block of pixels (lane l at (l % 8, l / 8)), blocks laid
// row-major over the tile.  A compact warp footprint means fewer warps that
// a Gaussian's square only partly covers, so fewer idle lanes when a warp
// blends or differentiates an entry.
__device__ __forceinline__ void tile_pixel(int tid, int tw, int& lx, int& ly) {
  const int w = tid >> 5, l = tid & 31, bpr = tw >> 3;  // 8-wide blocks per tile row
  lx = ((w % bpr) << 3) + (l & 7);
  ly = ((w / bpr) << 2) + (l >> 3);
}

// alpha of record `rec` at pixel centre (pxc, pyc); one evaluation order,
// shared by the forward and reverse kernels so both take the same skip,
// clamp and inclusion decisions.  Returns false when the pair is skipped.
struct PairEval {
  float dx, dy, G, alpha;
  bool clamped;
};

// 2^x by the hardware approximation (ex2.approx.ftz: about 2 ulp; results
// below the normal range flush to 0, which the alpha >= 1/255 test rejects
// either way).
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// rec: a 16-byte aligned render record (u, v, A, B | Cc, opacity, ...,
// radius at word 10), read as two 16-byte and one 4-byte shared loads.
__device__ __forceinline__ bool eval_pair(const float* rec, float pxc, float pyc, PairEval& e) {
  const float4 q0 = *reinterpret_cast<const float4*>(rec);      // u, v, A, B
  const float2 q1 = *reinterpret_cast<const float2*>(rec + 4);  // Cc, opacity
  const float r = rec[10];
  e.dx = __fsub_rn(pxc, q0.x);
  e.dy = __fsub_rn(pyc, q0.y);
  if (fabsf(e.dx) > r || fabsf(e.dy) > r) return false;
  // power2 = A dx^2 + B dx dy + Cc dy^2 = (A dx + B dy) dx + Cc dy dy, with
  // explicit FMAs so the forward and reverse kernels round identically.
  const float t = __fmaf_rn(q0.z, e.dx, __fmul_rn(q0.w, e.dy));
  const float p2 = __fmaf_rn(t, e.dx, __fmul_rn(__fmul_rn(q1.x, e.dy), e.dy));
  if (p2 > 0.0f) return false;
  e.G = fast_exp2(p2);
  const float oG = __fmul_rn(q1.y, e.G);
  e.clamped = oG > kAlphaMax;
  e.alpha = e.clamped ? kAlphaMax : oG;
  return e.alpha >= kAlphaMin;
}

// The same evaluation without early exits (every lane runs every step, so
// the evaluations of several entries interleave): identical arithmetic, so
// identical decisions and values wherever it returns true.  Lanes that
// return false leave e with values that are not used.
__device__ __forceinline__ bool eval_pair_flat(const float* rec, float pxc, float pyc, PairEval& e) {
  const float4 q0 = *reinterpret_cast<const float4*>(rec);      // u, v, A, B
  const float2 q1 = *reinterpret_cast<const float2*>(rec + 4);  // Cc, opacity
  const float r = rec[10];
  e.dx = __fsub_rn(pxc, q0.x);
  e.dy = __fsub_rn(pyc, q0.y);
  const bool inside = !(fabsf(e.dx) > r) && !(fabsf(e.dy) > r);
  const float t = __fmaf_rn(q0.z, e.dx, __fmul_rn(q0.w, e.dy));
  const float p2 = __fmaf_rn(t, e.dx, __fmul_rn(__fmul_rn(q1.x, e.dy), e.dy));
  const bool below = !(p2 > 0.0f);
  e.G = fast_exp2(below ? p2 : 0.0f);
  const float oG = __fmul_rn(q1.y, e.G);
  e.clamped = oG > kAlphaMax;
  e.alpha = e.clamped ? kAlphaMax : oG;
  return inside && below && e.alpha >= kAlphaMin;
}

__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bits) { atomicOr(err, bits); }

// ---------------------------------------------------------------------------
// TMA bulk copies into shared memory with mbarrier completion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of incoming transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Generic-proxy accesses of a buffer before it is overwritten by the async proxy.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 1-D bulk copy global -> shared (addresses and size multiples of 16 bytes).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Polls of a staging wait before it gives up, and of the drain that waits
// for a block's copies in flight before its shared memory is released.
constexpr int kWaitPolls = 1 << 20;
constexpr int kDrainPolls = 1 << 22;

// Bounded wait for the phase of the given parity; false after `limit`
// polls (each poll may suspend the thread for a short time; limit 0 gives
// up at once).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = kWaitPolls) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace fe
