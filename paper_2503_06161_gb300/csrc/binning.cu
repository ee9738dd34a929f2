// Integer stage of the pass: the tile-based binning of 3DGS that the paper
// builds on (Sec. 2.1), reorganised for one GPU with large HBM:
//   1. stable LSD radix sort of the P depth keys (4 x 8-bit passes);
//   2. one fused kernel: exclusive scan of tiles_touched in depth order
//      (decoupled look-back), emission of each Gaussian's tiles row-major,
//      and the digit histograms of the tile ids;
//   3. stable LSD radix sort of the K tile ids (1-2 x 8-bit passes) whose
//      payload is the emission index;
//   4. tile ranges from the sorted tile ids.
// Emitting in depth order and sorting stably by tile gives exactly the order
// of a stable sort on (tile << 32 | depth bits) with ties by index, while
// moving 32-bit keys through 2 passes instead of 64-bit keys through 6.
// Every inter-block wait is a bounded spin that records kErrTimeout and
// carries on, so no launch can hang.
#include "common.cuh"
#include "kernels.h"

namespace fe {

namespace {

constexpr uint32_t kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kValMask = (1u << 30) - 1;
constexpr uint64_t kFlagAgg64 = 1ull << 62, kFlagPre64 = 2ull << 62, kValMask64 = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t ld_vol(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }
__device__ __forceinline__ void st_vol(uint32_t* p, uint32_t v) { *reinterpret_cast<volatile uint32_t*>(p) = v; }
__device__ __forceinline__ uint64_t ld_vol64(const uint64_t* p) { return *reinterpret_cast<const volatile uint64_t*>(p); }
__device__ __forceinline__ void st_vol64(uint64_t* p, uint64_t v) { *reinterpret_cast<volatile uint64_t*>(p) = v; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const uint32_t v = s_warp[w];
    if (w < warp) wpre += v;
    tot += v;
  }
  __syncthreads();
  total = tot;
  return wpre + incl - x;
}

// ---------------------------------------------------------------------------
// Global digit histograms of the depth keys (all four passes at once).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) depth_hist_kernel(const uint32_t* __restrict__ keys, int n, uint32_t* hist) {
  __shared__ uint32_t s[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += kThreads) (&s[0][0])[i] = 0;
  __syncthreads();
  const int start = blockIdx.x * kPChunk;
  const int end = min(n, start + kPChunk);
  for (int i = start + threadIdx.x; i < end; i += kThreads) {
    const uint32_t k = keys[i];
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&s[p][(k >> (8 * p)) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 256; i += kThreads) {
    const uint32_t v = (&s[0][0])[i];
    if (v) atomicAdd(hist + i, v);
  }
}

// ---------------------------------------------------------------------------
// One stable LSD radix pass (8-bit digit at `shift`) with decoupled look-back.
// Block b (taken from an atomic ticket so predecessors are always running)
// handles elements [b*4096, b*4096+4096); warp w its sub-chunk of 512.
// ---------------------------------------------------------------------------
template <int ITEMS>
struct PassSmem {
  uint32_t wcnt[8][256];
  uint32_t gbase[256];
  uint32_t bstart[256];
  uint32_t keys[kThreads * ITEMS];
  uint32_t vals[kThreads * ITEMS];
  uint32_t scan[8];
  uint32_t ticket;
};

template <bool kIdentVals, int ITEMS>
__global__ void __launch_bounds__(kThreads) onesweep_kernel(const uint32_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint32_t* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out,
                                                            const uint32_t* n_dev, int64_t n_cap, int shift,
                                                            const uint32_t* __restrict__ hist, uint32_t* status,
                                                            uint32_t* ticket, uint32_t* err) {
  constexpr int CHUNK = kThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassSmem<ITEMS>& sm = *reinterpret_cast<PassSmem<ITEMS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 8 * 256; i += kThreads) (&sm.wcnt[0][0])[i] = 0;
  if (tid == 0) sm.ticket = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t b = sm.ticket;
  const uint64_t n = n_dev ? min((uint64_t)*n_dev, (uint64_t)n_cap) : (uint64_t)n_cap;
  const uint64_t start = (uint64_t)b * CHUNK;
  if (start >= n) return;
  const uint32_t cnt = (uint32_t)min((uint64_t)CHUNK, n - start);

  uint32_t k[ITEMS], v[ITEMS], rk[ITEMS];
  int dg[ITEMS];
  const uint64_t wbase = start + (uint64_t)warp * (CHUNK / 8);
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
    const bool valid = idx < n;
    const uint32_t key = valid ? keys_in[idx] : 0u;
    const uint32_t val = valid ? (kIdentVals ? (uint32_t)idx : vals_in[idx]) : 0u;
    const int d = valid ? (int)((key >> shift) & 255u) : 256;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    const int lead = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid) base = sm.wcnt[warp][d];
    __syncwarp();
    if (valid && lane == lead) sm.wcnt[warp][d] = base + __popc(peers);
    __syncwarp();
    rk[r] = base + __popc(peers & lanemask_lt());
    k[r] = key;
    v[r] = val;
    dg[r] = d;
  }
  __syncthreads();
  // Digit `tid`: prefix over warps and the block count.
  uint32_t bcount = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const uint32_t c = sm.wcnt[w][tid];
    sm.wcnt[w][tid] = bcount;
    bcount += c;
  }
  // Publish the aggregate, look back for the exclusive prefix of this digit.
  uint32_t excl = 0;
  if (b == 0) {
    st_vol(status + tid, kFlagPre | bcount);
  } else {
    st_vol(status + (size_t)b * 256 + tid, kFlagAgg | bcount);
    for (int64_t j = (int64_t)b - 1; j >= 0; --j) {
      uint32_t s = ld_vol(status + (size_t)j * 256 + tid);
      int spins = 0;
      while ((s & ~kValMask) == 0u) {
        if (++spins > kSpinLimit) {
          set_err(err, kErrTimeout);
          s = kFlagPre;
          break;
        }
        __nanosleep(32);
        s = ld_vol(status + (size_t)j * 256 + tid);
      }
      excl += s & kValMask;
      if (s & kFlagPre) break;
    }
    st_vol(status + (size_t)b * 256 + tid, kFlagPre | ((excl + bcount) & kValMask));
  }
  uint32_t tot;
  const uint32_t gexcl = block_excl_scan(hist[tid], sm.scan, tot);
  sm.gbase[tid] = gexcl + excl;
  const uint32_t bst = block_excl_scan(bcount, sm.scan, tot);
  sm.bstart[tid] = bst;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (dg[r] < 256) {
      const uint32_t lp = sm.bstart[dg[r]] + sm.wcnt[warp][dg[r]] + rk[r];
      sm.keys[lp] = k[r];
      sm.vals[lp] = v[r];
    }
  }
  __syncthreads();
  for (uint32_t i = tid; i < cnt; i += kThreads) {
    const uint32_t key = sm.keys[i];
    const uint32_t d = (key >> shift) & 255u;
    const uint32_t gp = sm.gbase[d] + (i - sm.bstart[d]);
    keys_out[gp] = key;
    vals_out[gp] = sm.vals[i];
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan of tiles_touched in depth order + tile emission + tile
// digit histograms.  Block b owns depth ranks [1024 b, 1024 b + 1024);
// thread t scans ranks 4t..4t+3 of it.  Emission is load balanced: each
// thread writes whole output entries, finding the owning Gaussian by a
// binary search over the block's offsets in shared memory, so the writes
// are coalesced and no thread walks a long rect alone.
struct KeygenArgs {
  int P, tiles_x, tile_passes;
  int64_t cap;
  const uint32_t* order;     // depth-sorted Gaussian ids
  const uint32_t* touched;
  const ushort4* rect;
  uint32_t *offs, *offs_by_gid, *tile_out, *gid_of_emit;
  uint32_t* hist;            // [3][256] tile digit histograms
  uint64_t* status;
  uint32_t* ticket;
  Header* hdr;
};

__global__ void __launch_bounds__(kThreads) scan_keygen_kernel(const KeygenArgs a) {
  __shared__ uint32_t s_hist[3][256];
  __shared__ uint32_t s_off[kPChunk];
  __shared__ uint32_t s_gid[kPChunk];
  __shared__ ushort4 s_rect[kPChunk];
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_ticket;
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * 256; i += kThreads) (&s_hist[0][0])[i] = 0;
  if (tid == 0) s_ticket = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t b = s_ticket;
  const int64_t start = (int64_t)b * kPChunk;
  if (start >= a.P) return;
  uint32_t cnt[kPItems];
  uint32_t tsum = 0;
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    const int li = tid * kPItems + i;
    const int64_t r = start + li;
    uint32_t g = 0, c = 0;
    ushort4 rc = make_ushort4(1, 1, 0, 0);
    if (r < a.P) {
      g = a.order[r];
      c = a.touched[g];
      if (c) rc = a.rect[g];
    }
    s_gid[li] = g;
    s_rect[li] = rc;
    cnt[i] = c;
    tsum += c;
  }
  uint32_t btot;
  const uint32_t texcl = block_excl_scan(tsum, s_scan, btot);
  if (tid == 0) {
    uint64_t excl = 0;
    if (b == 0) {
      st_vol64(a.status, kFlagPre64 | (uint64_t)btot);
    } else {
      st_vol64(a.status + b, kFlagAgg64 | (uint64_t)btot);
      for (int64_t j = (int64_t)b - 1; j >= 0; --j) {
        uint64_t s = ld_vol64(a.status + j);
        int spins = 0;
        while ((s & ~kValMask64) == 0ull) {
          if (++spins > kSpinLimit) {
            set_err(&a.hdr->err, kErrTimeout);
            s = kFlagPre64;
            break;
          }
          __nanosleep(32);
          s = ld_vol64(a.status + j);
        }
        excl += s & kValMask64;
        if (s & kFlagPre64) break;
      }
      st_vol64(a.status + b, kFlagPre64 | (excl + btot));
    }
    s_prefix = excl;
  }
  // Local offsets of this thread's ranks.
  uint32_t run = texcl;
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    s_off[tid * kPItems + i] = run;
    run += cnt[i];
  }
  __syncthreads();
  const uint64_t base = s_prefix;
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    const int li = tid * kPItems + i;
    const int64_t r = start + li;
    if (r < a.P) {
      const uint32_t o32 = (uint32_t)min(base + s_off[li], (uint64_t)0xFFFFFFFFu);
      a.offs[r] = o32;
      a.offs_by_gid[s_gid[li]] = o32;
    }
  }
  const uint64_t cap = (uint64_t)a.cap;
  const int nloc = (int)min((int64_t)kPChunk, (int64_t)a.P - start);
  for (uint32_t i = tid; i < btot; i += kThreads) {
    const uint64_t e = base + i;
    if (e >= cap) break;
    // Owner: last local Gaussian whose offset is <= i.
    int lo = 0, hi = nloc;  // invariant: s_off[lo] <= i < s_off[hi] (s_off[nloc] = btot)
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_off[mid] <= i) lo = mid; else hi = mid;
    }
    const ushort4 rc = s_rect[lo];
    const uint32_t loc = i - s_off[lo];
    const uint32_t wdt = (uint32_t)(rc.z - rc.x + 1);
    const uint32_t ty = rc.y + loc / wdt, tx = rc.x + loc % wdt;
    const uint32_t tile = ty * (uint32_t)a.tiles_x + tx;
    a.tile_out[e] = tile;
    a.gid_of_emit[e] = s_gid[lo];
    atomicAdd(&s_hist[0][tile & 255u], 1u);
    if (a.tile_passes > 1) atomicAdd(&s_hist[1][(tile >> 8) & 255u], 1u);
    if (a.tile_passes > 2) atomicAdd(&s_hist[2][(tile >> 16) & 255u], 1u);
  }
  if (start + kPChunk >= a.P && tid == 0) {
    // Last block: total K.
    const uint64_t total = base + btot;
    a.offs[a.P] = (uint32_t)min(total, (uint64_t)0xFFFFFFFFu);
    a.hdr->num_dups = (uint32_t)min(total, (uint64_t)0xFFFFFFFFu);
    if (total > cap) set_err(&a.hdr->err, kErrOverflow);
  }
  __syncthreads();
  for (int i = tid; i < a.tile_passes * 256; i += kThreads) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(a.hist + i, v);
  }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ tiles, const Header* hdr, int64_t cap, uint2* ranges,
                              uint32_t* has_forward) {
  const uint64_t n = min((uint64_t)hdr->num_dups, (uint64_t)cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && has_forward) *has_forward = 1u;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = tiles[i];
    if (i == 0 || tiles[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i + 1 == n || tiles[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

__global__ void bin_prep_kernel(int P, const float* __restrict__ uv, const int* __restrict__ radius,
                                const float* __restrict__ depth, int W, int H, int tw, int th, ushort4* rect,
                                uint32_t* touched, uint32_t* dkey, uint32_t* num_visible) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  bool vis = false;
  if (g < P) {
    ushort4 rc = make_ushort4(1, 1, 0, 0);
    uint32_t t = 0, key = 0xFFFFFFFFu;
    const int r = radius[g];
    const float u = uv[2 * g], v = uv[2 * g + 1];
    int x0, y0, x1, y1;
    if (r > 0 && isfinite(u) && isfinite(v) && pixel_rect(u, v, r, W, H, x0, y0, x1, y1)) {
      const int tx0 = x0 / tw, tx1 = x1 / tw, ty0 = y0 / th, ty1 = y1 / th;
      rc = make_ushort4(tx0, ty0, tx1, ty1);
      t = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
      key = __float_as_uint(depth[g]);
      vis = true;
    }
    rect[g] = rc;
    touched[g] = t;
    dkey[g] = key;
  }
  const unsigned vote = __ballot_sync(0xFFFFFFFFu, vis);
  if ((threadIdx.x & 31) == 0 && vote) atomicAdd(num_visible, (uint32_t)__popc(vote));
}

int grid_for(int64_t n, int per_block) {
  const int64_t b = (n + per_block - 1) / per_block;
  const int64_t c = b < 152 * 16 ? b : 152 * 16;
  return (int)(c > 1 ? c : 1);
}

}  // namespace

cudaError_t launch_bin_prep(int P, const float* uv, const int* radius, const float* depth, int W, int H, int tw,
                            int th, ushort4* rect, uint32_t* touched, uint32_t* dkey, uint32_t* num_visible,
                            cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  bin_prep_kernel<<<ceil_div(P, kThreads), kThreads, 0, st>>>(P, uv, radius, depth, W, H, tw, th, rect, touched,
                                                              dkey, num_visible);
  return cudaGetLastError();
}

cudaError_t launch_binning(BinArgs& b, cudaStream_t st) {
  Header* hdr = static_cast<Header*>(b.hdr);
  const size_t pass_smem = sizeof(PassSmem<kSortItems>);
  const size_t ppass_smem = sizeof(PassSmem<kPItems>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(onesweep_kernel<true, kSortItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pass_smem);
    cudaFuncSetAttribute(onesweep_kernel<false, kSortItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pass_smem);
    attr_set = true;
  }
  cudaError_t e;
  const int P = b.P;
  const int pblocks = ceil_div(P > 0 ? P : 1, kPChunk);
  uint32_t* status_depth = b.status;
  uint32_t* status_tile = b.status + (size_t)pblocks * 256 * 4;
  const int kblocks = ceil_div(b.cap > 0 ? b.cap : 1, kSortChunk);
  uint64_t* status_scan = reinterpret_cast<uint64_t*>(status_tile + (size_t)kblocks * 256 * 3);
  if (P > 0) {
    // 1. depth sort (values: Gaussian ids)
    depth_hist_kernel<<<pblocks, kThreads, 0, st>>>(b.dkey[0], P, b.hist);
    int cur = 0;
    for (int p = 0; p < 4; ++p) {
      if (p == 0)
        onesweep_kernel<true, kPItems><<<pblocks, kThreads, ppass_smem, st>>>(
            b.dkey[cur], nullptr, b.dkey[cur ^ 1], b.dval[cur ^ 1], nullptr, P, 8 * p, b.hist + 256 * p,
            status_depth + (size_t)p * pblocks * 256, hdr->ticket + kTicketDepth0 + p, &hdr->err);
      else
        onesweep_kernel<false, kPItems><<<pblocks, kThreads, ppass_smem, st>>>(
            b.dkey[cur], b.dval[cur], b.dkey[cur ^ 1], b.dval[cur ^ 1], nullptr, P, 8 * p, b.hist + 256 * p,
            status_depth + (size_t)p * pblocks * 256, hdr->ticket + kTicketDepth0 + p, &hdr->err);
      cur ^= 1;
    }
    b.depth_final = cur;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // 2. scan + emission
    KeygenArgs ka;
    ka.P = P;
    ka.tiles_x = b.tiles_x;
    ka.tile_passes = b.tile_passes;
    ka.cap = b.cap;
    ka.order = b.dval[cur];
    ka.touched = b.touched;
    ka.rect = b.rect;
    ka.offs = b.offs;
    ka.offs_by_gid = b.offs_by_gid;
    ka.tile_out = b.tkey[0];
    ka.gid_of_emit = b.gid_of_emit;
    ka.hist = b.hist + 4 * 256;
    ka.status = status_scan;
    ka.ticket = hdr->ticket + kTicketScan;
    ka.hdr = hdr;
    scan_keygen_kernel<<<pblocks, kThreads, 0, st>>>(ka);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 3. tile sort (values: emission index)
  int cur = 0;
  for (int p = 0; p < b.tile_passes; ++p) {
    if (p == 0)
      onesweep_kernel<true, kSortItems><<<kblocks, kThreads, pass_smem, st>>>(
          b.tkey[cur], nullptr, b.tkey[cur ^ 1], b.tval[cur ^ 1], &hdr->num_dups, b.cap, 8 * p,
          b.hist + (4 + p) * 256, status_tile + (size_t)p * kblocks * 256, hdr->ticket + kTicketTile0 + p, &hdr->err);
    else
      onesweep_kernel<false, kSortItems><<<kblocks, kThreads, pass_smem, st>>>(
          b.tkey[cur], b.tval[cur], b.tkey[cur ^ 1], b.tval[cur ^ 1], &hdr->num_dups, b.cap, 8 * p,
          b.hist + (4 + p) * 256, status_tile + (size_t)p * kblocks * 256, hdr->ticket + kTicketTile0 + p, &hdr->err);
    cur ^= 1;
  }
  b.tile_final = cur;
  // 4. ranges
  ranges_kernel<<<grid_for(b.cap, 256), 256, 0, st>>>(b.tkey[cur], hdr, b.cap, b.ranges, &hdr->has_forward);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Debug dump of the forward state (parity tests).
// ---------------------------------------------------------------------------
__global__ void dump_kernel(const DumpArgs d) {
  const Header* hdr = static_cast<const Header*>(d.hdr);
  const uint64_t K = min((uint64_t)hdr->num_dups, (uint64_t)d.cap);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t i = i0; i < K; i += stride) {
    const uint32_t e = d.sorted_e[i];
    const uint32_t g = d.gid_of_emit[e];
    if (d.keys) {
      const float dep = d.rec[3 * (size_t)g + 1].z;
      d.keys[i] = ((uint64_t)d.sorted_tile[i] << 32) | __float_as_uint(dep);
    }
    if (d.gauss) d.gauss[i] = g;
  }
  for (uint64_t i = i0; i < (uint64_t)d.ntiles; i += stride)
    if (d.ranges_out) { d.ranges_out[2 * i] = d.ranges[i].x; d.ranges_out[2 * i + 1] = d.ranges[i].y; }
  for (uint64_t i = i0; i < (uint64_t)d.HW; i += stride) {
    if (d.ncontrib_out) d.ncontrib_out[i] = d.ncontrib[i];
    if (d.tfinal_out) d.tfinal_out[i] = d.tfinal[i];
  }
  for (uint64_t g = i0; g < (uint64_t)d.P; g += stride) {
    const float4 r0 = d.rec[3 * g], r1 = d.rec[3 * g + 1], r2 = d.rec[3 * g + 2];
    if (d.uv) { d.uv[2 * g] = r0.x; d.uv[2 * g + 1] = r0.y; }
    if (d.conic) {
      // Stored scaled conic back to (a, b, c).
      d.conic[3 * g] = r0.z / (-0.5f * kLog2e);
      d.conic[3 * g + 1] = r0.w / (-kLog2e);
      d.conic[3 * g + 2] = r1.x / (-0.5f * kLog2e);
    }
    if (d.opacity) d.opacity[g] = r1.y;
    if (d.depth) d.depth[g] = r1.z;
    if (d.rgb) { d.rgb[3 * g] = r1.w; d.rgb[3 * g + 1] = r2.x; d.rgb[3 * g + 2] = r2.y; }
    if (d.radius) d.radius[g] = (int32_t)r2.z;
    if (d.touched_out) d.touched_out[g] = d.touched[g];
  }
}

cudaError_t launch_dump(const DumpArgs& d, cudaStream_t st) {
  int64_t n = d.cap;
  if (d.P > n) n = d.P;
  if (d.HW > n) n = d.HW;
  if (d.ntiles > n) n = d.ntiles;
  dump_kernel<<<grid_for(n, 256), 256, 0, st>>>(d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 FMA throughput probe: 8 independent FMA chains per thread.
// ---------------------------------------------------------------------------
__device__ float g_probe_sink[1];

__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float seed, float* out) {
  float a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
        a7 = a0 + 7;
  const float m = 0.999999f, c = 1e-7f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
      a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
    }
  }
  const float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.678f) out[0] = s;  // keeps the chains alive
}

cudaError_t probe_fp32(int iters, double* flops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float* sink = nullptr;
  cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), g_probe_sink);
  if (!sink) return cudaErrorInvalidSymbol;
  fma_probe_kernel<<<blocks, 256, 0, st>>>(iters / 8 + 1, 1.0f, sink);  // warm-up
  cudaEventRecord(e0, st);
  fma_probe_kernel<<<blocks, 256, 0, st>>>(iters, 1.0f, sink);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  *flops = (double)blocks * 256.0 * iters * 16.0 * 8.0 * 2.0 / (ms * 1e-3);
  return cudaGetLastError();
}

}  // namespace fe
