// Integer stage of the pass: the tile-based binning of 3DGS that the paper
// builds on (Sec. 2.1), reorganised for one GPU:
//   1. stable LSD radix sort of the P depth keys (4 x 8-bit passes);
//   2. exclusive scan of tiles_touched in depth order (decoupled look-back)
//      and, per block of 1024 depth-ordered Gaussians, its count of
//      entries per tile (a tile-major (tile, block) table);
//   3. exclusive scan of that table: the start of every (tile, block)
//      segment of the final list, and the tile ranges;
//   4. a scatter in which each warp walks its Gaussians in depth order with
//      per-warp tile counters, so every entry lands at its final position.
// The result is the order of a stable sort on (tile << 32 | depth bits) with
// ties by index, built with one write per entry instead of radix passes over
// 64-bit keys.  Every inter-block wait is a bounded spin that records
// kErrTimeout and carries on, so no launch can hang.
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
  // Publish the aggregate; the two block scans, which do not need the
  // prefix, run before the look-back for the exclusive prefix of this digit,
  // so predecessors have more time to resolve theirs.  Predecessors are read
  // four at a time (independent loads, overlapping latencies), then taken in
  // order until the first inclusive prefix.
  st_vol(status + (size_t)b * 256 + tid, (b == 0 ? kFlagPre : kFlagAgg) | bcount);
  uint32_t tot;
  const uint32_t gexcl = block_excl_scan(hist[tid], sm.scan, tot);
  const uint32_t bst = block_excl_scan(bcount, sm.scan, tot);
  sm.bstart[tid] = bst;
  uint32_t excl = 0;
  if (b > 0) {
    bool fin = false;
    for (int64_t j = (int64_t)b - 1; !fin && j >= 0; j -= 4) {
      uint32_t sv[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) sv[w] = j - w >= 0 ? ld_vol(status + (size_t)(j - w) * 256 + tid) : 0u;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        if (!fin && j - w >= 0) {
          uint32_t s = sv[w];
          int spins = 0;
          while ((s & ~kValMask) == 0u) {
            if (++spins > kSpinLimit) {
              set_err(err, kErrTimeout);
              s = kFlagPre;
              break;
            }
            __nanosleep(32);
            s = ld_vol(status + (size_t)(j - w) * 256 + tid);
          }
          excl += s & kValMask;
          if (s & kFlagPre) fin = true;
        }
      }
    }
    st_vol(status + (size_t)b * 256 + tid, kFlagPre | ((excl + bcount) & kValMask));
  }
  sm.gbase[tid] = gexcl + excl;
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
// Decoupled look-back over a 64-bit running total: block b publishes its
// aggregate, then sums its predecessors back to the first inclusive prefix,
// reading them eight at a time.
// In two halves, so a block can do independent work between them: publish
// the aggregate (block 0: its inclusive prefix), then resolve the exclusive
// prefix from the predecessors.
__device__ __forceinline__ void lookback64_publish(uint64_t* status, uint32_t b, uint64_t aggregate) {
  st_vol64(status + b, (b == 0 ? kFlagPre64 : kFlagAgg64) | aggregate);
}

__device__ __forceinline__ uint64_t lookback64_resolve(uint64_t* status, uint32_t b, uint64_t aggregate, uint32_t* err) {
  if (b == 0) return 0;
  uint64_t excl = 0;
  bool fin = false;
  for (int64_t j = (int64_t)b - 1; !fin && j >= 0; j -= 8) {
    uint64_t sv[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) sv[w] = j - w >= 0 ? ld_vol64(status + (j - w)) : 0ull;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      if (!fin && j - w >= 0) {
        uint64_t s = sv[w];
        int spins = 0;
        while ((s & ~kValMask64) == 0ull) {
          if (++spins > kSpinLimit) {
            set_err(err, kErrTimeout);
            s = kFlagPre64;
            break;
          }
          __nanosleep(32);
          s = ld_vol64(status + (j - w));
        }
        excl += s & kValMask64;
        if (s & kFlagPre64) fin = true;
      }
    }
  }
  st_vol64(status + b, kFlagPre64 | (excl + aggregate));
  return excl;
}

__device__ __forceinline__ uint64_t lookback64(uint64_t* status, uint32_t b, uint64_t aggregate, uint32_t* err) {
  lookback64_publish(status, b, aggregate);
  return lookback64_resolve(status, b, aggregate, err);
}

// Step 2: block b (ticket) owns depth ranks [512 b, 512 b + 512); thread t
// scans ranks 2t..2t+1.  Writes offs / offs_by_gid and column b of the
// tile-major count table.
struct CountArgs {
  int P, tiles_x, ntiles, nblocks;
  int64_t cap;
  const uint32_t* order;  // depth-sorted Gaussian ids
  const uint32_t* touched;
  const ushort4* rect;
  uint32_t *offs, *offs_by_gid, *table;
  uint64_t* status;
  uint32_t* ticket;
  Header* hdr;
};

__global__ void __launch_bounds__(kThreads) bin_count_kernel(const CountArgs a) {
  extern __shared__ uint32_t s_cnt[];  // [ntiles]
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_ticket;
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_c[kBinChunk];
  __shared__ float s_iw[kBinChunk];  // 1 / (rect width in tiles), once per Gaussian
  __shared__ ushort4 s_rect[kBinChunk];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < a.ntiles; i += kThreads) s_cnt[i] = 0;
  if (tid == 0) s_ticket = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t b = s_ticket;
  const int64_t start = (int64_t)b * kBinChunk;
  if (start >= a.P) return;
  uint32_t gid[kBinItems], cnt[kBinItems];
  uint32_t tsum = 0;
#pragma unroll
  for (int i = 0; i < kBinItems; ++i) {
    const int li = tid * kBinItems + i;
    const int64_t r = start + li;
    gid[i] = r < a.P ? a.order[r] : 0u;
    cnt[i] = r < a.P ? a.touched[gid[i]] : 0u;
    s_c[li] = cnt[i];
    const ushort4 rc = cnt[i] ? a.rect[gid[i]] : make_ushort4(0, 0, 0, 0);
    s_rect[li] = rc;
    s_iw[li] = 1.0f / (float)(rc.z - rc.x + 1u);
    tsum += cnt[i];
  }
  uint32_t btot;
  const uint32_t texcl = block_excl_scan(tsum, s_scan, btot);
  // The block's total goes out at once; its tile counts, which do not need
  // the prefix, are taken while the predecessors resolve theirs.
  if (tid == 0) lookback64_publish(a.status, b, btot);
  // Tile counts: each warp walks its Gaussians, lanes over one rect's tiles.
  const int nloc = (int)min((int64_t)kBinChunk, (int64_t)a.P - start);
  const int i0 = warp * (kBinChunk / 8), i1 = min(nloc, i0 + kBinChunk / 8);
  for (int i = i0; i < i1; ++i) {
    const uint32_t c = s_c[i];
    if (!c) continue;
    const ushort4 rc = s_rect[i];
    const uint32_t wdt = rc.z - rc.x + 1u;
    const float iw = s_iw[i];
    for (uint32_t k = lane; k < c; k += 32) {
      const uint32_t dy = (uint32_t)(((float)k + 0.5f) * iw), dx = k - dy * wdt;  // exact for these sizes
      atomicAdd(&s_cnt[(rc.y + dy) * (uint32_t)a.tiles_x + rc.x + dx], 1u);
    }
  }
  if (tid == 0) s_prefix = lookback64_resolve(a.status, b, btot, &a.hdr->err);
  __syncthreads();
  uint64_t run = s_prefix + texcl;
#pragma unroll
  for (int i = 0; i < kBinItems; ++i) {
    const int64_t r = start + tid * kBinItems + i;
    if (r < a.P) {
      const uint32_t o32 = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
      a.offs[r] = o32;
      a.offs_by_gid[gid[i]] = o32;
    }
    run += cnt[i];
  }
  if (start + kBinChunk >= a.P && tid == kThreads - 1) {
    a.offs[a.P] = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
    a.hdr->num_dups = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
    if (run > (uint64_t)a.cap) set_err(&a.hdr->err, kErrOverflow);
  }
  __syncthreads();
  for (int t = tid; t < a.ntiles; t += kThreads) a.table[(size_t)t * a.nblocks + b] = s_cnt[t];
}

// Step 3: in-place exclusive scan of the (tile, block) table, tile-major.
__global__ void __launch_bounds__(kThreads) table_scan_kernel(uint32_t* table, int64_t n, uint64_t* status,
                                                             uint32_t* ticket, uint32_t* err) {
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_ticket;
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x;
  if (tid == 0) s_ticket = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t b = s_ticket;
  const int64_t start = (int64_t)b * kPChunk;
  if (start >= n) return;
  uint32_t v[kPItems], tsum = 0;
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    const int64_t r = start + tid * kPItems + i;
    v[i] = r < n ? table[r] : 0u;
    tsum += v[i];
  }
  uint32_t btot;
  const uint32_t texcl = block_excl_scan(tsum, s_scan, btot);
  if (tid == 0) s_prefix = lookback64(status, b, btot, err);
  __syncthreads();
  uint64_t run = s_prefix + texcl;
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    const int64_t r = start + tid * kPItems + i;
    if (r < n) table[r] = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
    run += v[i];
  }
}

// Step 4: block b (= blockIdx.x) re-walks the ranks of count block b.  Each
// warp takes 64 consecutive Gaussians; its lanes cover one Gaussian's tiles
// at a time (all distinct), so per-warp tile counters give stable ranks.
// Block 0 also writes the tile ranges and marks the workspace as holding a
// forward's state.
struct ScatterArgs {
  int P, tiles_x, ntiles, nblocks;
  int64_t cap;
  const uint32_t *order, *touched, *offs, *table;
  const ushort4* rect;
  uint2* sorted;
  uint2* ranges;
  Header* hdr;
};

__global__ void __launch_bounds__(kThreads) bin_scatter_kernel(const ScatterArgs a) {
  extern __shared__ __align__(16) uint32_t s_dyn[];
  uint32_t* s_base = s_dyn;                                        // [ntiles]
  uint16_t* s_wc = reinterpret_cast<uint16_t*>(s_dyn + a.ntiles);  // [8][ntiles]
  __shared__ uint32_t s_gid[kBinChunk], s_cnt[kBinChunk], s_off[kBinChunk];
  __shared__ float s_iw[kBinChunk];  // 1 / (rect width in tiles), once per Gaussian
  __shared__ ushort4 s_rect[kBinChunk];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  const int64_t start = (int64_t)b * kBinChunk;
  const int nloc = (int)min((int64_t)kBinChunk, (int64_t)a.P - start);
  const uint64_t cap = (uint64_t)a.cap;
  // Past capacity the list is incomplete (and flagged): every range is
  // published empty so no later kernel follows an index beyond capacity.
  const bool overflow = (uint64_t)a.hdr->num_dups > cap;
  const uint64_t K = overflow ? 0 : (uint64_t)a.hdr->num_dups;
  for (int t = tid; t < a.ntiles; t += kThreads) {
    s_base[t] = a.table[(size_t)t * a.nblocks + b];
    if (b == 0) {
      const uint64_t lo = min((uint64_t)a.table[(size_t)t * a.nblocks], K);
      const uint64_t hi = t + 1 < a.ntiles ? min((uint64_t)a.table[(size_t)(t + 1) * a.nblocks], K) : K;
      a.ranges[t] = make_uint2((uint32_t)lo, (uint32_t)hi);
    }
  }
  if (b == 0 && tid == 0) a.hdr->has_forward = 1u;
  for (int i = tid; i < 8 * a.ntiles; i += kThreads) s_wc[i] = 0;
  for (int i = tid; i < nloc; i += kThreads) {
    const uint32_t g = a.order[start + i];
    const uint32_t c = a.touched[g];
    s_gid[i] = g;
    s_cnt[i] = c;
    s_off[i] = a.offs[start + i];
    const ushort4 rc = c ? a.rect[g] : make_ushort4(0, 0, 0, 0);
    s_rect[i] = rc;
    s_iw[i] = 1.0f / (float)(rc.z - rc.x + 1u);
  }
  __syncthreads();
  uint16_t* wc = s_wc + (size_t)warp * a.ntiles;
  const int i0 = warp * (kBinChunk / 8), i1 = min(nloc, i0 + kBinChunk / 8);
  for (int i = i0; i < i1; ++i) {
    const uint32_t c = s_cnt[i];
    if (!c) continue;
    const ushort4 rc = s_rect[i];
    const uint32_t wdt = rc.z - rc.x + 1u;
    const float iw = s_iw[i];
    for (uint32_t k = lane; k < c; k += 32) {
      const uint32_t dy = (uint32_t)(((float)k + 0.5f) * iw), dx = k - dy * wdt;  // exact for k < 2^20
      const uint32_t tile = (rc.y + dy) * (uint32_t)a.tiles_x + rc.x + dx;
      wc[tile] = (uint16_t)(wc[tile] + 1u);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int t = tid; t < a.ntiles; t += kThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t c = s_wc[w * a.ntiles + t];
      s_wc[w * a.ntiles + t] = (uint16_t)run;
      run += c;
    }
  }
  __syncthreads();
  for (int i = i0; i < i1; ++i) {
    const uint32_t c = s_cnt[i];
    if (!c) continue;
    const ushort4 rc = s_rect[i];
    const uint32_t wdt = rc.z - rc.x + 1u;
    const float iw = s_iw[i];
    const uint32_t g = s_gid[i], e0 = s_off[i];
    for (uint32_t k = lane; k < c; k += 32) {
      const uint32_t dy = (uint32_t)(((float)k + 0.5f) * iw), dx = k - dy * wdt;
      const uint32_t tile = (rc.y + dy) * (uint32_t)a.tiles_x + rc.x + dx;
      const uint32_t r = wc[tile];
      wc[tile] = (uint16_t)(r + 1u);
      const uint64_t pos = (uint64_t)s_base[tile] + r;
      const uint64_t e = (uint64_t)e0 + k;
      if (pos < cap) a.sorted[pos] = make_uint2((uint32_t)e, g);
    }
    __syncwarp();
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
  const size_t ppass_smem = sizeof(PassSmem<kPItems>);
  const int P = b.P;
  if (P <= 0) return cudaSuccess;  // K = 0: the cleared header and ranges already say so
  cudaError_t e;
  const int pblocks = b.pblocks;
  uint32_t* status_depth = b.status;
  const int bblocks = b.bblocks;
  uint64_t* status_count = reinterpret_cast<uint64_t*>(b.status + (size_t)pblocks * 256 * 4);
  uint64_t* status_table = status_count + bblocks;
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
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 2. tiles_touched scan + per-block tile counts
  CountArgs ca;
  ca.P = P;
  ca.tiles_x = b.tiles_x;
  ca.ntiles = b.ntiles;
  ca.nblocks = bblocks;
  ca.cap = b.cap;
  ca.order = b.dval[cur];
  ca.touched = b.touched;
  ca.rect = b.rect;
  ca.offs = b.offs;
  ca.offs_by_gid = b.offs_by_gid;
  ca.table = b.table;
  ca.status = status_count;
  ca.ticket = hdr->ticket + kTicketScan;
  ca.hdr = hdr;
  const size_t count_smem = (size_t)b.ntiles * 4;
  cudaFuncSetAttribute(bin_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)count_smem);
  bin_count_kernel<<<bblocks, kThreads, count_smem, st>>>(ca);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 3. scan of the (tile, block) table
  const int64_t tn = (int64_t)b.ntiles * bblocks;
  table_scan_kernel<<<ceil_div(tn, kPChunk), kThreads, 0, st>>>(b.table, tn, status_table,
                                                                hdr->ticket + kTicketTable, &hdr->err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 4. scatter into the final list
  ScatterArgs sa;
  sa.P = P;
  sa.tiles_x = b.tiles_x;
  sa.ntiles = b.ntiles;
  sa.nblocks = bblocks;
  sa.cap = b.cap;
  sa.order = b.dval[cur];
  sa.touched = b.touched;
  sa.offs = b.offs;
  sa.table = b.table;
  sa.rect = b.rect;
  sa.sorted = b.sorted;
  sa.ranges = b.ranges;
  sa.hdr = hdr;
  const size_t scat_smem = (size_t)b.ntiles * 4 + (size_t)8 * b.ntiles * 2;
  cudaFuncSetAttribute(bin_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scat_smem);
  bin_scatter_kernel<<<bblocks, kThreads, scat_smem, st>>>(sa);
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
    const uint32_t g = d.sorted[i].y;
    if (d.keys) {
      // Tile of list position i: the last tile whose range starts at or
      // before i (empty tiles share the start of the next tile).
      int lo = 0, hi = d.ntiles;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (d.ranges[mid].x <= i) lo = mid; else hi = mid;
      }
      const float dep = d.rec[3 * (size_t)g + 1].z;
      d.keys[i] = ((uint64_t)(uint32_t)lo << 32) | __float_as_uint(dep);
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
  // The sink's address first: nothing to release if the lookup fails.
  float* sink = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), g_probe_sink);
  if (e != cudaSuccess) return e;
  if (!sink) return cudaErrorInvalidSymbol;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  fma_probe_kernel<<<blocks, 256, 0, st>>>(iters / 8 + 1, 1.0f, sink);  // warm-up
  cudaEventRecord(e0, st);
  fma_probe_kernel<<<blocks, 256, 0, st>>>(iters, 1.0f, sink);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  *flops = (double)blocks * 256.0 * iters * 16.0 * 8.0 * 2.0 / (ms * 1e-3);
  return cudaGetLastError();
}

}  // namespace fe
