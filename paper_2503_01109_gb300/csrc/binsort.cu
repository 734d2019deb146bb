// binsort.cu -- tile binning and depth ordering of the splats eq1 blends front to back.
//
// The required order of every tile's list is (float32 depth bits, Gaussian id).
// The visible records are compacted in record order and sorted by depth once
// (stable LSD radix, so equal depths stay in id order; with several views, one
// more stable pass on the view index keeps each view's records together).  The
// (tile, Gaussian) pairs are then never sorted: two stable partitions -- records
// into the tile rows their rect spans, then each row's records into the row's
// tiles their support ellipse reaches -- write every pair straight to its place
// in (tile, depth, id) order.
//
// The radix sort is LSD with 8-bit digits in one sweep per pass: one kernel
// histograms every pass's digits, then each pass is one kernel whose CTAs rank a
// 1024-item tile stably with per-bit warp ballots, learn the counts of the earlier
// tiles by a decoupled look-back (bounded waits), reorder the tile in shared
// memory and write each digit run coalesced.  Every count the kernels need lives
// on the device, so the whole binning can be captured in a CUDA graph.
#include "common.cuh"

namespace fgs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;  // 1024: ~150 tiles for 150k records, every SM busy
constexpr int kSortMaxPasses = 4;

__device__ __forceinline__ uint32_t item_count(const int64_t *d_count, int64_t host_count, int64_t cap) {
  int64_t c = d_count ? *d_count : host_count;
  if (c > cap) c = cap;
  if (c < 0) c = 0;
  return (uint32_t)c;
}

// Lanes of the warp whose digit (the low `nbits` bits of d) equals this lane's,
// among the valid lanes: one ballot per digit bit, so the cost does not depend on
// how many distinct digits the warp holds.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid, int nbits) {
  uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < nbits) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
  }
  return peers;
}

// Exclusive scan over the values of a 256-thread block (one per thread) with
// warp shuffles; `total` receives the sum.  s_warp holds 8 words; the caller
// synchronises before s_warp is written again.
__device__ __forceinline__ uint32_t block_scan256(uint32_t x, uint32_t *s_warp, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) {
    const uint32_t t = s_warp[w];
    before += (w < warp) ? t : 0u;
    all += t;
  }
  total = all;
  return before + incl - x;
}

// Digit histograms of every pass in one sweep over the keys: hist[p][d] = items
// whose digit p ((key >> 8 p) & 255, the last pass masked to its bits) is d.
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t *__restrict__ keys,
                                                            const int64_t *d_count, int64_t host_count,
                                                            int64_t cap, int bits, uint32_t *__restrict__ hist) {
  pdl_enter();
  __shared__ uint32_t h[kSortMaxPasses][256];
  for (int i = threadIdx.x; i < kSortMaxPasses * 256; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int passes = (bits + 7) / 8;
  const uint32_t count = item_count(d_count, host_count, cap);
  const uint32_t stride = gridDim.x * kSortThreads;
  // every lane walks the same number of rounds, so the warp-wide match below is safe
  const uint32_t rounds = (count + stride - 1) / stride;
  uint32_t i = blockIdx.x * kSortThreads + threadIdx.x;
  for (uint32_t r = 0; r < rounds; ++r, i += stride) {
    const bool valid = i < count;
    const uint32_t k = valid ? keys[i] : 0u;
#pragma unroll
    for (int p = 0; p < kSortMaxPasses; ++p) {
      if (p < passes) {
        const int nb = min(8, bits - 8 * p);
        const uint32_t d = (k >> (8 * p)) & ((1u << nb) - 1u);
        // lanes with the same digit add once (the high digits repeat across the warp)
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0xFFFFFFFFu);
        if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < passes * 256; e += kSortThreads) {
    const uint32_t c = (&h[0][0])[e];
    if (c) atomicAdd(hist + e, c);
  }
}

// Look-back flags: one word per (tile, digit), the tile's count of the digit in
// the low 30 bits and its state in the top two: 0 not yet known, kFlagAgg the
// tile's own count, kFlagPrefix the count of this and every earlier tile.
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPrefix = 2u << 30, kFlagValue = (1u << 30) - 1u;
constexpr uint64_t kLookbackTimeoutNs = 1000000000ull;  // 1 s
constexpr int kLookback = 32;  // earlier tiles read per look-back step (loads in flight per thread)

__device__ __forceinline__ uint32_t ld_flag(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_flag(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t sort_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread d's decoupled look-back for tile t over flags [tiles][256]: the sum of
// digit d's counts over tiles 0 .. t - 1, reading kLookback earlier tiles' flags
// at a time and summing own counts until it meets a running prefix.  A flag that
// stays unknown for timeout_ns sets FGS_DEV_TIMEOUT and ends the wait (the sum is
// then incomplete).
__device__ __forceinline__ uint32_t lookback_sum(const uint32_t *flags, uint32_t t, int d, uint64_t timeout_ns,
                                                 int32_t *d_status) {
  uint32_t excl = 0;
  int64_t j = (int64_t)t - 1;
  const uint64_t t0 = sort_ns();
  for (;;) {
    uint32_t f[kLookback];
#pragma unroll
    for (int q = 0; q < kLookback; ++q) f[q] = j - q >= 0 ? ld_flag(flags + (size_t)(j - q) * 256 + d) : kFlagPrefix;
    int q = 0;
    bool done = false;
#pragma unroll
    for (; q < kLookback; ++q) {
      const uint32_t st = f[q] & ~kFlagValue;
      if (st == 0) break;  // not yet published: read again from here
      excl += f[q] & kFlagValue;
      if (st == kFlagPrefix) {
        done = true;
        break;
      }
    }
    if (done) break;
    j -= q;
    if (q == 0 && sort_ns() - t0 > timeout_ns) {
      if (d_status) atomicOr(d_status, FGS_DEV_TIMEOUT);
      break;
    }
  }
  return excl;
}

// The look-back alone, for its self-test: each CTA takes a tile by ticket and
// publishes a count of 1 for each of the 256 digits, except the first tile when
// skip_first (its flags then never become known, so every later wait can only end
// by its limit); each tile's sums go to sums[t][d].
__global__ void __launch_bounds__(kSortThreads) k_lookback_probe(uint32_t *__restrict__ flags,
                                                                 uint32_t *__restrict__ ticket, int skip_first,
                                                                 int64_t timeout_ns, int32_t *__restrict__ sums,
                                                                 int32_t *d_status) {
  __shared__ uint32_t s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int d = threadIdx.x;
  if (t == 0 && skip_first) return;
  st_flag(flags + (size_t)t * 256 + d, (t == 0 ? kFlagPrefix : kFlagAgg) | 1u);
  const uint32_t excl = t > 0 ? lookback_sum(flags, t, d, (uint64_t)timeout_ns, d_status) : 0u;
  if (t > 0) st_flag(flags + (size_t)t * 256 + d, kFlagPrefix | (excl + 1u));
  sums[(size_t)t * 256 + d] = (int32_t)excl;
}

// One stable LSD pass over the digit (key >> shift) & (2^nbits - 1).  Each CTA
// takes the next 1024-item tile by ticket (so every tile it waits for belongs to
// a CTA that is already running), ranks the tile stably with per-bit warp ballots,
// publishes its digit counts, and adds up the counts of the earlier tiles by a
// decoupled look-back: thread d reads the flags of kLookback earlier tiles at a
// time for digit d, summing own counts until it meets a running prefix.  A flag that
// stays unknown for kLookbackTimeoutNs sets FGS_DEV_TIMEOUT (the pass's output is
// then invalid) and the CTA goes on.  The tile is reordered in shared memory and
// each digit run is written out coalesced.
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const int64_t *d_count, int64_t host_count, int64_t cap, int shift, int nbits,
    const uint32_t *__restrict__ hist, uint32_t *__restrict__ flags, uint32_t *__restrict__ ticket,
    int32_t *d_status) {
  pdl_enter();
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t s_whist[W][256];  // per warp and digit: count, then the warp's offset in the tile's run
  __shared__ uint32_t s_base[256];      // output position of the tile's first item of each digit
  __shared__ uint32_t s_prefix[256];    // start of each digit's run in the reordered tile
  __shared__ uint32_t s_warp[W];
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t count = item_count(d_count, host_count, cap);
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  for (int d = lane; d < 256; d += 32) s_whist[warp][d] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t lo = t * (uint32_t)kSortTile;
  if (lo >= count) return;  // past the last tile (the whole CTA)
  const uint32_t hi = min(count, lo + (uint32_t)kSortTile);
  uint32_t k[kSortItems], v[kSortItems], local[kSortItems], dig[kSortItems];
  bool valid[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const uint32_t idx = lo + warp * (32 * kSortItems) + it * 32 + lane;
    valid[it] = idx < hi;
    k[it] = valid[it] ? keys_in[idx] : 0u;
    v[it] = valid[it] ? vals_in[idx] : 0u;
    dig[it] = (k[it] >> shift) & ((1u << nbits) - 1u);
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const uint32_t peers = digit_peers(dig[it], valid[it], nbits);
    uint32_t base = 0;
    if (valid[it]) base = s_whist[warp][dig[it]];
    __syncwarp();
    if (valid[it] && lane == __ffs(peers) - 1) s_whist[warp][dig[it]] = base + __popc(peers);
    __syncwarp();
    local[it] = base + __popc(peers & lt_mask);
  }
  __syncthreads();
  const int d = threadIdx.x;  // this thread's digit
  uint32_t run = 0;           // items of digit d in the tile
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = run;
    run += c;
  }
  uint32_t *my_flags = flags + (size_t)t * 256;
  st_flag(my_flags + d, (t == 0 ? kFlagPrefix : kFlagAgg) | run);
  uint32_t tile_items, all;
  s_prefix[d] = block_scan256(run, s_warp, tile_items);
  __syncthreads();
  const uint32_t digit_start = block_scan256(hist[d], s_warp, all);
  // look-back over the earlier tiles for digit d
  uint32_t excl = 0;
  if (t > 0) {
    excl = lookback_sum(flags, t, d, kLookbackTimeoutNs, d_status);
    st_flag(my_flags + d, kFlagPrefix | (excl + run));
  }
  s_base[d] = digit_start + excl;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    if (valid[it]) {
      const uint32_t pos = s_prefix[dig[it]] + s_whist[warp][dig[it]] + local[it];
      s_keys[pos] = k[it];
      s_vals[pos] = v[it];
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < tile_items; i += kSortThreads) {
    const uint32_t key = s_keys[i];
    const uint32_t dd = (key >> shift) & ((1u << nbits) - 1u);
    const uint32_t out = s_base[dd] + (i - s_prefix[dd]);
    if (out < count) {  // always, unless a look-back gave up
      keys_out[out] = key;
      vals_out[out] = s_vals[i];
    }
  }
}

// Scratch of a sort over at most `cap` items: the pass histograms and tickets, then
// the look-back flags of every pass, cleared by one memset per sort.
struct SortWs {
  uint32_t *hist;    // [kSortMaxPasses][256]
  uint32_t *ticket;  // [kSortMaxPasses] (+ padding)
  uint32_t *flags;   // [kSortMaxPasses][tiles][256]
  int64_t tiles;
  size_t bytes;      // the whole block, cleared per sort
};

static size_t sort_ws_bytes(int64_t cap) {
  const int64_t tiles = std::max<int64_t>(1, (cap + kSortTile - 1) / kSortTile);
  return (size_t)kSortMaxPasses * 256 * 4 + 256 + (size_t)kSortMaxPasses * tiles * 256 * 4;
}

static SortWs sort_ws(void *base, int64_t cap) {
  SortWs w;
  w.tiles = std::max<int64_t>(1, (cap + kSortTile - 1) / kSortTile);
  char *p = static_cast<char *>(base);
  w.hist = reinterpret_cast<uint32_t *>(p);
  w.ticket = reinterpret_cast<uint32_t *>(p + (size_t)kSortMaxPasses * 256 * 4);
  w.flags = reinterpret_cast<uint32_t *>(p + (size_t)kSortMaxPasses * 256 * 4 + 256);
  w.bytes = sort_ws_bytes(cap);
  return w;
}

// Stable LSD sort of (key, value) over bits [0, bits) of at most `cap` items
// (the count on the device when d_count is set).  Result lands in (k0, v0) when
// the number of passes is even, in (k1, v1) otherwise.  clear = false when the
// caller has already zeroed w's block.
static fgs_status radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const int64_t *d_count,
                             int64_t host_count, int64_t cap, int bits, const SortWs &w, int32_t *d_status,
                             cudaStream_t st, bool clear = true, bool hist_ready = false) {
  const int passes = (bits + 7) / 8;
  if (passes < 1 || passes > kSortMaxPasses || cap > (int64_t)kFlagValue) {
    set_error("radix_sort: %d key bits over up to %lld items", bits, (long long)cap);
    return FGS_ERR_INVALID_ARGUMENT;
  }
  if (clear) FGS_CUDA(cudaMemsetAsync(w.hist, 0, w.bytes, st), "radix_sort: clear");
  const int hist_grid = (int)std::max<int64_t>(1, std::min<int64_t>(w.tiles, 2 * (int64_t)num_sms()));
  if (!hist_ready) pdl_launch(k_sort_hist, hist_grid, kSortThreads, 0, st, k0, d_count, host_count, cap, bits, w.hist);
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const int nbits = std::min(8, bits - shift);
    uint32_t *ki = (p & 1) ? k1 : k0, *vi = (p & 1) ? v1 : v0;
    uint32_t *ko = (p & 1) ? k0 : k1, *vo = (p & 1) ? v0 : v1;
    pdl_launch(k_sort_pass, (int)w.tiles, kSortThreads, 0, st, ki, vi, ko, vo, d_count, host_count, cap, shift,
               nbits, w.hist + 256 * p, w.flags + (size_t)p * w.tiles * 256, w.ticket + p, d_status);
  }
  count_launch((hist_ready ? 0 : 1) + passes);
  FGS_CHECK_LAUNCH("radix_sort");
  return FGS_OK;
}

// ---------------------------------------------------------------------------------
// Visible records (radius > 0 and at least one tile) are compacted in record
// order before the depth sort, so the sort touches only them: a block count, a
// scan of the block counts, and an ordered scatter of (depth bits, record).


__device__ __forceinline__ bool record_visible(const int32_t *__restrict__ radius, const uint2 *__restrict__ rect,
                                               int64_t r) {
  if (radius[r] <= 0) return false;
  const uint2 rc = rect[r];
  return (rc.x & 0xFFFFu) <= (rc.y & 0xFFFFu) && (rc.x >> 16) <= (rc.y >> 16);
}

// record index of compact slot j (j < n_views * n): view-major, ids ascending
__device__ __forceinline__ int64_t record_of(int64_t j, int64_t n, int64_t stride) {
  const int64_t v = j / n;
  return v * stride + (j - v * n);
}

// Ordered compaction of the visible records in one pass: each CTA takes the next
// tile of kVisTile records by ticket (warp w holds records w * 256 .. + 255 of it,
// eight per lane in record order), counts its visible records, publishes the
// count, adds up the earlier tiles' counts by a decoupled look-back (its first
// warp reads 32 earlier tiles' flags at a time; flags as in k_sort_pass, bounded
// waits) and writes (depth bits, record) of its visible records in record order.
// The CTA of the last tile stores the total.
constexpr int kVisThreads = 512;
constexpr int kVisItems = 8;
constexpr int kVisTile = kVisThreads * kVisItems;  // 4096 records: ~250 tiles for a 1M map, one wave

__global__ void __launch_bounds__(kVisThreads) k_vis_compact(const float4 *__restrict__ splat,
                                                            const int32_t *__restrict__ radius,
                                                            const uint2 *__restrict__ rect, int64_t n_max,
                                                            const int64_t *__restrict__ d_n, int64_t stride,
                                                            int64_t R_max, uint32_t *__restrict__ flags,
                                                            uint32_t *__restrict__ ticket, int64_t *__restrict__ total,
                                                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                            uint32_t *__restrict__ hist, int32_t *d_status) {
  pdl_enter();
  constexpr int NW = kVisThreads / 32;
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t s_tile, s_excl, s_count;
  __shared__ uint32_t s_hist[4][256];  // the depth sort's four digit histograms of this tile's keys
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 4 * 256; i += kVisThreads) (&s_hist[0][0])[i] = 0u;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  // the records of the live slots only: n per view, the grid sized for n_max
  const int64_t n = live_count(d_n, n_max), R = R_max / n_max * n;
  const int64_t nt = (R + kVisTile - 1) / kVisTile;
  if ((int64_t)t >= nt) {  // (the whole CTA)
    if (t == 0 && threadIdx.x == 0) *total = 0;  // no live record at all
    return;
  }
  const int64_t j0 = (int64_t)t * kVisTile + warp * (32 * kVisItems) + lane;
  int64_t r[kVisItems];
  int32_t rad[kVisItems];
  uint2 rc[kVisItems];
  // every item's radius and rect are requested before any is tested: 16 loads in flight
#pragma unroll
  for (int it = 0; it < kVisItems; ++it) {
    const int64_t j = j0 + it * 32;
    r[it] = j < R ? record_of(j, n, stride) : 0;
    rad[it] = j < R ? radius[r[it]] : 0;
    rc[it] = j < R ? rect[r[it]] : make_uint2(1u, 0u);
  }
  uint32_t bal[kVisItems];
  uint32_t wcount = 0;
#pragma unroll
  for (int it = 0; it < kVisItems; ++it) {
    const bool vis = rad[it] > 0 && (rc[it].x & 0xFFFFu) <= (rc[it].y & 0xFFFFu) && (rc[it].x >> 16) <= (rc[it].y >> 16);
    bal[it] = __ballot_sync(0xffffffffu, vis);
    wcount += __popc(bal[it]);
  }
  if (lane == 0) wsum[warp] = wcount;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < NW ? wsum[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    wsum[lane] = wi - w;
    const uint32_t count = __shfl_sync(0xffffffffu, wi, 31);  // this tile's visible records
    if (lane == 0) st_flag(flags + t, (t == 0 ? kFlagPrefix : kFlagAgg) | count);
    uint32_t excl = 0;
    if (t > 0) {
      int64_t jn = (int64_t)t - 1;  // nearest tile not yet added
      const uint64_t t0 = sort_ns();
      for (;;) {
        const int64_t jj = jn - lane;
        const uint32_t f = jj >= 0 ? ld_flag(flags + jj) : kFlagPrefix;
        const uint32_t stat = f & ~kFlagValue;
        const uint32_t stop = __ballot_sync(0xffffffffu, stat != kFlagAgg);  // unknown or running prefix
        const int s = stop ? __ffs(stop) - 1 : 32;
        const bool prefix = s < 32 && __shfl_sync(0xffffffffu, stat, s & 31) == kFlagPrefix;
        uint32_t add = (lane < s || (prefix && lane == s)) ? (f & kFlagValue) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
        excl += add;
        if (prefix) break;
        jn -= s;
        if (s == 0 && sort_ns() - t0 > kLookbackTimeoutNs) {
          if (lane == 0 && d_status) atomicOr(d_status, FGS_DEV_TIMEOUT);
          break;
        }
      }
      if (lane == 0) st_flag(flags + t, kFlagPrefix | (excl + count));
    }
    if (lane == 0) {
      s_excl = excl;
      s_count = count;
    }
  }
  __syncthreads();
  if ((int64_t)t == nt - 1 && threadIdx.x == 0) *total = (int64_t)s_excl + s_count;
  uint32_t pos = s_excl + wsum[warp];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int it = 0; it < kVisItems; ++it) {
    const bool mine = (bal[it] >> lane) & 1u;
    const uint32_t key = mine ? __float_as_uint(splat[2 * r[it] + 1].z) : 0u;  // depth > 0: bits order like it
    if (mine) {
      const uint32_t q = pos + __popc(bal[it] & lt);
      if ((int64_t)q < R) {  // always, unless a look-back gave up
        keys[q] = key;
        vals[q] = (uint32_t)r[it];
      }
    }
    pos += __popc(bal[it]);
    if (hist && bal[it]) {  // lanes with the same digit add once (the high digits repeat across the warp)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint32_t d = (key >> (8 * p)) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, mine ? d : 0xFFFFFFFFu);
        if (mine && lane == __ffs(peers) - 1) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
      }
    }
  }
  if (hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += kVisThreads) {
      const uint32_t c = (&s_hist[0][0])[i];
      if (c) atomicAdd(hist + i, c);
    }
  }
}


// ---------------------------------------------------------------------------------
// Tile lists by row partition.
//
// The depth-sorted visible records are partitioned twice, each time stably, so
// that every list keeps depth order without a sort of the pairs:
//   rows:  the records whose rect spans tile row g, for every global row g
//          (views after one another), in depth order;
//   tiles: each row's list cut into chunks of kTileChunk entries; within its row a
//          record keeps the rect's tiles that its support ellipse reaches, and a
//          chunk writes its pairs of tile x after those of the row's earlier
//          chunks: positions come from per-(chunk, x) counts scanned over the
//          row's chunks, per-warp counts scanned over the chunk's warps and
//          ballot ranks within a warp.
// Rows ordered by view then y, tiles of a row by x: the pairs come out sorted by
// global tile, then depth, then id, and each step is a counting pass, a scan and
// a writing pass over small per-chunk tables.

constexpr int kRecChunk = 256;    // records per chunk of the row partition
constexpr int kTileChunk = 512;   // row-list entries per chunk of the tile partition
constexpr int kMaxRows = 4096;    // global tile rows (shared-memory row histogram)
constexpr int kPartGrid = 8;      // persistent CTAs per SM of the partition kernels

struct RowGeom {
  int n_views, n_rows, tx_max;
  int64_t stride;
  int row_base[FGS_MAX_VIEWS + 1];  // first global row of each view
  int tiles_x[FGS_MAX_VIEWS];
  int tile_base[FGS_MAX_VIEWS];
};

__device__ __forceinline__ int view_of_row(const RowGeom &G, int g) {
  int v = 0;
#pragma unroll 1
  while (v + 1 < G.n_views && g >= G.row_base[v + 1]) ++v;
  return v;
}

__device__ __forceinline__ void record_rows(const RowGeom &G, const uint2 *__restrict__ rect, uint32_t rec, int &g0,
                                            int &g1) {
  const int v = (int)(rec / (uint64_t)G.stride);
  const uint2 rc = rect[rec];
  g0 = G.row_base[v] + (int)(rc.x >> 16);
  g1 = G.row_base[v] + (int)(rc.y >> 16);
}

// Exclusive scan of one value per thread over a CTA of 1024 threads with warp
// shuffles and two barriers; `total` receives the sum.  s_warp holds 33 words;
// the caller synchronises before s_warp is written again.
__device__ __forceinline__ unsigned long long cta1024_exclusive(unsigned long long x, unsigned long long *s_warp,
                                                                unsigned long long &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = s_warp[lane];
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  return s_warp[warp] + v - x;
}

// Exclusive scan of n counts in place by one CTA of 1024 threads (a consecutive
// slice per thread); every thread gets the total.
__device__ uint64_t cta_scan_inplace(uint32_t *__restrict__ a, int64_t n, unsigned long long *part) {
  const int64_t per = (n + 1023) / 1024;
  const int64_t lo = threadIdx.x * per, hi = min(n, lo + per);
  unsigned long long s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  unsigned long long total;
  unsigned long long run = cta1024_exclusive(s, part, total);
  for (int64_t i = lo; i < hi; ++i) {
    const uint32_t v = a[i];
    a[i] = (uint32_t)run;
    run += v;
  }
  __syncthreads();
  return total;
}

// 32x32 bit transpose across a warp: on entry bit b of lane L's word is entry
// (L, b); on return lane b holds column b, i.e. the ballot of bit b over the
// warp.  Five exchange stages swap the off-diagonal blocks of size 16, 8, .., 1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  constexpr uint32_t kHi[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint32_t t = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & kHi[s]) | ((t >> j) & ~kHi[s])) : ((x & ~kHi[s]) | ((t << j) & kHi[s]));
  }
  return x;
}

// Stable multi-bin ranking in one warp: lane L belongs to bin b (of 32) where bit
// b of its m is set.  s_wc_row[b] receives the warp's count of bin b; the return
// value is column `lane` (the lanes in bin `lane`), from which a lane's rank in
// bin b is popc(column b & lanes below it).
__device__ __forceinline__ uint32_t warp_bin_counts(uint32_t m, int lane, uint32_t *s_wc_row) {
  const uint32_t col = warp_transpose32(m, lane);
  s_wc_row[lane] = __popc(col);
  return col;
}

// Rows, counting pass: per record chunk b, the number of its records spanning each
// global row, into rowcnt[g * nb_cap + b].
__global__ void __launch_bounds__(kRecChunk) k_row_count(RowGeom G, const uint32_t *__restrict__ srec,
                                                         const uint2 *__restrict__ rect,
                                                         const int64_t *__restrict__ d_vis, int64_t nb_cap,
                                                         uint32_t *__restrict__ rowcnt) {
  pdl_enter();
  __shared__ uint32_t s_rows[kMaxRows];
  const int64_t R = *d_vis;
  const int64_t nb = (R + kRecChunk - 1) / kRecChunk;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    for (int g = threadIdx.x; g < G.n_rows; g += kRecChunk) s_rows[g] = 0;
    __syncthreads();
    const int64_t j = b * kRecChunk + threadIdx.x;
    if (j < R) {
      int g0, g1;
      record_rows(G, rect, srec[j], g0, g1);
      for (int g = g0; g <= g1; ++g) atomicAdd(&s_rows[g], 1u);
    }
    __syncthreads();
    for (int g = threadIdx.x; g < G.n_rows; g += kRecChunk) rowcnt[(int64_t)g * nb_cap + b] = s_rows[g];
    __syncthreads();
  }
}

// Rows, scan: one CTA per row turns its chunk counts into exclusive offsets and
// writes the row's total.
__global__ void __launch_bounds__(1024) k_row_scan(const int64_t *__restrict__ d_vis, int64_t nb_cap,
                                                   uint32_t *__restrict__ rowcnt, uint32_t *__restrict__ rowtot) {
  pdl_enter();
  __shared__ unsigned long long part[33];
  const int64_t nb = (*d_vis + kRecChunk - 1) / kRecChunk;
  const uint64_t total = cta_scan_inplace(rowcnt + (int64_t)blockIdx.x * nb_cap, nb, part);
  if (threadIdx.x == 0) rowtot[blockIdx.x] = (uint32_t)min(total, (uint64_t)0xFFFFFFFFu);
}

// Rows, starts and the tile chunk table (one CTA): row_start[g] (exclusive scan of
// the row totals, total entries at [n_rows]); on overflow of the row-list
// capacity the status bit is set and every row is left empty.  chunk_start[g]:
// first tile chunk of row g, chunk_row[c]: row of chunk c, *d_nchunks: count.
__global__ void __launch_bounds__(1024) k_row_starts(RowGeom G, const uint32_t *__restrict__ rowtot,
                                                     int64_t row_cap, uint32_t *__restrict__ row_start,
                                                     uint32_t *__restrict__ chunk_start,
                                                     uint32_t *__restrict__ chunk_row, int64_t chunk_cap,
                                                     int64_t *__restrict__ d_nchunks, int32_t *__restrict__ d_status,
                                                     int64_t *__restrict__ d_num_pairs,
                                                     int64_t *__restrict__ d_sort_count) {
  pdl_enter();
  __shared__ unsigned long long part[33];
  __shared__ int s_over;
  const int NR = G.n_rows;
  for (int g = threadIdx.x; g < NR; g += 1024) row_start[g] = rowtot[g];
  __syncthreads();
  const uint64_t E = cta_scan_inplace(row_start, NR, part);
  if (threadIdx.x == 0) {
    s_over = E > (uint64_t)row_cap;
    row_start[NR] = s_over ? 0u : (uint32_t)E;
    // -1 marks the overflow for k_tile_row_starts, which sets the final count
    *d_sort_count = s_over ? -1 : 0;
    if (s_over) {
      if (d_status) atomicOr(d_status, FGS_DEV_PAIR_OVERFLOW);
      *d_num_pairs = (int64_t)E;  // a lower bound of the pairs needed
    }
  }
  __syncthreads();
  const bool over = s_over;
  for (int g = threadIdx.x; g < NR; g += 1024) {
    if (over) row_start[g] = 0;
    chunk_start[g] = over ? 0u : (rowtot[g] + kTileChunk - 1) / kTileChunk;
  }
  __syncthreads();
  const uint64_t NC = cta_scan_inplace(chunk_start, NR, part);
  if (threadIdx.x == 0) {
    chunk_start[NR] = (uint32_t)NC;
    *d_nchunks = (int64_t)min(NC, (uint64_t)chunk_cap);
  }
  __syncthreads();
  const int64_t nc = (int64_t)min(NC, (uint64_t)chunk_cap);
  for (int64_t c = threadIdx.x; c < nc; c += 1024) {  // row of chunk c: last g with chunk_start[g] <= c
    int lo = 0, hi = NR - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_start[mid] <= (uint64_t)c) lo = mid;
      else hi = mid - 1;
    }
    chunk_row[c] = (uint32_t)lo;
  }
}

// Rows, writing pass: record j (depth rank) goes to rowlist at row_start[g] + the
// offset of its chunk in row g + its rank among the chunk's earlier records that
// span g (warp prefix in shared memory, ballot rank inside the warp).
__global__ void __launch_bounds__(kRecChunk) k_row_emit(RowGeom G, const uint32_t *__restrict__ srec,
                                                        const uint2 *__restrict__ rect,
                                                        const int64_t *__restrict__ d_vis, int64_t nb_cap,
                                                        const uint32_t *__restrict__ rowcnt,
                                                        const uint32_t *__restrict__ row_start,
                                                        uint32_t *__restrict__ rowlist) {
  pdl_enter();
  constexpr int NW = kRecChunk / 32;
  __shared__ uint32_t s_wc[NW][32];
  __shared__ int s_lo, s_hi;
  const int64_t R = *d_vis;
  const int64_t nb = (R + kRecChunk - 1) / kRecChunk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if (row_start[G.n_rows] == 0) return;  // no entries, or the row lists overflowed
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    if (threadIdx.x == 0) {
      s_lo = 0x7FFFFFFF;
      s_hi = -1;
    }
    __syncthreads();
    const int64_t j = b * kRecChunk + threadIdx.x;
    int g0 = 0, g1 = -1;
    if (j < R) record_rows(G, rect, srec[j], g0, g1);
    if (g0 <= g1) {
      atomicMin(&s_lo, g0);
      atomicMax(&s_hi, g1);
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    for (int gb = lo; gb <= hi; gb += 32) {
      // rows gb .. gb + 31 this record spans, as bits
      uint32_t m = 0;
      if (g0 <= g1 && g1 >= gb && g0 < gb + 32) {
        const int a = max(g0, gb) - gb, e = min(g1, gb + 31) - gb;
        m = (e == 31 ? 0xFFFFFFFFu : ((1u << (e + 1)) - 1u)) & ~((1u << a) - 1u);
      }
      const uint32_t col = warp_bin_counts(m, lane, s_wc[warp]);
      __syncthreads();
      // lane L: first position of row gb + L for this warp's records
      uint32_t before = 0;
      for (int w = 0; w < warp; ++w) before += s_wc[w][lane];
      if (gb + lane < G.n_rows) before += row_start[gb + lane] + rowcnt[(int64_t)(gb + lane) * nb_cap + b];
      for (uint32_t rem = m; __any_sync(0xffffffffu, rem != 0u);) {
        const int bit = rem ? __ffs(rem) - 1 : 0;
        const uint32_t c = __shfl_sync(0xffffffffu, col, bit);
        const uint32_t base = __shfl_sync(0xffffffffu, before, bit);
        if (rem) {
          rowlist[base + __popc(c & lt)] = (uint32_t)j;
          rem &= rem - 1u;
        }
      }
      __syncthreads();
    }
  }
}

struct TileChunk {
  int g, v, y, tx;
  uint32_t e0, e1;
};

__device__ __forceinline__ TileChunk tile_chunk(const RowGeom &G, const uint32_t *__restrict__ chunk_row,
                                                const uint32_t *__restrict__ chunk_start,
                                                const uint32_t *__restrict__ row_start, int64_t c) {
  TileChunk k;
  k.g = (int)chunk_row[c];
  k.v = view_of_row(G, k.g);
  k.y = k.g - G.row_base[k.v];
  k.tx = G.tiles_x[k.v];
  k.e0 = row_start[k.g] + (uint32_t)(c - chunk_start[k.g]) * kTileChunk;
  k.e1 = min(k.e0 + kTileChunk, row_start[k.g + 1]);
  return k;
}

// One row-list entry as the tile writing pass needs it: Gaussian id and the kept
// tile columns a | b << 16 (a > b: none).
struct EntryInfo {
  uint32_t id, xr;
};

// The tiles of rect columns [x0, x1] in tile row y that a splat keeps.  It can
// reach alpha >= 1/255 only inside E = {q <= thr}, q = a dx^2 + 2 b dx dy + c dy^2;
// a tile spans the row's pixel-centre rows, so it meets E iff its pixel-centre
// columns meet [xl, xr], E's x-extent within that strip.  E's left boundary is
// convex in dy with its minimum -sqrt(thr c / det) at dy = b sqrt(thr c / det) / c
// (det = a c - b^2); over the strip cut to E's y-range the leftmost point lies at
// that dy clamped into the range, the rightmost one mirrors it.  Every step is
// rounded to float32 in a fixed order (explicit intrinsics), so the decision is
// the same wherever it is taken.  Writes a > b when no tile is kept.
__device__ __forceinline__ void kept_columns(float mx, float my, float a, float b, float c, float thr, int x0, int x1,
                                             int y, int tw, int th, int &ta, int &tb) {
  ta = 1;
  tb = 0;
  const float y0 = __fsub_rn((float)(y * th), my), y1 = __fsub_rn((float)(y * th + th - 1), my);
  const float det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
  if (!(det > 0.f) || !(thr >= 0.f)) return;
  const float tA = __fmul_rn(thr, a);
  const float ys = __fsqrt_rn(__fdiv_rn(tA, det)), xs = __fsqrt_rn(__fdiv_rn(__fmul_rn(thr, c), det));
  const float lo = fmaxf(y0, -ys), hi = fminf(y1, ys);
  if (lo > hi) return;
  const float dl = __fdiv_rn(__fmul_rn(b, xs), c);
  const float yl = fminf(fmaxf(dl, lo), hi), yr = fminf(fmaxf(-dl, lo), hi);
  const float rl = __fsqrt_rn(fmaxf(__fsub_rn(tA, __fmul_rn(det, __fmul_rn(yl, yl))), 0.f));
  const float rr = __fsqrt_rn(fmaxf(__fsub_rn(tA, __fmul_rn(det, __fmul_rn(yr, yr))), 0.f));
  const float xl = __fdiv_rn(__fsub_rn(-__fmul_rn(b, yl), rl), a);
  const float xr = __fdiv_rn(__fadd_rn(-__fmul_rn(b, yr), rr), a);
  // tile t is kept iff t tw + tw - 1 >= mx + xl and t tw <= mx + xr (clamped in
  // float to [x0 - 1, x1 + 1] before the conversion)
  const float fa = fminf(fmaxf(ceilf(__fdiv_rn(__fsub_rn(__fadd_rn(mx, xl), (float)(tw - 1)), (float)tw)), (float)x0),
                         (float)x1 + 1.f);
  const float fb = fminf(fmaxf(floorf(__fdiv_rn(__fadd_rn(mx, xr), (float)tw)), (float)x0 - 1.f), (float)x1);
  ta = (int)fa;
  tb = (int)fb;
  if (ta > tb) {
    ta = 1;
    tb = 0;
  }
}

// Tiles, counting pass: per chunk c of a row list, the number of its records that
// keep tile x of the row, into tcnt[c * tx_max + x], and every entry's EntryInfo.
// A thread finds its own record's kept columns.
__global__ void __launch_bounds__(kTileChunk) k_tile_count(RowGeom G, const float4 *__restrict__ splat,
                                                           const uint32_t *__restrict__ srec,
                                                           const uint2 *__restrict__ rect, int tw, int th,
                                                           const uint32_t *__restrict__ rowlist,
                                                           const uint32_t *__restrict__ row_start,
                                                           const uint32_t *__restrict__ chunk_start,
                                                           const uint32_t *__restrict__ chunk_row,
                                                           const int64_t *__restrict__ d_nchunks,
                                                           uint32_t *__restrict__ tcnt,
                                                           EntryInfo *__restrict__ einfo) {
  pdl_enter();
  extern __shared__ uint32_t s_cnt[];  // [tx_max + 1]: +1 at each kept interval's start, -1 past its end
  const int64_t NC = *d_nchunks;
  const int lane = threadIdx.x & 31;
  for (int64_t c = blockIdx.x; c < NC; c += gridDim.x) {
    const TileChunk k = tile_chunk(G, chunk_row, chunk_start, row_start, c);
    for (int x = threadIdx.x; x <= k.tx; x += kTileChunk) s_cnt[x] = 0;
    __syncthreads();
    const uint32_t e = k.e0 + threadIdx.x;
    if (e < k.e1) {
      const uint32_t rec = srec[rowlist[e]];
      const uint2 rc = rect[rec];
      const float4 s0 = splat[2 * (int64_t)rec], s1 = splat[2 * (int64_t)rec + 1];
      int a, b;
      kept_columns(s0.x, s0.y, s0.z, s0.w, s1.x, s1.w, (int)(rc.x & 0xFFFFu), (int)(rc.y & 0xFFFFu), k.y, tw, th, a,
                   b);
      if (a <= b) {
        atomicAdd(&s_cnt[a], 1u);
        atomicAdd(&s_cnt[b + 1], 0xFFFFFFFFu);  // -1 modulo 2^32
      }
      einfo[e] = EntryInfo{rec - (uint32_t)k.v * (uint32_t)G.stride, (uint32_t)a | ((uint32_t)b << 16)};
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // the differences summed along the row: the records keeping tile x
      uint32_t carry = 0;
      for (int xb = 0; xb < k.tx; xb += 32) {
        const int x = xb + lane;
        uint32_t v = x < k.tx ? s_cnt[x] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        v += carry;
        if (x < k.tx) tcnt[c * G.tx_max + x] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
      }
    }
    __syncthreads();
  }
}

// Tiles, scan over chunks: one CTA per row; tpre[c][x] = pairs of tile x in the
// row's chunks before c, ttot[g][x] = the tile's total, rowp[g] = the row's total.
// Lane L of every warp takes columns L, L + 32, ...; the eight warps split the
// row's chunks into eight consecutive ranges: each warp sums its range per column
// (all its loads in flight together), the ranges' sums are scanned across warps in
// shared memory, and each warp writes its range's prefixes.
__global__ void __launch_bounds__(256) k_tile_chunk_scan(RowGeom G, const uint32_t *__restrict__ chunk_start,
                                                         const uint32_t *__restrict__ tcnt,
                                                         uint32_t *__restrict__ tpre, uint32_t *__restrict__ ttot,
                                                         unsigned long long *__restrict__ rowp) {
  pdl_enter();
  constexpr int NW = 8;
  __shared__ uint32_t s_part[NW][128];  // per warp and column (columns in slices of 128)
  const int g = blockIdx.x;
  const int v = view_of_row(G, g);
  const int tx = G.tiles_x[v];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c0 = chunk_start[g], c1 = chunk_start[g + 1];
  const uint32_t nc = c1 - c0, per = (nc + NW - 1) / NW;
  const uint32_t ca = c0 + min(nc, warp * per), cb = c0 + min(nc, (warp + 1) * per);
  unsigned long long row_sum = 0;
  for (int xs = 0; xs < tx; xs += 128) {  // column slices of 128 (4 per lane)
    uint32_t sum[4] = {0u, 0u, 0u, 0u};
#pragma unroll 4
    for (uint32_t c = ca; c < cb; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = xs + lane + 32 * k;
        if (x < tx) sum[k] += tcnt[(int64_t)c * G.tx_max + x];
      }
#pragma unroll
    for (int k = 0; k < 4; ++k) s_part[warp][lane + 32 * k] = sum[k];
    __syncthreads();
    uint32_t run[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t before = 0, all = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t t = s_part[w][lane + 32 * k];
        before += w < warp ? t : 0u;
        all += t;
      }
      run[k] = before;
      const int x = xs + lane + 32 * k;
      if (warp == 0 && x < tx) {
        ttot[(int64_t)g * G.tx_max + x] = all;
        row_sum += all;
      }
    }
#pragma unroll 4
    for (uint32_t c = ca; c < cb; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = xs + lane + 32 * k;
        if (x < tx) {
          const uint32_t t = tcnt[(int64_t)c * G.tx_max + x];
          tpre[(int64_t)c * G.tx_max + x] = run[k];
          run[k] += t;
        }
      }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) row_sum += __shfl_xor_sync(0xffffffffu, row_sum, o);
  if (threadIdx.x == 0) rowp[g] = row_sum;
}

// Tiles, row starts (one CTA): exclusive scan of the rows' pair totals; the total
// is the pair count, checked against the capacity.
__global__ void __launch_bounds__(1024) k_tile_row_starts(RowGeom G, unsigned long long *__restrict__ rowp,
                                                          int64_t pair_cap, int64_t *__restrict__ d_num_pairs,
                                                          int32_t *__restrict__ d_status,
                                                          int64_t *__restrict__ d_sort_count) {
  pdl_enter();
  __shared__ unsigned long long part[33];
  const int NR = G.n_rows;
  const int per = (NR + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(NR, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += rowp[i];
  unsigned long long total;
  unsigned long long run = cta1024_exclusive(s, part, total);
  for (int i = lo; i < hi; ++i) {
    const unsigned long long v = rowp[i];
    rowp[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) {
    if (*d_sort_count < 0) {  // the row lists overflowed: no pairs, count already recorded
      *d_sort_count = 0;
    } else {
      *d_num_pairs = (int64_t)total;
      const bool over = total > (unsigned long long)pair_cap;
      if (over && d_status) atomicOr(d_status, FGS_DEV_PAIR_OVERFLOW);
      *d_sort_count = over ? 0 : (int64_t)total;
    }
  }
}

// Tiles, ranges: one CTA per row scans the row's tile totals: tstart[g][x] = first
// pair of tile x, tile_ranges = [start, end) ((0, 0) for an empty tile or when the
// pairs overflowed).
__global__ void __launch_bounds__(256) k_tile_ranges_rows(RowGeom G, const unsigned long long *__restrict__ rowp,
                                                          const uint32_t *__restrict__ ttot,
                                                          const int64_t *__restrict__ d_sort_count,
                                                          uint32_t *__restrict__ tstart,
                                                          int2 *__restrict__ ranges) {
  pdl_enter();
  __shared__ uint32_t s_warp[8];
  const int g = blockIdx.x;
  const int v = view_of_row(G, g);
  const int tx = G.tiles_x[v];
  const int y = g - G.row_base[v];
  const bool ok = *d_sort_count > 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t carry = (uint32_t)rowp[g];
  for (int xb = 0; xb < tx; xb += 256) {
    const int x = xb + threadIdx.x;
    const uint32_t t = x < tx ? ttot[(int64_t)g * G.tx_max + x] : 0u;
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < 8; ++w) {
      before += w < warp ? s_warp[w] : 0u;
      all += s_warp[w];
    }
    const uint32_t start = carry + before + incl - t;
    if (x < tx) {
      tstart[(int64_t)g * G.tx_max + x] = start;
      ranges[G.tile_base[v] + y * tx + x] = (ok && t > 0) ? make_int2((int)start, (int)(start + t)) : make_int2(0, 0);
    }
    carry += all;
    __syncthreads();
  }
}

// Tiles, writing pass: the chunk's records in order, 32 tiles of the row at a time;
// pair (tile x, record) goes to tstart[g][x] + tpre[c][x] + the pairs of x kept by
// the chunk's earlier warps + its rank among the warp's lanes that keep x.  The
// kept intervals come from the counting pass.
__global__ void __launch_bounds__(kTileChunk) k_tile_emit(RowGeom G, const uint32_t *__restrict__ row_start,
                                                          const uint32_t *__restrict__ chunk_start,
                                                          const uint32_t *__restrict__ chunk_row,
                                                          const int64_t *__restrict__ d_nchunks,
                                                          const EntryInfo *__restrict__ einfo,
                                                          const uint32_t *__restrict__ tpre,
                                                          const uint32_t *__restrict__ tstart,
                                                          const int64_t *__restrict__ d_sort_count,
                                                          uint32_t *__restrict__ tile_keys,
                                                          uint32_t *__restrict__ ids) {
  pdl_enter();
  constexpr int NW = kTileChunk / 32;
  extern __shared__ uint32_t s_base[];  // [tx_max]: first position of tile x for this chunk
  __shared__ uint32_t s_wc[NW][32];
  __shared__ int s_lo, s_hi;
  if (*d_sort_count == 0) return;
  const int64_t NC = *d_nchunks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  for (int64_t c = blockIdx.x; c < NC; c += gridDim.x) {
    const TileChunk k = tile_chunk(G, chunk_row, chunk_start, row_start, c);
    if (threadIdx.x == 0) {
      s_lo = 0x7FFFFFFF;
      s_hi = -1;
    }
    const int64_t trow = (int64_t)k.g * G.tx_max, crow = c * G.tx_max;
    for (int x = threadIdx.x; x < k.tx; x += kTileChunk) s_base[x] = tstart[trow + x] + tpre[crow + x];
    __syncthreads();
    const uint32_t e = k.e0 + threadIdx.x;
    int x0 = 1, x1 = 0;
    EntryInfo inf{0u, 1u};
    if (e < k.e1) {
      inf = einfo[e];
      x0 = (int)(inf.xr & 0xFFFFu);
      x1 = (int)(inf.xr >> 16);
      if (x0 <= x1) {
        atomicMin(&s_lo, x0);
        atomicMax(&s_hi, x1);
      }
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    const uint32_t tbase = (uint32_t)(G.tile_base[k.v] + k.y * k.tx);
    for (int xb = lo; xb <= hi; xb += 32) {
      uint32_t m = 0;  // tiles xb .. xb + 31 this record keeps: bits a - xb .. b - xb
      const int a = max(x0, xb), b = min(x1, xb + 31);
      if (a <= b) m = (b - xb == 31 ? 0xFFFFFFFFu : ((1u << (b - xb + 1)) - 1u)) & ~((1u << (a - xb)) - 1u);
      const uint32_t col = warp_bin_counts(m, lane, s_wc[warp]);
      __syncthreads();
      uint32_t before = xb + lane < k.tx ? s_base[xb + lane] : 0u;
      for (int w = 0; w < warp; ++w) before += s_wc[w][lane];
      // tile by tile, so that the lanes keeping a tile store to consecutive slots;
      // only the tiles some lane of the warp keeps
      for (uint32_t any = __reduce_or_sync(0xffffffffu, m); any; any &= any - 1u) {
        const int bit = __ffs(any) - 1;
        const uint32_t cb = __shfl_sync(0xffffffffu, col, bit);
        const uint32_t base = __shfl_sync(0xffffffffu, before, bit);
        if ((m >> bit) & 1u) {
          const uint32_t pos = base + __popc(cb & lt);
          if (tile_keys) tile_keys[pos] = tbase + (uint32_t)(xb + bit);
          ids[pos] = inf.id;
        }
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

__global__ void k_view_keys(const uint32_t *__restrict__ recs, const int64_t *__restrict__ d_vis, int64_t stride,
                            uint32_t *__restrict__ keys) {
  pdl_enter();
  const int64_t R = *d_vis;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < R; j += (int64_t)gridDim.x * blockDim.x)
    keys[j] = (uint32_t)(recs[j] / (uint64_t)stride);
}

struct BinWs {
  uint32_t *dk0, *dv0, *dk1, *dv1;  // depth sort ping-pong, R each
  uint32_t *vis_flags;              // ceil(R / kVisTile) look-back flags, then the ticket (cleared with `sort`)
  void *sort;                       // SortWs block: sort_ws_bytes(R), right after vis_flags
  size_t clear_bytes;               // vis_flags and sort, one memset per call
  int64_t *vis_count, *sort_count, *nchunks;
  uint32_t *rowcnt;                 // n_rows * nb_cap
  uint32_t *rowtot;                 // n_rows
  uint32_t *row_start;              // n_rows + 1
  uint32_t *chunk_start;            // n_rows + 1
  uint32_t *chunk_row;              // chunk_cap
  uint32_t *rowlist;                // row_cap
  EntryInfo *einfo;                 // row_cap
  uint32_t *tcnt, *tpre;            // chunk_cap * tx_max
  uint32_t *ttot, *tstart;          // n_rows * tx_max
  unsigned long long *rowp;         // n_rows
  int64_t nb_cap, row_cap, chunk_cap;
  size_t bytes;
};

static BinWs carve(void *base, int64_t R, int64_t cap, int n_rows, int tx_max) {
  BinWs w;
  char *p = static_cast<char *>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *q = p ? p + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1));
    return q;
  };
  R = std::max<int64_t>(R, 1);
  w.nb_cap = (R + kRecChunk - 1) / kRecChunk;
  w.row_cap = std::max<int64_t>(cap, 1);
  w.chunk_cap = (w.row_cap + kTileChunk - 1) / kTileChunk + n_rows;
  const size_t r4 = (size_t)R * 4, nr = (size_t)n_rows, txm = (size_t)tx_max;
  w.dk0 = (uint32_t *)take(r4);
  w.dv0 = (uint32_t *)take(r4);
  w.dk1 = (uint32_t *)take(r4);
  w.dv1 = (uint32_t *)take(r4);
  const size_t vis_bytes = align_up((size_t)((R + kVisTile - 1) / kVisTile + 1) * 4);
  w.vis_flags = (uint32_t *)take(vis_bytes);
  w.sort = take(sort_ws_bytes(R));
  w.clear_bytes = vis_bytes + align_up(sort_ws_bytes(R));
  w.vis_count = (int64_t *)take(8);
  w.sort_count = (int64_t *)take(8);
  w.nchunks = (int64_t *)take(8);
  w.rowcnt = (uint32_t *)take(nr * (size_t)w.nb_cap * 4);
  w.rowtot = (uint32_t *)take(nr * 4);
  w.row_start = (uint32_t *)take((nr + 1) * 4);
  w.chunk_start = (uint32_t *)take((nr + 1) * 4);
  w.chunk_row = (uint32_t *)take((size_t)w.chunk_cap * 4);
  w.rowlist = (uint32_t *)take((size_t)w.row_cap * 4);
  w.einfo = (EntryInfo *)take((size_t)w.row_cap * sizeof(EntryInfo));
  w.tcnt = (uint32_t *)take((size_t)w.chunk_cap * txm * 4);
  w.tpre = (uint32_t *)take((size_t)w.chunk_cap * txm * 4);
  w.ttot = (uint32_t *)take(nr * txm * 4);
  w.tstart = (uint32_t *)take(nr * txm * 4);
  w.rowp = (unsigned long long *)take(nr * 8);
  w.bytes = off;
  return w;
}

static bool row_geom(const DevViews &vs, int64_t stride, RowGeom *G) {
  G->n_views = vs.n;
  G->stride = stride;
  G->tx_max = 0;
  int rows = 0;
  for (int v = 0; v < vs.n; ++v) {
    G->row_base[v] = rows;
    G->tiles_x[v] = vs.cam[v].tiles_x;
    G->tile_base[v] = vs.cam[v].tile_base;
    G->tx_max = std::max(G->tx_max, vs.cam[v].tiles_x);
    rows += vs.cam[v].tiles_y;
  }
  G->row_base[vs.n] = rows;
  G->n_rows = rows;
  return rows <= kMaxRows;
}

static int bits_for(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_bin_sort_workspace_size(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                              int64_t n_records, int64_t pair_capacity) {
  if (n_records < 0 || pair_capacity < 0 || !tiling_ok(tiling)) return 0;
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return 0;
  RowGeom G;
  if (!row_geom(vs, 1, &G)) return 0;
  return carve(nullptr, n_records, pair_capacity, G.n_rows, G.tx_max).bytes;
}

extern "C" fgs_status fgs_bin_sort(const fgs_projected *proj, int64_t n, const int64_t *d_n, const fgs_camera *cams,
                                   int32_t n_views, fgs_tiling tiling, void *ws, size_t ws_bytes,
                                   uint32_t *tile_keys, int32_t *ids, int64_t pair_capacity,
                                   int32_t *tile_ranges, int64_t *d_num_pairs, int32_t *d_status,
                                   void *stream) {
  FGS_CHECK_ARG(proj && proj->splat && proj->radius && proj->rect, "fgs_bin_sort: NULL projection");
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_bin_sort: unsupported tiling");
  FGS_CHECK_ARG(n >= 0 && proj->stride >= n, "fgs_bin_sort: need 0 <= n <= stride");
  FGS_CHECK_ARG(pair_capacity >= 1 && pair_capacity <= 0x7FFFFFFFll, "fgs_bin_sort: pair_capacity");
  FGS_CHECK_ARG(ids && tile_ranges && d_num_pairs, "fgs_bin_sort: NULL output");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG((int64_t)n_views * proj->stride < 0xFFFFFFFFll, "fgs_bin_sort: too many records");
  RowGeom G;
  FGS_CHECK_ARG(row_geom(vs, proj->stride, &G), "fgs_bin_sort: more than %d tile rows", kMaxRows);
  const int64_t R = (int64_t)n_views * n;
  FGS_CHECK_ARG(R <= (int64_t)kFlagValue, "fgs_bin_sort: %lld records (n_views * n) exceed %u", (long long)R,
                kFlagValue);
  BinWs w = carve(ws, R, pair_capacity, G.n_rows, G.tx_max);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= w.bytes, "fgs_bin_sort: workspace %zu < %zu bytes", ws_bytes,
                w.bytes);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fgs_bin_sort: workspace not 256-byte aligned");
  cudaStream_t st = as_stream(stream);
  if (R == 0) {
    FGS_CUDA(cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)vs.total_tiles, st), "memset ranges");
    FGS_CUDA(cudaMemsetAsync(d_num_pairs, 0, 8, st), "memset pairs");
    return FGS_OK;
  }
  const float4 *splat = reinterpret_cast<const float4 *>(proj->splat);
  const uint2 *rect = reinterpret_cast<const uint2 *>(proj->rect);
  const int64_t nb = (R + kVisTile - 1) / kVisTile;
  // ordered compaction of the visible records, then the depth sort over them
  // (4 passes, stable: equal depths keep record order = id order within a view)
  FGS_CUDA(cudaMemsetAsync(w.vis_flags, 0, w.clear_bytes, st), "fgs_bin_sort: clear");
  const SortWs sw = sort_ws(w.sort, R);
  // the compaction also forms the depth sort's four digit histograms (sw.hist, cleared above)
  pdl_launch(k_vis_compact, (unsigned)nb, kVisThreads, 0, st, splat, proj->radius, rect, n, d_n, proj->stride, R,
             w.vis_flags, w.vis_flags + nb, w.vis_count, w.dk0, w.dv0, sw.hist, d_status);
  count_launch();
  fgs_status s = radix_sort(w.dk0, w.dv0, w.dk1, w.dv1, w.vis_count, 0, R, 32, sw, d_status, st, false, true);
  if (s != FGS_OK) return s;
  const uint32_t *srec = w.dv0;
  if (n_views > 1) {
    // views made contiguous again (stable): rows of one view stay together
    pdl_launch(k_view_keys, 4 * num_sms(), 256, 0, st, w.dv0, w.vis_count, proj->stride, w.dk0);
    count_launch();
    s = radix_sort(w.dk0, w.dv0, w.dk1, w.dv1, w.vis_count, 0, R, bits_for(n_views), sw, d_status, st);
    if (s != FGS_OK) return s;
    srec = w.dv1;  // one pass: the result is in the second buffer
  }
  const int grid = kPartGrid * num_sms();
  const int NR = G.n_rows;
  pdl_launch(k_row_count, grid, kRecChunk, 0, st, G, srec, rect, w.vis_count, w.nb_cap, w.rowcnt);
  pdl_launch(k_row_scan, NR, 1024, 0, st, w.vis_count, w.nb_cap, w.rowcnt, w.rowtot);
  pdl_launch(k_row_starts, 1, 1024, 0, st, G, w.rowtot, w.row_cap, w.row_start, w.chunk_start, w.chunk_row,
             w.chunk_cap, w.nchunks, d_status, d_num_pairs, w.sort_count);
  pdl_launch(k_row_emit, grid, kRecChunk, 0, st, G, srec, rect, w.vis_count, w.nb_cap, w.rowcnt, w.row_start,
             w.rowlist);
  count_launch(4);
  FGS_CHECK_LAUNCH("fgs_bin_sort rows");
  const int tw = tiling.tile_w, th = tiling.tile_h;
  const size_t tx_smem = sizeof(uint32_t) * (size_t)(G.tx_max + 1);
  if (tx_smem > 16384) {  // with the static arrays, past the default 48 KB of shared memory
    FGS_CUDA(cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tx_smem),
             "k_tile_count smem");
    FGS_CUDA(cudaFuncSetAttribute(k_tile_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tx_smem),
             "k_tile_emit smem");
  }
  pdl_launch(k_tile_count, grid, kTileChunk, tx_smem, st, G, splat, srec, rect, tw, th, w.rowlist, w.row_start,
             w.chunk_start, w.chunk_row, w.nchunks, w.tcnt, w.einfo);
  pdl_launch(k_tile_chunk_scan, NR, 256, 0, st, G, w.chunk_start, w.tcnt, w.tpre, w.ttot, w.rowp);
  pdl_launch(k_tile_row_starts, 1, 1024, 0, st, G, w.rowp, pair_capacity, d_num_pairs, d_status, w.sort_count);
  pdl_launch(k_tile_ranges_rows, NR, 256, 0, st, G, w.rowp, w.ttot, w.sort_count, w.tstart,
             reinterpret_cast<int2 *>(tile_ranges));
  pdl_launch(k_tile_emit, grid, kTileChunk, tx_smem, st, G, w.row_start, w.chunk_start, w.chunk_row,
             w.nchunks, w.einfo, w.tpre, w.tstart, w.sort_count, tile_keys, reinterpret_cast<uint32_t *>(ids));
  count_launch(5);
  FGS_CHECK_LAUNCH("fgs_bin_sort tiles");
  return FGS_OK;
}

extern "C" fgs_status fgs_lookback_probe(int32_t n_tiles, int32_t skip_first, int64_t timeout_ns, void *ws,
                                         size_t ws_bytes, int32_t *sums, int32_t *d_status, void *stream) {
  FGS_CHECK_ARG(n_tiles >= 1 && n_tiles <= 4096, "fgs_lookback_probe: n_tiles must be 1..4096");
  FGS_CHECK_ARG(timeout_ns >= 1000 && timeout_ns <= 5000000000ll, "fgs_lookback_probe: timeout_ns");
  FGS_CHECK_ARG(sums && d_status, "fgs_lookback_probe: NULL argument");
  const size_t need = fgs_lookback_probe_workspace_size(n_tiles);
  FGS_CHECK_ARG(ws && ws_bytes >= need && (reinterpret_cast<uintptr_t>(ws) & 255) == 0,
                "fgs_lookback_probe: workspace");
  cudaStream_t st = as_stream(stream);
  FGS_CUDA(cudaMemsetAsync(ws, 0, need, st), "fgs_lookback_probe: clear");
  uint32_t *flags = static_cast<uint32_t *>(ws);
  uint32_t *ticket = flags + (size_t)n_tiles * 256;
  k_lookback_probe<<<n_tiles, kSortThreads, 0, st>>>(flags, ticket, skip_first, timeout_ns, sums, d_status);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_lookback_probe");
  return FGS_OK;
}

extern "C" size_t fgs_lookback_probe_workspace_size(int32_t n_tiles) {
  return n_tiles < 1 ? 0 : align_up((size_t)n_tiles * 256 * 4 + 4);
}
