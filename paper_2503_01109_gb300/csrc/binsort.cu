// binsort.cu -- tile binning and depth ordering of the splats eq1 blends front to back.
//
// The required order of every tile's list is (float32 depth bits, Gaussian id).
// Instead of radix-sorting 64-bit (tile | depth) keys of every (tile, Gaussian)
// pair, the visible records are compacted in record order and sorted by depth
// ONCE (stable, so equal depths stay in id order), pairs are emitted in that
// order, and a stable sort on
// the tile index alone (a few bits, one or two 8-bit passes) finishes the job:
// within a tile the pairs keep their emission order, which is depth then id.
//
// The radix sort is LSD, 8-bit digits, reduce-then-scan: an upsweep histogram per
// block chunk, a per-digit scan of the blocks' counts, and a downsweep that
// ranks 2048-item tiles stably with per-bit warp ballots, reorders them in shared memory
// and writes each digit run coalesced.  Item counts may live on the device (the
// pair count), so the whole binning can be captured in a CUDA graph.
#include "common.cuh"

namespace fgs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048
constexpr int kSortMaxBlocks = 1024;
constexpr int kScanThreads = 1024;  // also the largest block count of a sort pass

__device__ __forceinline__ uint32_t item_count(const int64_t *d_count, int64_t host_count, int64_t cap) {
  int64_t c = d_count ? *d_count : host_count;
  if (c > cap) c = cap;
  if (c < 0) c = 0;
  return (uint32_t)c;
}

__device__ __forceinline__ void block_chunk(uint32_t count, uint32_t nb, uint32_t b, uint32_t &lo,
                                            uint32_t &hi) {
  uint32_t tiles = (count + kSortTile - 1) / kSortTile;
  uint32_t per = (tiles + nb - 1) / nb;
  uint64_t l = (uint64_t)b * per * kSortTile, h = l + (uint64_t)per * kSortTile;
  lo = (uint32_t)(l < count ? l : count);
  hi = (uint32_t)(h < count ? h : count);
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

__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                                const int64_t *d_count, int64_t host_count,
                                                                int64_t cap, int shift, int nbits,
                                                                uint32_t *__restrict__ counts) {
  __shared__ uint32_t hist[kSortThreads / 32][256];
  const int warp = threadIdx.x >> 5;
  for (int d = threadIdx.x & 31; d < 256; d += 32) hist[warp][d] = 0;
  __syncthreads();
  const uint32_t count = item_count(d_count, host_count, cap);
  uint32_t lo, hi;
  block_chunk(count, gridDim.x, blockIdx.x, lo, hi);
  const int lane = threadIdx.x & 31;
  // kSortItems keys per thread in flight, warp-striped like the downsweep
  for (uint32_t tile = lo; tile < hi; tile += kSortTile) {
    uint32_t d[kSortItems];
    bool valid[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const uint32_t i = tile + warp * (32 * kSortItems) + it * 32 + lane;
      valid[it] = i < hi;
      d[it] = valid[it] ? (keys[i] >> shift) & 255u : 0u;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const uint32_t peers = digit_peers(d[it], valid[it], nbits);
      if (valid[it] && lane == __ffs(peers) - 1) atomicAdd(&hist[warp][d[it]], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) s += hist[w][threadIdx.x];
  counts[threadIdx.x * gridDim.x + blockIdx.x] = s;  // digit-major
}

// Per-digit exclusive scan over the blocks' counts (one CTA per digit, nb <= 1024),
// in place; digit_total[d] receives the digit's item count.
__global__ void __launch_bounds__(kScanThreads) k_digit_scan(uint32_t *__restrict__ counts, int nb,
                                                             uint32_t *__restrict__ digit_total) {
  __shared__ uint32_t warp_sum[kScanThreads / 32];
  const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *row = counts + (size_t)d * nb;
  const uint32_t c = threadIdx.x < nb ? row[threadIdx.x] : 0u;
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = warp_sum[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_sum[lane] = wi - w;
    if (lane == 31) digit_total[d] = wi;
  }
  __syncthreads();
  if (threadIdx.x < nb) row[threadIdx.x] = warp_sum[warp] + incl - c;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_downsweep(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const int64_t *d_count,
    int64_t host_count, int64_t cap, int shift, int nbits, const uint32_t *__restrict__ offsets,
    const uint32_t *__restrict__ digit_total) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t s_whist[W][256];  // per warp and digit: count, then the warp's offset in the tile's run
  __shared__ uint32_t s_base[256];      // output position of this block's next item of each digit
  __shared__ uint32_t s_prefix[256];    // start of each digit's run in the reordered tile
  __shared__ uint32_t s_warp[W];
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t count = item_count(d_count, host_count, cap);
  uint32_t lo, hi;
  block_chunk(count, gridDim.x, blockIdx.x, lo, hi);
  // start of each digit in the output, plus this block's offset inside the digit
  {
    uint32_t all;
    const uint32_t start = block_scan256(digit_total[threadIdx.x], s_warp, all);
    s_base[threadIdx.x] = start + offsets[threadIdx.x * gridDim.x + blockIdx.x];
  }
  __syncthreads();
  for (uint32_t tile = lo; tile < hi; tile += kSortTile) {
    for (int d = lane; d < 256; d += 32) s_whist[warp][d] = 0;
    __syncwarp();
    uint32_t k[kSortItems], v[kSortItems], local[kSortItems], dig[kSortItems];
    bool valid[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const uint32_t idx = tile + warp * (32 * kSortItems) + it * 32 + lane;
      valid[it] = idx < hi;
      k[it] = valid[it] ? keys_in[idx] : 0u;
      v[it] = valid[it] ? vals_in[idx] : 0u;
      dig[it] = (k[it] >> shift) & 255u;
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
    uint32_t run = 0;  // this thread's digit: items in the tile
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = s_whist[w][threadIdx.x];
      s_whist[w][threadIdx.x] = run;
      run += c;
    }
    uint32_t tile_items;
    s_prefix[threadIdx.x] = block_scan256(run, s_warp, tile_items);
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
      const uint32_t d = (key >> shift) & 255u;
      const uint32_t out = s_base[d] + (i - s_prefix[d]);
      keys_out[out] = key;
      vals_out[out] = s_vals[i];
    }
    __syncthreads();
    s_base[threadIdx.x] += run;
    __syncthreads();
  }
}

// Stable LSD sort of (key, value) over bits [0, bits).  Result lands in (k0, v0)
// when the number of passes is even, in (k1, v1) otherwise.
static fgs_status radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const int64_t *d_count,
                             int64_t host_count, int64_t cap, int bits, int nblocks, uint32_t *counts,
                             uint32_t *digit_total, cudaStream_t st) {
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const int nbits = std::min(8, bits - shift);
    uint32_t *ki = (p & 1) ? k1 : k0, *vi = (p & 1) ? v1 : v0;
    uint32_t *ko = (p & 1) ? k0 : k1, *vo = (p & 1) ? v0 : v1;
    k_radix_upsweep<<<nblocks, kSortThreads, 0, st>>>(ki, d_count, host_count, cap, shift, nbits, counts);
    k_digit_scan<<<256, kScanThreads, 0, st>>>(counts, nblocks, digit_total);
    k_radix_downsweep<<<nblocks, kSortThreads, 0, st>>>(ki, vi, ko, vo, d_count, host_count, cap, shift,
                                                        nbits, counts, digit_total);
    count_launch(3);
  }
  FGS_CHECK_LAUNCH("radix_sort");
  return FGS_OK;
}

static int sort_blocks(int64_t cap) {
  int64_t tiles = (cap + kSortTile - 1) / kSortTile;
  int64_t nb = std::min<int64_t>(std::min<int64_t>(tiles, kSortMaxBlocks), 4 * (int64_t)num_sms());
  return (int)std::max<int64_t>(nb, 1);
}

// ---------------------------------------------------------------------------------
// Visible records (radius > 0 and at least one tile) are compacted in record
// order before the depth sort, so the sort touches only them: a block count, a
// scan of the block counts, and an ordered scatter of (depth bits, record).

constexpr int kScanBlock = 1024;

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

__global__ void __launch_bounds__(kScanBlock) k_vis_count(const int32_t *__restrict__ radius,
                                                          const uint2 *__restrict__ rect, int64_t n, int64_t stride,
                                                          int64_t R, uint32_t *__restrict__ bsum) {
  __shared__ uint32_t red[kScanBlock / 32];
  const int64_t j = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const bool vis = j < R && record_visible(radius, rect, record_of(j, n, stride));
  const uint32_t b = __ballot_sync(0xffffffffu, vis);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of nb block counts in place by one CTA; *total = their sum.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t *__restrict__ bsum, int nb, int64_t *total) {
  __shared__ unsigned long long part[1024];
  const int per = (nb + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += bsum[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    const uint32_t v = bsum[i];
    bsum[i] = (uint32_t)run;
    run += v;
  }
  if (threadIdx.x == 1023) *total = (int64_t)part[1023];
}

__global__ void __launch_bounds__(kScanBlock) k_vis_scatter(const float4 *__restrict__ splat,
                                                            const int32_t *__restrict__ radius,
                                                            const uint2 *__restrict__ rect, int64_t n, int64_t stride,
                                                            int64_t R, const uint32_t *__restrict__ bsum,
                                                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  __shared__ uint32_t wsum[kScanBlock / 32];
  const int64_t j = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r = j < R ? record_of(j, n, stride) : 0;
  const bool vis = j < R && record_visible(radius, rect, r);
  const uint32_t b = __ballot_sync(0xffffffffu, vis);
  if (lane == 0) wsum[warp] = __popc(b);
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = wsum[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    wsum[lane] = wi - w;
  }
  __syncthreads();
  if (!vis) return;
  const uint32_t pos = bsum[blockIdx.x] + wsum[warp] + __popc(b & ((1u << lane) - 1u));
  keys[pos] = __float_as_uint(splat[2 * r + 1].z);  // depth > 0: its bits order like the value
  vals[pos] = (uint32_t)r;
}


// A visible record prepared by its own lane (box and support), so that a warp
// walking its 32 records one after the other only broadcasts them.
struct PreparedRecord {
  uint32_t rec, x0, y0, x1, y1;
  SupportSplat sp;
};

__device__ __forceinline__ PreparedRecord prepare_record(const float4 *__restrict__ splat,
                                                         const uint2 *__restrict__ rect, uint32_t rec, bool valid) {
  PreparedRecord p{};
  if (!valid) {
    p.x0 = 1;  // empty box
    return p;
  }
  const uint2 rc = rect[rec];
  p.rec = rec;
  p.x0 = rc.x & 0xFFFFu;
  p.y0 = rc.x >> 16;
  p.x1 = rc.y & 0xFFFFu;
  p.y1 = rc.y >> 16;
  p.sp = support_splat(splat[2 * (int64_t)rec], splat[2 * (int64_t)rec + 1]);
  return p;
}

__device__ __forceinline__ PreparedRecord shfl_record(const PreparedRecord &p, int src) {
  PreparedRecord q;
  q.rec = __shfl_sync(0xffffffffu, p.rec, src);
  q.x0 = __shfl_sync(0xffffffffu, p.x0, src);
  q.y0 = __shfl_sync(0xffffffffu, p.y0, src);
  q.x1 = __shfl_sync(0xffffffffu, p.x1, src);
  q.y1 = __shfl_sync(0xffffffffu, p.y1, src);
  q.sp.mx = __shfl_sync(0xffffffffu, p.sp.mx, src);
  q.sp.my = __shfl_sync(0xffffffffu, p.sp.my, src);
  q.sp.a = __shfl_sync(0xffffffffu, p.sp.a, src);
  q.sp.b = __shfl_sync(0xffffffffu, p.sp.b, src);
  q.sp.c = __shfl_sync(0xffffffffu, p.sp.c, src);
  q.sp.thr = __shfl_sync(0xffffffffu, p.sp.thr, src);
  q.sp.sx = __shfl_sync(0xffffffffu, p.sp.sx, src);
  q.sp.sy = __shfl_sync(0xffffffffu, p.sp.sy, src);
  return q;
}

// Tiles per sorted visible record (those of its box that its opacity-aware
// ellipse reaches), then per-block sums for the scan.  A warp counts its 32
// records one after the other, its lanes testing 32 of the record's tiles at a
// time, so large footprints do not serialise one thread.
__global__ void __launch_bounds__(kScanBlock) k_counts_blocksum(const float4 *__restrict__ splat,
                                                                const uint32_t *__restrict__ svals,
                                                                const uint2 *__restrict__ rect,
                                                                const int64_t *__restrict__ d_vis, int tw, int th,
                                                                uint32_t *__restrict__ cnt,
                                                                uint32_t *__restrict__ bsum) {
  __shared__ uint32_t red[kScanBlock / 32];
  const int64_t j = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int64_t R = *d_vis;
  const int lane = threadIdx.x & 31;
  const PreparedRecord mine = prepare_record(splat, rect, j < R ? svals[j] : 0u, j < R);
  uint32_t c = 0;
  uint32_t pending = __ballot_sync(0xffffffffu, j < R && mine.x0 <= mine.x1 && mine.y0 <= mine.y1);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const PreparedRecord pr = shfl_record(mine, src);
    const uint32_t x0 = pr.x0, y0 = pr.y0, x1 = pr.x1, y1 = pr.y1;
    const SupportSplat &sp = pr.sp;
    uint32_t n = 0;
    {
      const uint32_t w = x1 - x0 + 1u, box = w * (y1 - y0 + 1u);
      for (uint32_t q0 = 0; q0 < box; q0 += 32) {
        const uint32_t q = q0 + lane;
        bool keep = false;
        if (q < box) {
          const uint32_t dy = q / w, dx = q - dy * w;
          keep = tile_in_support(sp, (int)(x0 + dx), (int)(y0 + dy), tw, th);
        }
        n += __popc(__ballot_sync(0xffffffffu, keep));
      }
    }
    if (lane == src) c = n;
  }
  if (j < R) cnt[j] = c;
  uint32_t s = c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of the block sums with 64-bit total; the total is the pair count.
__global__ void __launch_bounds__(kScanThreads) k_scan_bsum(uint32_t *__restrict__ bsum, int nb,
                                                            int64_t *__restrict__ d_num_pairs,
                                                            int64_t pair_cap, int32_t *__restrict__ d_status,
                                                            int64_t *__restrict__ d_sort_count) {
  __shared__ unsigned long long part[kScanThreads];
  const int per = (nb + kScanThreads - 1) / kScanThreads;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += bsum[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    uint32_t v = bsum[i];
    bsum[i] = (uint32_t)(run > 0xFFFFFFFFull ? 0xFFFFFFFFull : run);
    run += v;
  }
  if (threadIdx.x == kScanThreads - 1) {
    const unsigned long long total = part[kScanThreads - 1];
    *d_num_pairs = (int64_t)total;
    const bool over = total > (unsigned long long)pair_cap;
    if (over && d_status) atomicOr(d_status, FGS_DEV_PAIR_OVERFLOW);
    *d_sort_count = over ? 0 : (int64_t)total;
  }
}

// Emits the (tile, id) pairs of every sorted record at its scanned offset.  A
// warp cooperates on one record at a time so that large footprints do not
// serialise a single thread.
__global__ void __launch_bounds__(kScanBlock) k_emit(const float4 *__restrict__ splat, int tw, int th,
                                                     const uint32_t *__restrict__ svals,
                                                     const uint2 *__restrict__ rect,
                                                     const uint32_t *__restrict__ cnt,
                                                     const uint32_t *__restrict__ bsum,
                                                     const int64_t *__restrict__ d_vis, int64_t stride, DevViews vs,
                                                     const int64_t *d_sort_count, uint32_t *__restrict__ tile_keys,
                                                     uint32_t *__restrict__ ids) {
  __shared__ uint32_t warp_sum[kScanBlock / 32];
  const int64_t j = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int64_t R = *d_vis;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c = j < R ? cnt[j] : 0u;
  // block-local exclusive scan of c
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kScanBlock / 32 ? warp_sum[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanBlock / 32) warp_sum[lane] = wi - w;
  }
  __syncthreads();
  const uint32_t off = bsum[blockIdx.x] + warp_sum[warp] + (incl - c);
  const int64_t sort_count = *d_sort_count;  // 0 on overflow: emit nothing
  // warp-cooperative emission: each lane's record in turn
  const bool has = c > 0 && sort_count > 0;
  const PreparedRecord mine = prepare_record(splat, rect, has ? svals[j] : 0u, has);
  uint32_t pending = __ballot_sync(0xffffffffu, has);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const uint32_t rc_off = __shfl_sync(0xffffffffu, off, src);
    const uint32_t rc_cnt = __shfl_sync(0xffffffffu, c, src);
    const PreparedRecord pr = shfl_record(mine, src);
    const uint32_t rec = pr.rec;
    const uint32_t v = (uint32_t)(rec / stride), id = (uint32_t)(rec - (uint64_t)v * stride);
    const uint32_t x0 = pr.x0, y0 = pr.y0, x1 = pr.x1;
    const uint32_t w = x1 - x0 + 1u, box = w * (pr.y1 - y0 + 1u);
    const uint32_t tb = (uint32_t)vs.cam[v].tile_base, tx = (uint32_t)vs.cam[v].tiles_x;
    const SupportSplat &sp = pr.sp;
    // the box's tiles in row-major order, 32 candidates per step; the ones the
    // ellipse reaches are written at consecutive positions (rc_cnt in total)
    uint32_t out = rc_off;
    for (uint32_t q0 = 0; q0 < box; q0 += 32) {
      const uint32_t q = q0 + lane;
      bool keep = false;
      uint32_t t = 0;
      if (q < box) {
        const uint32_t dy = q / w, dx = q - dy * w;
        keep = tile_in_support(sp, (int)(x0 + dx), (int)(y0 + dy), tw, th);
        t = tb + (y0 + dy) * tx + (x0 + dx);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const uint32_t pos = out + __popc(m & ((1u << lane) - 1u));
        tile_keys[pos] = t;
        ids[pos] = id;
      }
      out += __popc(m);
    }
    (void)rc_cnt;
  }
}

__global__ void k_tile_ranges(const uint32_t *__restrict__ tile_keys, const int64_t *d_sort_count,
                              int64_t cap, int2 *__restrict__ ranges) {
  const int64_t P = min(*d_sort_count, cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += stride) {
    const uint32_t t = tile_keys[k];
    const uint32_t prev = k > 0 ? tile_keys[k - 1] : 0xFFFFFFFFu;
    const uint32_t next = k + 1 < P ? tile_keys[k + 1] : 0xFFFFFFFFu;
    if (prev != t) ranges[t].x = (int)k;
    if (next != t) ranges[t].y = (int)(k + 1);
  }
}

struct BinWs {
  uint32_t *dk0, *dv0, *dk1, *dv1;  // depth sort ping-pong, R each
  uint32_t *cnt;                    // R
  uint32_t *bsum;                   // ceil(R / 1024)
  uint32_t *tk1, *tv1;              // tile sort ping-pong, pair_capacity each
  uint32_t *counts;                 // 256 * kSortMaxBlocks
  uint32_t *digit_total;            // 256
  int64_t *sort_count;              // 1
  int64_t *vis_count;               // 1
  size_t bytes;
};

static BinWs carve(void *base, int64_t R, int64_t cap) {
  BinWs w;
  char *p = static_cast<char *>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *q = p ? p + off : nullptr;
    off += align_up(bytes);
    return q;
  };
  const size_t r4 = (size_t)std::max<int64_t>(R, 1) * 4, c4 = (size_t)std::max<int64_t>(cap, 1) * 4;
  w.dk0 = (uint32_t *)take(r4);
  w.dv0 = (uint32_t *)take(r4);
  w.dk1 = (uint32_t *)take(r4);
  w.dv1 = (uint32_t *)take(r4);
  w.cnt = (uint32_t *)take(r4);
  w.bsum = (uint32_t *)take((size_t)((R + kScanBlock - 1) / kScanBlock + 1) * 4);
  w.tk1 = (uint32_t *)take(c4);
  w.tv1 = (uint32_t *)take(c4);
  w.counts = (uint32_t *)take((size_t)256 * kSortMaxBlocks * 4);
  w.digit_total = (uint32_t *)take(256 * 4);
  w.sort_count = (int64_t *)take(8);
  w.vis_count = (int64_t *)take(8);
  w.bytes = off;
  return w;
}

static int bits_for(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_bin_sort_workspace_size(int64_t n_records, int64_t pair_capacity) {
  if (n_records < 0 || pair_capacity < 0) return 0;
  return carve(nullptr, n_records, pair_capacity).bytes;
}

extern "C" fgs_status fgs_bin_sort(const fgs_projected *proj, int64_t n, const fgs_camera *cams,
                                   int32_t n_views, fgs_tiling tiling, void *ws, size_t ws_bytes,
                                   uint32_t *tile_keys, int32_t *ids, int64_t pair_capacity,
                                   int32_t *tile_ranges, int64_t *d_num_pairs, int32_t *d_status,
                                   void *stream) {
  FGS_CHECK_ARG(proj && proj->splat && proj->radius && proj->rect, "fgs_bin_sort: NULL projection");
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_bin_sort: unsupported tiling");
  FGS_CHECK_ARG(n >= 0 && proj->stride >= n, "fgs_bin_sort: need 0 <= n <= stride");
  FGS_CHECK_ARG(pair_capacity >= 1 && pair_capacity <= 0x7FFFFFFFll, "fgs_bin_sort: pair_capacity");
  FGS_CHECK_ARG(tile_keys && ids && tile_ranges && d_num_pairs, "fgs_bin_sort: NULL output");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG((int64_t)n_views * proj->stride < 0xFFFFFFFFll, "fgs_bin_sort: too many records");
  const int64_t R = (int64_t)n_views * n;
  BinWs w = carve(ws, R, pair_capacity);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= w.bytes, "fgs_bin_sort: workspace %zu < %zu bytes", ws_bytes,
                w.bytes);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fgs_bin_sort: workspace not 256-byte aligned");
  cudaStream_t st = as_stream(stream);
  FGS_CUDA(cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)vs.total_tiles, st), "memset ranges");
  if (R == 0) {
    FGS_CUDA(cudaMemsetAsync(d_num_pairs, 0, 8, st), "memset pairs");
    return FGS_OK;
  }
  const float4 *splat = reinterpret_cast<const float4 *>(proj->splat);
  const uint2 *rect = reinterpret_cast<const uint2 *>(proj->rect);
  const int64_t nb = (R + kScanBlock - 1) / kScanBlock;
  // ordered compaction of the visible records, then the depth sort over them
  // (4 passes, stable: equal depths keep record order = id order within a view)
  k_vis_count<<<(unsigned)nb, kScanBlock, 0, st>>>(proj->radius, rect, n, proj->stride, R, w.bsum);
  k_scan_blocks<<<1, 1024, 0, st>>>(w.bsum, (int)nb, w.vis_count);
  k_vis_scatter<<<(unsigned)nb, kScanBlock, 0, st>>>(splat, proj->radius, rect, n, proj->stride, R, w.bsum, w.dk0,
                                                     w.dv0);
  count_launch(3);
  fgs_status s = radix_sort(w.dk0, w.dv0, w.dk1, w.dv1, w.vis_count, 0, R, 32, sort_blocks(R), w.counts,
                            w.digit_total, st);
  if (s != FGS_OK) return s;
  k_counts_blocksum<<<(unsigned)nb, kScanBlock, 0, st>>>(splat, w.dv0, rect, w.vis_count, tiling.tile_w,
                                                         tiling.tile_h, w.cnt, w.bsum);
  k_scan_bsum<<<1, kScanThreads, 0, st>>>(w.bsum, (int)nb, d_num_pairs, pair_capacity, d_status, w.sort_count);
  // emit into the buffer the tile sort ends in the caller's arrays
  const int tbits = std::max(1, bits_for(vs.total_tiles));
  const int passes = (tbits + 7) / 8;
  uint32_t *ek = (passes & 1) ? w.tk1 : tile_keys;
  uint32_t *ev = (passes & 1) ? w.tv1 : reinterpret_cast<uint32_t *>(ids);
  k_emit<<<(unsigned)nb, kScanBlock, 0, st>>>(splat, tiling.tile_w, tiling.tile_h, w.dv0, rect, w.cnt, w.bsum,
                                              w.vis_count, proj->stride, vs, w.sort_count, ek, ev);
  count_launch(3);
  FGS_CHECK_LAUNCH("fgs_bin_sort emit");
  s = radix_sort(ek, ev, (passes & 1) ? tile_keys : w.tk1, (passes & 1) ? reinterpret_cast<uint32_t *>(ids) : w.tv1,
                 w.sort_count, 0, pair_capacity, tbits, sort_blocks(pair_capacity), w.counts, w.digit_total, st);
  if (s != FGS_OK) return s;
  k_tile_ranges<<<32 * num_sms(), 256, 0, st>>>(tile_keys, w.sort_count, pair_capacity,
                                               reinterpret_cast<int2 *>(tile_ranges));
  count_launch();
  FGS_CHECK_LAUNCH("fgs_bin_sort ranges");
  return FGS_OK;
}
