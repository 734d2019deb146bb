// tile_order.cu -- the order in which the render kernels take their tiles:
// heaviest first.
//
// The blend (eq1) and its adjoint run one CTA per tile, and the tiles' work
// differs several-fold: a tile's walk over its sorted list ends at the largest
// contributor count of its pixels (n_contrib).  A launch holds about 2-3 waves
// of CTAs, so a heavy tile dispatched late keeps its SM busy while the others
// run dry.  Dispatching the tiles in decreasing order of work (longest
// processing time first) fills that tail.  The render calls take the
// permutation as `tile_order`; fgs_tile_order computes it from a render's
// n_contrib:
//
//   k_tile_cost   one CTA per tile: the largest n_contrib of its pixels, capped
//                 at kOrderKeys - 1
//   k_tile_order  one CTA: counting sort of the tiles by that key, descending;
//                 tiles of equal key come in no fixed order
//
// The order decides only which CTA renders which tile, never what a tile
// computes, so any permutation gives the same render.
#include "common.cuh"

namespace fgs {

constexpr int kOrderKeys = 4096;  // distinct sort keys (contributor counts 0 .. 4095+)
constexpr int kOrderThreads = 1024;

__global__ void __launch_bounds__(256) k_tile_cost(DevViews vs, int tw, int th, const int32_t *__restrict__ n_contrib,
                                                   int32_t *__restrict__ cost) {
  pdl_enter();
  __shared__ int s_max[8];
  const int t = blockIdx.x;
  const int v = view_of_tile(vs, t);
  const DevCam &cm = vs.cam[v];
  const int lt = t - cm.tile_base;
  const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
  int m = 0;
  for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
    const int x = tx * tw + i % tw, y = ty * th + i / tw;
    if (x < cm.W && y < cm.H) m = max(m, n_contrib[cm.pix_base + (int64_t)y * cm.W + x]);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, s_max[w]);
    cost[t] = min(max(r, 0), kOrderKeys - 1);
  }
}

__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const int32_t *__restrict__ cost, int n,
                                                              int32_t *__restrict__ order) {
  pdl_enter();
  constexpr int KPT = kOrderKeys / kOrderThreads;  // keys per thread
  __shared__ int s_pos[kOrderKeys];
  __shared__ int s_warp[kOrderThreads / 32];
  for (int k = threadIdx.x; k < kOrderKeys; k += kOrderThreads) s_pos[k] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += kOrderThreads) atomicAdd(&s_pos[cost[t]], 1);
  __syncthreads();
  // Exclusive prefix sum of the counts in descending key order: thread i owns
  // the keys kOrderKeys - 1 - (KPT i + u), u = 0 .. KPT - 1, and reads and
  // writes only those.
  int c[KPT], sum = 0;
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    c[u] = s_pos[kOrderKeys - 1 - (KPT * (int)threadIdx.x + u)];
    sum += c[u];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = s_warp[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    s_warp[lane] = wi - w;
  }
  __syncthreads();
  int run = s_warp[warp] + incl - sum;
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    s_pos[kOrderKeys - 1 - (KPT * (int)threadIdx.x + u)] = run;
    run += c[u];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += kOrderThreads) order[atomicAdd(&s_pos[cost[t]], 1)] = t;
}

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_tile_order_workspace_size(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling) {
  DevViews vs;
  if (!tiling_ok(tiling) || !make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return 0;
  return ((size_t)vs.total_tiles * sizeof(int32_t) + 255) / 256 * 256;
}

extern "C" fgs_status fgs_tile_order(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                     const int32_t *n_contrib, int32_t *tile_order, void *ws, size_t ws_bytes,
                                     void *stream) {
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_tile_order: unsupported tiling");
  FGS_CHECK_ARG(n_contrib && tile_order && ws, "fgs_tile_order: NULL argument");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(vs.total_tiles > 0, "fgs_tile_order: no tiles");
  FGS_CHECK_ARG(ws_bytes >= (size_t)vs.total_tiles * sizeof(int32_t), "fgs_tile_order: workspace of %zu bytes < %zu",
                ws_bytes, (size_t)vs.total_tiles * sizeof(int32_t));
  cudaStream_t st = as_stream(stream);
  int32_t *cost = static_cast<int32_t *>(ws);
  pdl_launch(k_tile_cost, vs.total_tiles, 256, 0, st, vs, (int)tiling.tile_w, (int)tiling.tile_h, n_contrib, cost);
  pdl_launch(k_tile_order, 1, kOrderThreads, 0, st, (const int32_t *)cost, vs.total_tiles, tile_order);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_tile_order");
  return FGS_OK;
}
