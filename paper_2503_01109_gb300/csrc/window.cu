// window.cu -- a keyframe window (the co-visible and random keyframes the map is
// optimised over, Sec. III-C/D) rendered forward, scored with eq16 and
// differentiated in ONE persistent launch.
//
// The CTAs of a cooperative grid (all resident at once) pull work items from
// atomic counters in three phases separated by grid barriers:
//   1. eq1 forward of every (view, tile) of every view, whatever its resolution;
//   2. the fused L1 + SSIM loss tiles of every view (they read neighbouring
//      tiles' pixels, hence the barrier);
//   3. the adjoint of every (view, tile).
// Work is claimed dynamically, so mixed resolutions and uneven tiles balance
// across the SMs.  Every barrier wait is bounded in time: a CTA that waits more
// than FGS_WINDOW_TIMEOUT_NS sets FGS_DEV_TIMEOUT in the status word and returns
// (the outputs of that launch are then invalid), so a broken launch cannot hang.
#include "loss_tile.cuh"
#include "render_tile.cuh"

namespace fgs {

constexpr int64_t kBarrierTimeoutNs = 2000000000ll;  // 2 s

struct WindowArgs {
  RenderArgs f;
  RenderBwdArgs b;
  LossArgs l;
  int n_tiles, n_loss_tiles;
  uint32_t *ctl;  // [0..2] work counters of the phases, [3] barrier arrivals, [4] barrier generation
  int32_t *status;
  uint32_t nblocks;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait over the counters ctl[3] (arrivals) and
// ctl[4] (generation) for a grid of nblocks CTAs.  Returns false (for every thread
// of the CTA) when the wait gave up after timeout_ns; FGS_DEV_TIMEOUT is then set.
__device__ __forceinline__ bool grid_barrier_bounded(uint32_t *ctl, int32_t *status, uint32_t nblocks,
                                                     int64_t timeout_ns, int *s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t *gen = ctl + 4;
    const uint32_t g = *gen;
    __threadfence();
    const uint32_t arrived = atomicAdd(ctl + 3, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      ctl[3] = 0;
      __threadfence();
      atomicAdd(ctl + 4, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*gen == g) {
        if (global_ns() - t0 > (uint64_t)timeout_ns) {
          ok = 0;
          atomicOr(status, FGS_DEV_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

__device__ __forceinline__ bool grid_barrier(const WindowArgs &w, int *s_flag) {
  return grid_barrier_bounded(w.ctl, w.status, w.nblocks, kBarrierTimeoutNs, s_flag);
}

// The barrier alone, for its self-test: every CTA arrives once at a barrier that
// expects `expected` arrivals; the CTAs that got through count themselves.
__global__ void k_barrier_probe(uint32_t *ctl, int32_t *status, uint32_t expected, int64_t timeout_ns,
                                uint32_t *passed) {
  __shared__ int s_flag;
  if (grid_barrier_bounded(ctl, status, expected, timeout_ns, &s_flag) && threadIdx.x == 0) atomicAdd(passed, 1u);
}

__device__ __forceinline__ int claim(uint32_t *counter, int *s_item) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return *s_item;
}

// Loss tile side inside the window: 16, so that the loss phase's shared memory
// (38 KB) stays below the render phases' and does not lower the grid's residency.
constexpr int kWinLT = 16;

// Tile of render work item i: i itself, or its entry of the launch order
// (fgs_tile_order: heaviest first); an entry outside the tiles is reported and
// skipped.
__device__ __forceinline__ int window_tile(const WindowArgs &w, int i) {
  if (!w.f.order) return i;
  const int t = w.f.order[i];
  if ((unsigned)t < (unsigned)w.n_tiles) return t;
  if (threadIdx.x == 0) atomicOr(w.status, FGS_DEV_BAD_ORDER);
  return -1;
}

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW *TH / 2) k_window(WindowArgs w) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int s_item, s_flag;
  for (;;) {
    const int i = claim(w.ctl + 0, &s_item);
    if (i >= w.n_tiles) break;
    const int t = window_tile(w, i);
    if (t >= 0) render_fwd_tile<TW, TH, BATCH, 2>(w.f, t, smem);
  }
  if (!grid_barrier(w, &s_flag)) return;
  for (;;) {
    const int t = claim(w.ctl + 1, &s_item);
    if (t >= w.n_loss_tiles) break;
    loss_tile<kWinLT>(w.l, t, reinterpret_cast<float *>(smem));
  }
  if (!grid_barrier(w, &s_flag)) return;
  for (;;) {
    const int i = claim(w.ctl + 2, &s_item);
    if (i >= w.n_tiles) break;
    const int t = window_tile(w, i);
    if (t >= 0) render_bwd_tile<TW, TH, BATCH, 2>(w.b, t, smem);
  }
}

__global__ void k_window_reduce(const double *__restrict__ partials, int64_t count, float *d_loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += 256) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *d_loss += (float)red[0];
}

template <int TW, int TH, int BATCH>
static size_t window_smem() {
  size_t s = std::max<size_t>(TileSmem<BATCH>::fwd, TileSmem<BATCH>::bwd);
  return std::max<size_t>(s, sizeof(float) * LossGeom<kWinLT>::SmemFloats);
}

template <int TW, int TH, int BATCH>
static fgs_status launch_window(WindowArgs &w, cudaStream_t st, int *grid_out) {
  const int threads = TW * TH / 2;
  const size_t smem = window_smem<TW, TH, BATCH>();
  int per_sm = 0;
  FGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_window<TW, TH, BATCH>, threads, smem),
           "window occupancy");
  if (per_sm < 1) {
    set_error("fgs_render_window: kernel does not fit on an SM");
    return FGS_ERR_UNSUPPORTED;
  }
  const int grid = per_sm * num_sms();
  w.nblocks = (uint32_t)grid;
  void *args[] = {&w};
  FGS_CUDA(cudaLaunchCooperativeKernel((const void *)k_window<TW, TH, BATCH>, dim3(grid), dim3(threads), args, smem,
                                       st),
           "fgs_render_window launch");
  if (grid_out) *grid_out = grid;
  return FGS_OK;
}

#define FGS_WINDOW_DISPATCH(tiling, ...)                                                     \
  (((tiling).tile_w == 16 && (tiling).tile_h == 16)                                          \
       ? ((tiling).batch_depth == 32    ? launch_window<16, 16, 32>(__VA_ARGS__)             \
          : (tiling).batch_depth == 64  ? launch_window<16, 16, 64>(__VA_ARGS__)             \
          : (tiling).batch_depth == 128 ? launch_window<16, 16, 128>(__VA_ARGS__)            \
                                        : launch_window<16, 16, 256>(__VA_ARGS__))           \
   : ((tiling).tile_w == 8)                                                                  \
       ? ((tiling).batch_depth == 32    ? launch_window<8, 8, 32>(__VA_ARGS__)               \
          : (tiling).batch_depth == 64  ? launch_window<8, 8, 64>(__VA_ARGS__)               \
          : (tiling).batch_depth == 128 ? launch_window<8, 8, 128>(__VA_ARGS__)              \
                                        : launch_window<8, 8, 256>(__VA_ARGS__))             \
       : ((tiling).batch_depth == 32    ? launch_window<16, 32, 32>(__VA_ARGS__)             \
          : (tiling).batch_depth == 64  ? launch_window<16, 32, 64>(__VA_ARGS__)             \
          : (tiling).batch_depth == 128 ? launch_window<16, 32, 128>(__VA_ARGS__)            \
                                        : launch_window<16, 32, 256>(__VA_ARGS__)))

static bool window_loss_views(const fgs_camera *cams, int32_t n_views, LossViews *lv, int *tiles) {
  lv->n = n_views;
  int t = 0;
  int64_t pix = 0;
  for (int v = 0; v < n_views; ++v) {
    lv->v[v].W = cams[v].width;
    lv->v[v].H = cams[v].height;
    lv->v[v].tiles_x = (cams[v].width + kWinLT - 1) / kWinLT;
    lv->v[v].tile_base = t;
    lv->v[v].pix_base = pix;
    t += lv->v[v].tiles_x * ((cams[v].height + kWinLT - 1) / kWinLT);
    pix += (int64_t)cams[v].width * cams[v].height;
  }
  *tiles = t;
  return true;
}

}  // namespace fgs

using namespace fgs;

extern "C" fgs_status fgs_grid_barrier_probe(int32_t n_blocks, int32_t n_expected, int64_t timeout_ns,
                                             void *ws, size_t ws_bytes, uint32_t *d_passed, int32_t *d_status,
                                             void *stream) {
  FGS_CHECK_ARG(n_blocks >= 1 && n_blocks <= num_sms() && n_expected >= n_blocks,
                "fgs_grid_barrier_probe: need 1 <= n_blocks <= SM count and n_expected >= n_blocks");
  FGS_CHECK_ARG(timeout_ns >= 1000 && timeout_ns <= 5000000000ll, "fgs_grid_barrier_probe: timeout_ns");
  FGS_CHECK_ARG(ws && ws_bytes >= 8 * sizeof(uint32_t) && d_passed && d_status, "fgs_grid_barrier_probe: NULL");
  cudaStream_t st = as_stream(stream);
  FGS_CUDA(cudaMemsetAsync(ws, 0, 8 * sizeof(uint32_t), st), "fgs_grid_barrier_probe memset");
  uint32_t *ctl = static_cast<uint32_t *>(ws);
  uint32_t expected = (uint32_t)n_expected;
  void *args[] = {&ctl, &d_status, &expected, &timeout_ns, &d_passed};
  FGS_CUDA(cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(n_blocks), dim3(32), args, 0, st),
           "fgs_grid_barrier_probe launch");
  count_launch();
  return FGS_OK;
}

extern "C" size_t fgs_render_window_workspace_size(const fgs_camera *cams, int32_t n_views) {
  if (!cams || n_views < 1 || n_views > FGS_MAX_VIEWS) return 0;
  LossViews lv;
  int tiles = 0;
  window_loss_views(cams, n_views, &lv, &tiles);
  return align_up(sizeof(double) * (size_t)tiles) + align_up(8 * sizeof(uint32_t));
}

extern "C" fgs_status fgs_render_window(const fgs_gaussians *g, const fgs_projected *proj,
                                        const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                        const int32_t *ids, const int32_t *tile_ranges,
                                        const int32_t *tile_order, const float *color_gt,
                                        const float *depth_gt, const fgs_loss_params *lp, float *color,
                                        float *depth, float *alpha, float *t_final, int32_t *n_contrib,
                                        float *dL_dcolor, float *dL_ddepth, float *grad2d, fgs_gaussians *grads,
                                        float *d_loss, void *ws, size_t ws_bytes, int32_t *d_status,
                                        void *stream) {
  if (!gaussians_ok(g, "g") || !gaussians_ok(grads, "grads")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(proj && proj->splat && proj->stride >= g->n, "fgs_render_window: projection");
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_render_window: unsupported tiling");
  FGS_CHECK_ARG(ids && tile_ranges && color_gt && depth_gt && lp && color && depth && alpha && t_final &&
                    n_contrib && dL_dcolor && dL_ddepth && grad2d && d_loss && d_status,
                "fgs_render_window: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(grad2d) & 15) == 0 && (reinterpret_cast<uintptr_t>(ws) & 255) == 0,
                "fgs_render_window: alignment");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  const size_t need = fgs_render_window_workspace_size(cams, n_views);
  FGS_CHECK_ARG(ws && ws_bytes >= need, "fgs_render_window: workspace %zu < %zu bytes", ws_bytes, need);
  WindowArgs w;
  w.f = RenderArgs{vs, reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity, ids,
                   reinterpret_cast<const int2 *>(tile_ranges), color, depth, alpha, t_final, n_contrib,
                   tile_order, d_status};
  w.b = RenderBwdArgs{vs,        reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity,
                      ids,       reinterpret_cast<const int2 *>(tile_ranges), t_final, n_contrib, dL_dcolor,
                      dL_ddepth, nullptr, grad2d, grads->rgb};
  int loss_tiles = 0;
  window_loss_views(cams, n_views, &w.l.lv, &loss_tiles);
  w.l.color = color;
  w.l.depth = depth;
  w.l.color_gt = color_gt;
  w.l.depth_gt = depth_gt;
  w.l.w_c = lp->w_l1_color;
  w.l.w_d = lp->w_l1_depth;
  w.l.w_s = lp->w_ssim;
  w.l.dC = dL_dcolor;
  w.l.dD = dL_ddepth;
  w.l.partials = static_cast<double *>(ws);
  double gw[11], gs = 0.0;
  for (int i = 0; i < 11; ++i) {
    gw[i] = std::exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
    gs += gw[i];
  }
  for (int i = 0; i < 11; ++i) w.l.g[i] = (float)(gw[i] / gs);
  w.n_tiles = vs.total_tiles;
  w.n_loss_tiles = loss_tiles;
  w.ctl = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + align_up(sizeof(double) * (size_t)loss_tiles));
  w.status = d_status;
  cudaStream_t st = as_stream(stream);
  FGS_CUDA(cudaMemsetAsync(w.ctl, 0, 8 * sizeof(uint32_t), st), "window counters");
  fgs_status s = FGS_WINDOW_DISPATCH(tiling, w, st, nullptr);
  if (s != FGS_OK) return s;
  k_window_reduce<<<1, 256, 0, st>>>(w.l.partials, loss_tiles, d_loss);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_render_window");
  return FGS_OK;
}
