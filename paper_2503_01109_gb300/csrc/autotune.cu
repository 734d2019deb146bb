// autotune.cu -- the tiling autotuner of the batched keyframe window.
//
// The window of Sec. III-C renders a handful of keyframes of mixed resolutions
// forward and backward in one persistent launch.  Which tile shape and batch
// depth is fastest depends on the views and the map (splat footprints, list
// lengths per tile), so the library times every supported tiling on the caller's
// own window -- projection, binning, the persistent forward / loss / adjoint
// launch and the projection adjoint, i.e. every stage whose cost depends on the
// tiling -- and returns the fastest.  The map is only read: its gradients go to
// scratch, and no optimiser step is taken.
#include <cfloat>

#include "common.cuh"

namespace fgs {

static const fgs_tiling kTunings[FGS_AUTOTUNE_CONFIGS] = {
    {8, 8, 32},   {8, 8, 64},   {8, 8, 128},   {8, 8, 256},   {16, 16, 32}, {16, 16, 64},
    {16, 16, 128}, {16, 16, 256}, {16, 32, 32}, {16, 32, 64}, {16, 32, 128}, {16, 32, 256}};

// Byte offsets of the scratch buffers inside the caller's workspace.
struct TuneLayout {
  size_t splat, radius, rect, keys, ids, ranges, order, order_ws, counters, bin, win, color, depth, alpha, t_final,
      n_contrib, dC, dD, grad2d, grads, total;
  size_t bin_bytes, win_bytes, order_bytes;
  int64_t max_tiles, pix;
};

static bool tune_layout(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views, int64_t pair_capacity,
                        TuneLayout *L) {
  if (!g || !cams || n_views < 1 || n_views > FGS_MAX_VIEWS || pair_capacity < 1 ||
      pair_capacity > (int64_t(1) << 31) - 1 || g->capacity < 1)
    return false;
  const int64_t cap = g->capacity, V = n_views;
  L->max_tiles = 0;
  L->bin_bytes = 0;
  for (const fgs_tiling &t : kTunings) {
    const int64_t tiles = fgs_num_tiles(cams, n_views, t);
    if (tiles < 0) return false;
    L->max_tiles = std::max(L->max_tiles, tiles);
    const size_t b = fgs_bin_sort_workspace_size(cams, n_views, t, V * cap, pair_capacity);
    if (b == 0) return false;
    L->bin_bytes = std::max(L->bin_bytes, b);
  }
  L->win_bytes = fgs_render_window_workspace_size(cams, n_views);
  if (L->win_bytes == 0) return false;
  L->pix = 0;
  for (int v = 0; v < n_views; ++v) L->pix += (int64_t)cams[v].width * cams[v].height;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L->splat = take(sizeof(float) * 8 * V * cap);
  L->radius = take(sizeof(int32_t) * V * cap);
  L->rect = take(sizeof(uint16_t) * 4 * V * cap);
  L->keys = take(sizeof(uint32_t) * pair_capacity);
  L->ids = take(sizeof(int32_t) * pair_capacity);
  L->ranges = take(sizeof(int32_t) * 2 * L->max_tiles);
  L->order = take(sizeof(int32_t) * L->max_tiles);
  L->order_bytes = align_up(sizeof(int32_t) * L->max_tiles);
  L->order_ws = take(L->order_bytes);
  L->counters = take(64);  // num_pairs (int64), status (int32), loss (float)
  L->bin = take(L->bin_bytes);
  L->win = take(L->win_bytes);
  L->color = take(sizeof(float) * 3 * L->pix);
  L->depth = take(sizeof(float) * L->pix);
  L->alpha = take(sizeof(float) * L->pix);
  L->t_final = take(sizeof(float) * L->pix);
  L->n_contrib = take(sizeof(int32_t) * L->pix);
  L->dC = take(sizeof(float) * 3 * L->pix);
  L->dD = take(sizeof(float) * L->pix);
  L->grad2d = take(sizeof(float) * 8 * V * cap);
  L->grads = take(sizeof(float) * 14 * cap);
  L->total = o;
  return true;
}

// One window pass of tiling t: everything whose cost depends on the tiling.  The
// window takes its tiles in the heaviest-first order of the previous pass's
// render (none on the first pass), and the pass ends by ordering them for the
// next, as a mapping loop over the window does.
static fgs_status tune_pass(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views, const float *color_gt,
                            const float *depth_gt, const fgs_loss_params *lp, int64_t pair_capacity, char *ws,
                            const TuneLayout &L, fgs_tiling t, bool ordered, cudaStream_t st) {
  const int64_t cap = g->capacity;
  fgs_projected proj{cap, reinterpret_cast<float *>(ws + L.splat), reinterpret_cast<int32_t *>(ws + L.radius),
                     reinterpret_cast<uint16_t *>(ws + L.rect)};
  int64_t *num_pairs = reinterpret_cast<int64_t *>(ws + L.counters);
  int32_t *status = reinterpret_cast<int32_t *>(ws + L.counters + 8);
  float *loss = reinterpret_cast<float *>(ws + L.counters + 16);
  float *gr = reinterpret_cast<float *>(ws + L.grads);
  fgs_gaussians grads{g->n, cap, g->d_n, gr, gr + 3 * cap, gr + 6 * cap, gr + 10 * cap, gr + 11 * cap};
  fgs_status s = fgs_project(g, cams, n_views, t, &proj, status, st);
  if (s != FGS_OK) return s;
  s = fgs_bin_sort(&proj, g->d_n ? cap : g->n, g->d_n, cams, n_views, t, ws + L.bin, L.bin_bytes,
                   reinterpret_cast<uint32_t *>(ws + L.keys), reinterpret_cast<int32_t *>(ws + L.ids), pair_capacity,
                   reinterpret_cast<int32_t *>(ws + L.ranges), num_pairs, status, st);
  if (s != FGS_OK) return s;
  FGS_CUDA(cudaMemsetAsync(ws + L.grad2d, 0, sizeof(float) * 8 * n_views * cap, st), "fgs_autotune: memset");
  FGS_CUDA(cudaMemsetAsync(ws + L.grads, 0, sizeof(float) * 14 * cap, st), "fgs_autotune: memset");
  FGS_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st), "fgs_autotune: memset");
  int32_t *order = reinterpret_cast<int32_t *>(ws + L.order);
  s = fgs_render_window(g, &proj, cams, n_views, t, reinterpret_cast<int32_t *>(ws + L.ids),
                        reinterpret_cast<int32_t *>(ws + L.ranges), ordered ? order : nullptr, color_gt, depth_gt, lp,
                        reinterpret_cast<float *>(ws + L.color), reinterpret_cast<float *>(ws + L.depth),
                        reinterpret_cast<float *>(ws + L.alpha), reinterpret_cast<float *>(ws + L.t_final),
                        reinterpret_cast<int32_t *>(ws + L.n_contrib), reinterpret_cast<float *>(ws + L.dC),
                        reinterpret_cast<float *>(ws + L.dD), reinterpret_cast<float *>(ws + L.grad2d), &grads, loss,
                        ws + L.win, L.win_bytes, status, st);
  if (s != FGS_OK) return s;
  s = fgs_tile_order(cams, n_views, t, reinterpret_cast<int32_t *>(ws + L.n_contrib), order, ws + L.order_ws,
                     L.order_bytes, st);
  if (s != FGS_OK) return s;
  return fgs_project_bwd(g, &proj, cams, n_views, reinterpret_cast<float *>(ws + L.grad2d), &grads, st);
}

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_autotune_workspace_size(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views,
                                              int64_t pair_capacity) {
  TuneLayout L;
  return tune_layout(g, cams, n_views, pair_capacity, &L) ? L.total : 0;
}

extern "C" fgs_status fgs_autotune(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views,
                                   const float *color_gt, const float *depth_gt, const fgs_loss_params *loss,
                                   int64_t pair_capacity, int32_t reps, void *ws, size_t ws_bytes,
                                   fgs_tiling *best, float *ms_out, void *stream) {
  if (!gaussians_ok(g, "fgs_autotune: g")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(color_gt && depth_gt && loss && best && reps >= 1 && reps <= 1000,
                "fgs_autotune: NULL argument or reps outside 1..1000");
  TuneLayout L;
  FGS_CHECK_ARG(tune_layout(g, cams, n_views, pair_capacity, &L), "fgs_autotune: bad views or pair_capacity");
  FGS_CHECK_ARG(ws && (reinterpret_cast<uintptr_t>(ws) & 255) == 0 && ws_bytes >= L.total,
                "fgs_autotune: workspace %zu < %zu bytes or not 256-byte aligned", ws_bytes, L.total);
  cudaStream_t st = as_stream(stream);
  char *w = static_cast<char *>(ws);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FGS_CUDA(cudaEventCreate(&e0), "fgs_autotune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("fgs_autotune: event");
    return FGS_ERR_CUDA;
  }
  fgs_status result = FGS_OK;
  float best_ms = FLT_MAX;
  int best_i = -1;
  for (int i = 0; i < FGS_AUTOTUNE_CONFIGS && result == FGS_OK; ++i) {
    const fgs_tiling t = kTunings[i];
    float ms = FLT_MAX;
    if (cudaMemsetAsync(w + L.counters, 0, 64, st) != cudaSuccess) {
      set_error("fgs_autotune: memset");
      result = FGS_ERR_CUDA;
      break;
    }
    // one untimed pass (first use of the tiling's kernels), then `reps` timed ones
    result = tune_pass(g, cams, n_views, color_gt, depth_gt, loss, pair_capacity, w, L, t, false, st);
    if (result != FGS_OK) break;
    if (cudaEventRecord(e0, st) != cudaSuccess) result = FGS_ERR_CUDA;
    for (int r = 0; r < reps && result == FGS_OK; ++r)
      result = tune_pass(g, cams, n_views, color_gt, depth_gt, loss, pair_capacity, w, L, t, true, st);
    if (result != FGS_OK) break;
    int32_t status = 0;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaMemcpy(&status, w + L.counters + 8, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("fgs_autotune: timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      result = FGS_ERR_CUDA;
      break;
    }
    ms /= (float)reps;
    if (status != 0) ms = FLT_MAX;  // e.g. the pairs of this tiling exceed pair_capacity
    if (ms_out) ms_out[i] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != FGS_OK) return result;
  if (best_i < 0) {
    set_error("fgs_autotune: every tiling set a device status bit (pair_capacity too small?)");
    return FGS_ERR_CAPACITY;
  }
  *best = kTunings[best_i];
  return FGS_OK;
}
