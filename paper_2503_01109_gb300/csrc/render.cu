// render.cu -- eq1 alpha blending (colour, depth and opacity readings) per tile,
// and its reverse-order adjoint.
//
// One CTA per (view, tile); each thread owns one or two pixels of a compact warp
// block.  The tile's depth-ordered list is walked in batches of BATCH splats:
// each batch is gathered by id from the splat records (two float4 loads plus
// three colour planes per splat) into shared memory once and then evaluated by
// every pixel of the tile.  The walk stops when every pixel of the tile is
// saturated (T < 1e-4).
//
// The backward walks the same lists back to front from each warp's largest
// contributor position, recovering each pixel's transmittance by division by
// (1 - alpha) (alpha <= 0.99) instead of storing it.  Per-splat sums are
// accumulated over a thread's pixels, reduced across the warp with a 10-field
// butterfly, added per batch in shared memory and flushed with one global atomic
// per (CTA, splat, field).
#include "render_tile.cuh"

namespace fgs {


// Tile of this CTA: blockIdx.x, or its entry of the launch order (fgs_tile_order).
// An entry outside the view set's tiles is reported and its CTA does nothing.
__device__ __forceinline__ int ordered_tile(const int32_t *order, int total_tiles, int32_t *d_status) {
  if (!order) return blockIdx.x;
  const int t = order[blockIdx.x];
  if ((unsigned)t < (unsigned)total_tiles) return t;
  if (d_status && threadIdx.x == 0) atomicOr(d_status, FGS_DEV_BAD_ORDER);
  return -1;
}

template <int TW, int TH, int BATCH, int PX, int S = 1>
__global__ void __launch_bounds__((TW / S) * (TH / S) / PX) k_render_fwd(RenderArgs a) {
  pdl_enter();
  __shared__ __align__(16) char smem[TileSmem<BATCH>::fwd];
  const int t = ordered_tile(a.order, a.vs.total_tiles, a.d_status);
  if (t >= 0) render_fwd_tile<TW, TH, BATCH, PX, S>(a, t, smem);
}

#ifndef FGS_BWD_MINB
#define FGS_BWD_MINB 1
#endif
template <int TW, int TH, int BATCH, int PX>
__global__ void __launch_bounds__(TW *TH / PX, FGS_BWD_MINB) k_render_bwd(RenderBwdArgs a) {
  pdl_enter();
  __shared__ __align__(16) char smem[TileSmem<BATCH>::bwd];
  const int t = ordered_tile(a.order, a.vs.total_tiles, a.d_status);
  if (t >= 0) render_bwd_tile<TW, TH, BATCH, PX>(a, t, smem);
}

template <int TW, int TH, int BATCH>
static void launch_fwd(const RenderArgs &a, int blocks, cudaStream_t st) {
  constexpr int PX = PxPerThread<TW, TH>::fwd;
  pdl_launch(k_render_fwd<TW, TH, BATCH, PX>, blocks, TW * TH / PX, 0, st, a);
}
// The forward on the grid of every second pixel in x and y (one pixel per thread).
template <int TW, int TH, int BATCH>
static void launch_fwd_sampled(const RenderArgs &a, int blocks, cudaStream_t st) {
  pdl_launch(k_render_fwd<TW, TH, BATCH, 1, 2>, blocks, (TW / 2) * (TH / 2), 0, st, a);
}
template <int TW, int TH, int BATCH>
static void launch_bwd(const RenderBwdArgs &a, int blocks, cudaStream_t st) {
  constexpr int PX = PxPerThread<TW, TH>::bwd;
  pdl_launch(k_render_bwd<TW, TH, BATCH, PX>, blocks, TW * TH / PX, 0, st, a);
}

#define FGS_DISPATCH_TILING(tiling, FN, ...)                                          \
  do {                                                                                \
    const int tw__ = (tiling).tile_w, th__ = (tiling).tile_h, bd__ = (tiling).batch_depth; \
    if (tw__ == 16 && th__ == 16) {                                                   \
      if (bd__ == 32) FN<16, 16, 32>(__VA_ARGS__);                                    \
      else if (bd__ == 64) FN<16, 16, 64>(__VA_ARGS__);                               \
      else if (bd__ == 128) FN<16, 16, 128>(__VA_ARGS__);                             \
      else FN<16, 16, 256>(__VA_ARGS__);                                              \
    } else if (tw__ == 8) {                                                           \
      if (bd__ == 32) FN<8, 8, 32>(__VA_ARGS__);                                      \
      else if (bd__ == 64) FN<8, 8, 64>(__VA_ARGS__);                                 \
      else if (bd__ == 128) FN<8, 8, 128>(__VA_ARGS__);                               \
      else FN<8, 8, 256>(__VA_ARGS__);                                                \
    } else {                                                                          \
      if (bd__ == 32) FN<16, 32, 32>(__VA_ARGS__);                                    \
      else if (bd__ == 64) FN<16, 32, 64>(__VA_ARGS__);                               \
      else if (bd__ == 128) FN<16, 32, 128>(__VA_ARGS__);                             \
      else FN<16, 32, 256>(__VA_ARGS__);                                              \
    }                                                                                 \
  } while (0)

fgs_status launch_project_bwd(const fgs_gaussians *g, const DevViews &vs, const int32_t *radius,
                              const float *grad2d, int64_t stride, fgs_gaussians *grads, cudaStream_t st);

}  // namespace fgs

using namespace fgs;

extern "C" fgs_status fgs_render_fwd(const fgs_projected *proj, const fgs_gaussians *g,
                                     const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                     const int32_t *ids, const int32_t *tile_ranges,
                                     const int32_t *tile_order, float *color, float *depth, float *alpha,
                                     float *t_final, int32_t *n_contrib, int32_t *d_status, void *stream) {
  FGS_CHECK_ARG(proj && proj->splat, "fgs_render_fwd: NULL projection");
  if (!gaussians_ok(g, "g")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_render_fwd: unsupported tiling");
  FGS_CHECK_ARG(ids && tile_ranges && color && depth && alpha && t_final && n_contrib,
                "fgs_render_fwd: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(proj->splat) & 15) == 0, "fgs_render_fwd: splat alignment");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  RenderArgs a{vs, reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity, ids,
               reinterpret_cast<const int2 *>(tile_ranges), color, depth, alpha, t_final, n_contrib,
               tile_order, d_status};
  FGS_DISPATCH_TILING(tiling, launch_fwd, a, vs.total_tiles, as_stream(stream));
  count_launch();
  FGS_CHECK_LAUNCH("fgs_render_fwd");
  return FGS_OK;
}

extern "C" fgs_status fgs_render_fwd_sampled(const fgs_projected *proj, const fgs_gaussians *g,
                                             const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                             const int32_t *ids, const int32_t *tile_ranges,
                                             const int32_t *tile_order, int32_t sample_stride, float *color,
                                             float *depth, float *alpha, float *t_final, int32_t *n_contrib,
                                             int32_t *d_status, void *stream) {
  FGS_CHECK_ARG(proj && proj->splat, "fgs_render_fwd_sampled: NULL projection");
  if (!gaussians_ok(g, "g")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_render_fwd_sampled: unsupported tiling");
  FGS_CHECK_ARG(sample_stride == 2, "fgs_render_fwd_sampled: sample_stride must be 2");
  FGS_CHECK_ARG(tiling.tile_w == 16, "fgs_render_fwd_sampled: needs 16x16 or 16x32 tiles");
  FGS_CHECK_ARG(ids && tile_ranges && color && depth && alpha && t_final && n_contrib,
                "fgs_render_fwd_sampled: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(proj->splat) & 15) == 0, "fgs_render_fwd_sampled: splat alignment");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  RenderArgs a{vs, reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity, ids,
               reinterpret_cast<const int2 *>(tile_ranges), color, depth, alpha, t_final, n_contrib,
               tile_order, d_status};
  cudaStream_t st = as_stream(stream);
  const int bd = tiling.batch_depth, blocks = vs.total_tiles;
  if (tiling.tile_h == 16) {
    if (bd == 32) launch_fwd_sampled<16, 16, 32>(a, blocks, st);
    else if (bd == 64) launch_fwd_sampled<16, 16, 64>(a, blocks, st);
    else if (bd == 128) launch_fwd_sampled<16, 16, 128>(a, blocks, st);
    else launch_fwd_sampled<16, 16, 256>(a, blocks, st);
  } else {
    if (bd == 32) launch_fwd_sampled<16, 32, 32>(a, blocks, st);
    else if (bd == 64) launch_fwd_sampled<16, 32, 64>(a, blocks, st);
    else if (bd == 128) launch_fwd_sampled<16, 32, 128>(a, blocks, st);
    else launch_fwd_sampled<16, 32, 256>(a, blocks, st);
  }
  count_launch();
  FGS_CHECK_LAUNCH("fgs_render_fwd_sampled");
  return FGS_OK;
}

static fgs_status render_bwd_splats(const fgs_gaussians *g, const fgs_projected *proj, const DevViews &vs,
                                    fgs_tiling tiling, const int32_t *ids, const int32_t *tile_ranges,
                                    const int32_t *tile_order, const float *t_final, const int32_t *n_contrib,
                                    const float *dL_dcolor, const float *dL_ddepth, const float *dL_dalpha,
                                    float *grad2d, fgs_gaussians *grads, int32_t *d_status, cudaStream_t st) {
  RenderBwdArgs a{vs,      reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity,
                  ids,     reinterpret_cast<const int2 *>(tile_ranges), t_final, n_contrib, dL_dcolor,
                  dL_ddepth, dL_dalpha, grad2d, grads->rgb, tile_order, d_status};
  FGS_DISPATCH_TILING(tiling, launch_bwd, a, vs.total_tiles, st);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_render_bwd");
  return FGS_OK;
}

static fgs_status check_bwd_args(const fgs_gaussians *g, const fgs_projected *proj, fgs_tiling tiling,
                                 const int32_t *ids, const int32_t *tile_ranges, const float *t_final,
                                 const int32_t *n_contrib, const float *dL_dcolor, const float *grad2d,
                                 const fgs_gaussians *grads) {
  if (!gaussians_ok(g, "g") || !gaussians_ok(grads, "grads")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(grads->n >= g->n, "fgs_render_bwd: grads->n < g->n");
  FGS_CHECK_ARG(proj && proj->splat && proj->radius && proj->stride >= g->n, "fgs_render_bwd: projection");
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_render_bwd: unsupported tiling");
  FGS_CHECK_ARG(ids && tile_ranges && t_final && n_contrib && dL_dcolor && grad2d,
                "fgs_render_bwd: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(grad2d) & 15) == 0, "fgs_render_bwd: grad2d alignment");
  return FGS_OK;
}

extern "C" fgs_status fgs_render_bwd_splats(const fgs_gaussians *g, const fgs_projected *proj,
                                            const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                            const int32_t *ids, const int32_t *tile_ranges,
                                            const int32_t *tile_order, const float *t_final,
                                            const int32_t *n_contrib, const float *dL_dcolor,
                                            const float *dL_ddepth, const float *dL_dalpha, float *grad2d,
                                            fgs_gaussians *grads, int32_t *d_status, void *stream) {
  fgs_status s = check_bwd_args(g, proj, tiling, ids, tile_ranges, t_final, n_contrib, dL_dcolor, grad2d, grads);
  if (s != FGS_OK) return s;
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  return render_bwd_splats(g, proj, vs, tiling, ids, tile_ranges, tile_order, t_final, n_contrib, dL_dcolor,
                           dL_ddepth, dL_dalpha, grad2d, grads, d_status, as_stream(stream));
}

extern "C" fgs_status fgs_render_bwd(const fgs_gaussians *g, const fgs_projected *proj,
                                     const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                     const int32_t *ids, const int32_t *tile_ranges,
                                     const int32_t *tile_order, const float *t_final,
                                     const int32_t *n_contrib, const float *dL_dcolor,
                                     const float *dL_ddepth, const float *dL_dalpha, float *grad2d,
                                     fgs_gaussians *grads, int32_t *d_status, void *stream) {
  fgs_status s = check_bwd_args(g, proj, tiling, ids, tile_ranges, t_final, n_contrib, dL_dcolor, grad2d, grads);
  if (s != FGS_OK) return s;
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = as_stream(stream);
  FGS_CUDA(cudaMemsetAsync(grad2d, 0, sizeof(float) * 8 * (size_t)n_views * (size_t)proj->stride, st),
           "memset grad2d");
  s = render_bwd_splats(g, proj, vs, tiling, ids, tile_ranges, tile_order, t_final, n_contrib, dL_dcolor,
                        dL_ddepth, dL_dalpha, grad2d, grads, d_status, st);
  if (s != FGS_OK) return s;
  return launch_project_bwd(g, vs, proj->radius, grad2d, proj->stride, grads, st);
}
