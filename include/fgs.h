/*
 * fgs.h -- C ABI of the GB300 (sm_103a) Fourier-seeded Gaussian-splatting mapping path.
 *
 * The paper (FGS-SLAM, arXiv 2503.01109) optimises a dense map of 3D Gaussians
 * G{mu, S, R, alpha, c} (Sec. III) by rasterisation rendering (eq1) and seeds new
 * Gaussians where a Fourier high-pass of the frame says detail lives (Sec. III-A,
 * eq2-eq11).  This library is that data-parallel path: every entry point launches
 * hand-written CUDA kernels on the caller's stream.
 *
 * Equations are named by their LaTeX labels eq1..eq16.  The paper has no eq6, so
 * from eq7 on the printed equation number is one less than the label.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every pointer named d_* or documented as "device" is device memory owned by
 *    the caller.  Host structs (fgs_camera, fgs_gaussians, ...) are read during the
 *    call only; the device pointers inside them must stay valid until the stream
 *    work completes.  The library never allocates device memory: scratch comes
 *    from caller-given workspace (size queried with the *_workspace_size calls).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous, never synchronise the host, and can be captured
 *    into a CUDA graph.  The projection, binning, render, loss, Adam, seeding,
 *    pruning, tracking and keyframe kernels are launched with programmatic
 *    dependent launch (each waits for its predecessor on the stream before
 *    touching memory, so plain stream order holds); FGS_PDL=0 in the
 *    environment launches them without it.
 *  - The return value reports argument and launch errors (fgs_status).  On a
 *    non-zero return nothing was launched or the launch failed; the message is in
 *    fgs_last_error() (thread-local).  No C++ exception crosses the ABI.
 *  - Conditions found on the device (capacity exceeded, bounded wait timed out,
 *    non-finite value) are OR-ed as FGS_DEV_* bits into *d_status (int32 device
 *    word).  The caller reads it after synchronising; outputs of a call that set
 *    a bit are not valid.
 *  - Camera model: pinhole, OpenCV axes (x right, y down, z forward), pixel (x, y)
 *    centred at integer coordinates, world_to_cam = [R | t] row-major 3x4.
 *  - Gaussian parameters are structure-of-arrays planes of float32 with plane
 *    stride `capacity`: means[3][cap], log_scales[3][cap], quats[4][cap] (w, x, y,
 *    z; normalised inside the kernels), opacity_logits[cap], rgb[3][cap] (colour
 *    directly, spherical-harmonics degree 0).  Scale = exp(log_scale), opacity =
 *    sigmoid(logit).
 *  - Multi-view images are concatenated view after view: view v starts at pixel
 *    offset sum_{u<v} W_u H_u; colour planes of a view are [3][H_v][W_v].
 *  - Tiles of every view are numbered globally: view v's tiles start at
 *    sum_{u<v} tiles_x(u) * tiles_y(u), row-major inside the view.
 */
#ifndef FGS_H
#define FGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGS_VERSION 100

typedef int32_t fgs_status;
enum {
  FGS_OK = 0,
  FGS_ERR_INVALID_ARGUMENT = 1,
  FGS_ERR_CUDA = 2,
  FGS_ERR_CAPACITY = 3,
  FGS_ERR_TIMEOUT = 4,
  FGS_ERR_UNSUPPORTED = 5,
  FGS_ERR_NONFINITE = 6
};

/* Bits OR-ed into the device status word. */
enum {
  FGS_DEV_PAIR_OVERFLOW = 1, /* (tile, Gaussian) pairs exceeded pair_capacity        */
  FGS_DEV_TIMEOUT = 2,       /* a bounded device wait gave up                         */
  FGS_DEV_NONFINITE = 4,     /* a non-finite value was met where one is not allowed   */
  FGS_DEV_MAP_FULL = 8,      /* seeding wanted more Gaussians than the map capacity   */
  FGS_DEV_WORK_OVERFLOW = 16, /* a window work list exceeded its capacity             */
  FGS_DEV_BAD_ORDER = 32      /* a tile_order entry outside the view set's tiles       */
};

#define FGS_MAX_VIEWS 16

typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float world_to_cam[12]; /* row-major [R | t] */
  float znear;            /* Gaussians with camera z < znear are culled */
} fgs_camera;

typedef struct {
  int64_t n;             /* Gaussians in use (host count, or upper bound when d_n is set) */
  int64_t capacity;      /* plane stride in elements                                     */
  int64_t *d_n;          /* optional device count (<= n); NULL = use n                     */
  float *means;          /* [3][capacity]                                                 */
  float *log_scales;     /* [3][capacity]                                                 */
  float *quats;          /* [4][capacity]  w, x, y, z                                     */
  float *opacity_logits; /* [capacity]                                                    */
  float *rgb;            /* [3][capacity]                                                 */
} fgs_gaussians;

/* Per-view screen-space splats (the "2D projection" of Sec. III).  Record r of
 * view v lives at index v * stride + r. */
typedef struct {
  int64_t stride;   /* records per view (>= the Gaussians' n)                          */
  float *splat;     /* [n_views][stride][8]: mean2d.x, mean2d.y, conic a, b, c,       */
                    /*   opacity, depth (camera z), support threshold (fgs_project)     */
  int32_t *radius;  /* [n_views][stride]  ceil(3 sqrt(lambda_max)); 0 = culled          */
  uint16_t *rect;   /* [n_views][stride][4] inclusive tile bounds x0, y0, x1, y1        */
                    /*   (x0 > x1 = touches no tile)                                    */
} fgs_projected;

typedef struct {
  int32_t tile_w, tile_h; /* 8x8, 16x16 or 16x32 (w x h)                             */
  int32_t batch_depth;    /* Gaussians staged per shared-memory batch: 32..256, pow2  */
} fgs_tiling;

/* ---------------------------------------------------------------------------------
 * fgs_project -- EWA projection of every Gaussian into every view (Sec. III: the
 * covariance C = R S S^T R^T and its 2D projection that eq1 blends).
 *   p = R_cam mu + t; culled if p.z < znear.
 *   Sigma' = J R_cam C R_cam^T J^T + 0.3 I, J the perspective Jacobian at p with
 *   x/z, y/z clamped to +-1.3 tan(half field of view).  conic = Sigma'^-1.
 *   mean2d = (fx x/z + cx, fy y/z + cy); radius = ceil(3 sqrt(lambda_max(Sigma')));
 *   opacity = sigmoid(logit); support threshold thr = 2 ln(255 opacity) + 0.01
 *   (alpha = opacity e^(-q/2) can reach 1/255 only where the Mahalanobis form
 *   q <= thr; -1 when 255 opacity <= 1); rect = tiles whose pixel-centre box
 *   meets [mean2d -+ min(3, sqrt(thr)) sqrt(diag Sigma')] (empty if thr < 0).
 *   The splat record's last slot holds thr; fgs_bin_sort further drops the
 *   tiles of the rect on which q exceeds thr at every pixel centre.
 * in : g (n Gaussians), cams[n_views] (host), tiling.
 * out: out->splat/radius/rect for n_views x g->n records (stride out->stride >= n).
 *   With g->d_n the slots at or past *g->d_n get radius 0 and keep their splat and
 *   rect as they were (only the records of live Gaussians are written in full).
 * Failure detection: a Gaussian whose mean, scales exp(log_scales), normalised
 *   quaternion, opacity or colour is not finite is culled from every view (radius
 *   0), and FGS_DEV_NONFINITE is or-ed into *d_status when d_status is not NULL.
 * err: INVALID_ARGUMENT for n_views outside 1..FGS_MAX_VIEWS, bad tiling, NULLs. */
fgs_status fgs_project(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views,
                       fgs_tiling tiling, fgs_projected *out, int32_t *d_status, void *stream);

/* Total tile count of a view set under a tiling (host helper; -1 on bad input). */
int64_t fgs_num_tiles(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling);

/* ---------------------------------------------------------------------------------
 * fgs_bin_sort -- tile binning and depth ordering of the splats that eq1 blends
 * front to back.  Produces, for every global tile, the list of Gaussians whose
 * rect contains the tile and whose support ellipse {q <= thr} meets the tile's
 * rectangle of pixel centres, decided per tile row from the ellipse's x-extent
 * within the row's strip (float32, a fixed order of rounded steps), ordered by
 * (float32 depth bits, Gaussian id).
 *   tile_keys[k], ids[k] for k < *d_num_pairs: global tile index and Gaussian id,
 *   sorted by (tile, depth, id).  tile_keys may be NULL: the renders read only ids
 *   and tile_ranges, which determine the tile of every pair.  tile_ranges[2*t], [2*t+1] = [start, end) of tile t
 *   (0, 0 for an empty tile).
 * ws/ws_bytes: scratch of at least fgs_bin_sort_workspace_size(cams, n_views,
 *   tiling, n_views*stride, pair_capacity) bytes, 256-byte aligned.
 * Device errors: FGS_DEV_PAIR_OVERFLOW when the pair count, or the count of
 *   (record, tile row) entries of the rows' lists, exceeds pair_capacity;
 *   *d_num_pairs then holds the required count (for the rows: a lower bound) and
 *   the lists are not valid.  The compaction and the depth sort chain their tiles
 *   through decoupled look-backs whose waits are bounded (1 s): one that gives up
 *   sets FGS_DEV_TIMEOUT and the lists are not valid.
 * n, d_n: the records of slots 0 .. n-1 of every view are binned, or, when d_n
 *   (device) is not NULL, of slots 0 .. min(n, *d_n) - 1: the live count of a map
 *   whose count stays on the device, whose records past it fgs_project leaves
 *   with radius 0 but does not rewrite.
 * err: INVALID_ARGUMENT for small workspace, pair_capacity outside 1..2^31-1, more
 *   than 4096 tile rows over all views, n_views * n above 2^30 - 1. */
fgs_status fgs_bin_sort(const fgs_projected *proj, int64_t n, const int64_t *d_n, const fgs_camera *cams,
                        int32_t n_views, fgs_tiling tiling, void *ws, size_t ws_bytes,
                        uint32_t *tile_keys, int32_t *ids, int64_t pair_capacity,
                        int32_t *tile_ranges, int64_t *d_num_pairs, int32_t *d_status,
                        void *stream);
/* Workspace of fgs_bin_sort for this view set and tiling (0 on bad input). */
size_t fgs_bin_sort_workspace_size(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                   int64_t n_records, int64_t pair_capacity);

/* ---------------------------------------------------------------------------------
 * fgs_render_fwd -- alpha blending of eq1 for the three readings the paper gives
 * (colour gamma = c, depth gamma = d, opacity gamma = 1), front to back per pixel:
 *   power = -(a dx^2 + c dy^2)/2 - b dx dy, d = mean2d - pixel; skipped if > 0;
 *   alpha = min(0.99, opacity e^power), skipped if < 1/255;
 *   stop before a Gaussian whose T (1 - alpha) < 1e-4;
 *   C += rgb alpha T, D += z alpha T, A += alpha T, T *= (1 - alpha).
 * out (per view, concatenated): color [3][H][W], depth [H][W] (unnormalised
 *   sum z alpha T), alpha [H][W] (sum alpha T), t_final [H][W] (T after the last
 *   blended Gaussian), n_contrib [H][W] (1 + list position of the last blended
 *   Gaussian, 0 if none).  The backward reads t_final and n_contrib.
 * Background is 0.
 * tile_order: NULL, or a permutation of the view set's tiles [total_tiles] int32
 *   (device; e.g. from fgs_tile_order) giving the order in which the tiles'
 *   CTAs are launched.  A permutation changes no output, only how well the
 *   launch fills the GPU.  The entries are not checked for being one: a tile
 *   missing from the list is not rendered, a repeated one is rendered (and by
 *   the adjoint accumulated) twice.  An entry outside 0 .. total_tiles - 1 is
 *   skipped and or-es FGS_DEV_BAD_ORDER into *d_status when d_status is not NULL. */
fgs_status fgs_render_fwd(const fgs_projected *proj, const fgs_gaussians *g,
                          const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                          const int32_t *ids, const int32_t *tile_ranges,
                          const int32_t *tile_order, float *color, float *depth, float *alpha,
                          float *t_final, int32_t *n_contrib, int32_t *d_status, void *stream);

/* fgs_render_fwd_sampled -- fgs_render_fwd on the grid of pixels with
 * x % s == 0 and y % s == 0 (s = sample_stride, which must be 2; tiling 16x16 or
 * 16x32): those pixels get exactly fgs_render_fwd's values (the same arithmetic
 * over the same lists), every other pixel the background (colour, depth and alpha
 * 0, t_final 1, n_contrib 0).  For a consumer that reads the render only on such
 * a grid: the seeding step (fgs_fourier_seed) places seeds only on the m- and
 * n-grids of Sec. III-A, so with m and n even its seeds are those of a full render
 * (its mask's bit 2, M_m, then reflects the background off the grid).  One thread
 * per grid pixel: a quarter of the blending work.  tile_order as fgs_render_fwd. */
fgs_status fgs_render_fwd_sampled(const fgs_projected *proj, const fgs_gaussians *g,
                                  const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                  const int32_t *ids, const int32_t *tile_ranges,
                                  const int32_t *tile_order, int32_t sample_stride, float *color,
                                  float *depth, float *alpha, float *t_final, int32_t *n_contrib,
                                  int32_t *d_status, void *stream);

/* fgs_tile_order -- the launch order of the render calls' tiles, heaviest first:
 * the view set's tiles sorted by the largest n_contrib of their pixels
 * (descending, capped at 4095; tiles with equal keys in no fixed order).  One
 * CTA renders one tile and a tile's work grows with that count, so launching
 * the heavy tiles first keeps the SMs busy to the end of the launch (longest
 * processing time first).  n_contrib: a render's [n_views][H][W] output (the
 * forward whose adjoint follows, or a recent render of the same views: any
 * n_contrib gives a valid permutation).
 * out: tile_order [total_tiles] int32 (device), a permutation of 0 .. total_tiles-1.
 * ws: fgs_tile_order_workspace_size(...) bytes (device).  Two kernel launches. */
fgs_status fgs_tile_order(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                          const int32_t *n_contrib, int32_t *tile_order, void *ws, size_t ws_bytes,
                          void *stream);
size_t fgs_tile_order_workspace_size(const fgs_camera *cams, int32_t n_views, fgs_tiling tiling);

/* ---------------------------------------------------------------------------------
 * fgs_render_bwd -- reverse-mode adjoint of fgs_render_fwd and fgs_project: the
 * gradient of the mapping loss (eq16) with respect to every Gaussian parameter,
 * given dL/d(colour, depth, alpha) per pixel.  The per-pixel transmittance is
 * recomputed back to front by division by (1 - alpha) (alpha <= 0.99), nothing is
 * stored per (pixel, Gaussian).
 * grad2d: scratch [n_views][stride][8] floats (zeroed by the call).
 * grads : gradients are ADDED into grads' planes (caller zeroes them); layout as g.
 * dL_ddepth and dL_dalpha may be NULL (treated as zero).
 * tile_order as fgs_render_fwd (the forward's n_contrib through fgs_tile_order
 *   gives this call's heaviest-first order). */
fgs_status fgs_render_bwd(const fgs_gaussians *g, const fgs_projected *proj,
                          const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                          const int32_t *ids, const int32_t *tile_ranges,
                          const int32_t *tile_order, const float *t_final, const int32_t *n_contrib,
                          const float *dL_dcolor, const float *dL_ddepth,
                          const float *dL_dalpha, float *grad2d, fgs_gaussians *grads,
                          int32_t *d_status, void *stream);

/* The two halves of fgs_render_bwd as separate calls (one kernel each):
 * fgs_render_bwd_splats ADDS the per-splat gradients (mean2d, conic, opacity,
 *   depth) into grad2d [n_views][stride][8] and the colour gradients into
 *   grads->rgb; the caller zeroes both first.
 * fgs_project_bwd ADDS the chain rule of fgs_project from grad2d into grads'
 *   means, log_scales, quats and opacity_logits. */
fgs_status fgs_render_bwd_splats(const fgs_gaussians *g, const fgs_projected *proj,
                                 const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                 const int32_t *ids, const int32_t *tile_ranges,
                                 const int32_t *tile_order, const float *t_final,
                                 const int32_t *n_contrib,
                                 const float *dL_dcolor, const float *dL_ddepth,
                                 const float *dL_dalpha, float *grad2d, fgs_gaussians *grads,
                                 int32_t *d_status, void *stream);
fgs_status fgs_project_bwd(const fgs_gaussians *g, const fgs_projected *proj,
                           const fgs_camera *cams, int32_t n_views, const float *grad2d,
                           fgs_gaussians *grads, void *stream);

/* ---------------------------------------------------------------------------------
 * fgs_loss -- the mapping loss of eq16 per view, summed over views:
 *   w_l1_color * mean|C - C_gt| + w_l1_depth * mean_px([D_gt > 0] |D - D_gt|)
 *   + w_ssim * (1 - mean SSIM(C, C_gt)),
 * SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero
 * padding, averaged over the 3 H W colour samples.  (eq16's (1 - lambda_i) is
 * w_ssim.)  Writes dL/dC and dL/dD and ADDS the loss value to *d_loss.
 * ws: fgs_loss_workspace_size(cams, n_views) bytes.  The value is reduced in a
 * fixed order, so it is bit-reproducible run to run. */
typedef struct {
  float w_l1_color, w_l1_depth, w_ssim;
} fgs_loss_params;
fgs_status fgs_loss(const fgs_camera *cams, int32_t n_views, const float *color,
                    const float *depth, const float *color_gt, const float *depth_gt,
                    const fgs_loss_params *params, float *dL_dcolor, float *dL_ddepth,
                    float *d_loss, void *ws, size_t ws_bytes, void *stream);
size_t fgs_loss_workspace_size(const fgs_camera *cams, int32_t n_views);

/* fgs_loss_noalloc -- fgs_loss without a workspace argument, for callers that
 * may not allocate device memory: a host that owns every device byte through
 * its own pool, or a real-time loop where cudaMalloc's latency and implicit
 * synchronisation are not acceptable.  The paper has no counterpart; this is a
 * deployment convenience.
 *   Same arguments, layouts, outputs and device behaviour as fgs_loss (the loss
 *   value is ADDED to *d_loss).  The per-tile partial sums go to a scratch array
 *   compiled into the library: FGS_LOSS_NOALLOC_MAX_TILES doubles (512 KiB),
 *   i.e. at most that many 32x32 loss tiles over all views (sum over views of
 *   ceil(W/32) * ceil(H/32); 65536 tiles = 67 M pixels, 78 views of 1200x680).
 *   Larger view sets return FGS_ERR_CAPACITY before anything is launched.
 *   Every device that loads the library holds the array until the process
 *   exits.  The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and caches it for the life of the process, so make
 *   that first call before any stream capture on that device, and do not call
 *   it again after cudaDeviceReset on that device (the reset unloads the
 *   array; the cached address would then be stale).  The call allocates
 *   nothing.
 *   All calls share the one array: calls whose kernels can overlap on the GPU
 *   (different streams without ordering) race on it and give wrong sums.
 *   Nothing in the array needs clearing: every call writes each partial it
 *   reads. */
#define FGS_LOSS_NOALLOC_MAX_TILES 65536
fgs_status fgs_loss_noalloc(const fgs_camera *cams, int32_t n_views, const float *color,
                            const float *depth, const float *color_gt, const float *depth_gt,
                            const fgs_loss_params *params, float *dL_dcolor, float *dL_ddepth,
                            float *d_loss, void *stream);

/* fgs_scale_reg -- scale regulariser eq15 (per-Gaussian mean of the first two
 * linear scales, epsilon = 0) times `weight`; ADDS its gradient to
 * grads->log_scales and its value to *d_loss.  ws: fgs_scale_reg_workspace_size. */
fgs_status fgs_scale_reg(const fgs_gaussians *g, float weight, fgs_gaussians *grads,
                         float *d_loss, void *ws, size_t ws_bytes, void *stream);
size_t fgs_scale_reg_workspace_size(int64_t n);

/* fgs_adam -- bias-corrected Adam step on every Gaussian parameter (the map
 * optimisation of Sec. III-D; the paper does not name the optimiser).
 * lr per group: means, log_scales, quats, opacity, rgb.  The step number t >= 1 is
 * params->step, or, when d_step is not NULL, *d_step + 1 read on the device
 * (the call then increments *d_step, so a captured graph can be replayed).
 * Per element: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), with the square root
 * and the quotient by the hardware approximations (a few ulp). */
typedef struct {
  float lr[5];
  float beta1, beta2, eps;
  int32_t step;
} fgs_adam_params;
fgs_status fgs_adam(fgs_gaussians *params, const fgs_gaussians *grads, fgs_gaussians *m,
                    fgs_gaussians *v, const fgs_adam_params *hp, int32_t *d_step,
                    void *stream);

/* fgs_project_bwd_adam -- the end of a mapping iteration (Sec. III-D) in two
 * passes instead of four calls: per Gaussian, the chain rule of fgs_project from
 * grad2d (as fgs_project_bwd) plus the eq15 gradient with weight reg_weight (as
 * fgs_scale_reg; 0 = none; its loss is added to *d_loss) is STORED into the 11
 * geometric planes of grads (their old contents are ignored); then the Adam step of
 * fgs_adam on all 14 parameters, with the RGB gradient taken from grads->rgb.
 * Afterwards grads->rgb and every grad2d record read are zero again, ready for the
 * next fgs_render_bwd_splats (the caller zeroes both once, before the first use);
 * the geometric planes keep this step's gradients.  m and v as in fgs_adam; the
 * step number as in fgs_adam.
 * ws: fgs_project_bwd_adam_workspace_size(params->n) bytes, 16-byte aligned.
 * err: INVALID_ARGUMENT for NULLs, small workspace, grads / m / v not covering params. */
fgs_status fgs_project_bwd_adam(fgs_gaussians *params, const fgs_projected *proj, const fgs_camera *cams,
                                int32_t n_views, float *grad2d, fgs_gaussians *grads, float reg_weight,
                                float *d_loss, fgs_gaussians *m, fgs_gaussians *v, const fgs_adam_params *hp,
                                int32_t *d_step, void *ws, size_t ws_bytes, void *stream);
size_t fgs_project_bwd_adam_workspace_size(int64_t n);

/* fgs_grid_barrier_probe -- self-test of the bounded grid barrier that separates
 * the phases of fgs_render_window (the paper has no counterpart: this is the
 * failure detection of the persistent launch).  n_blocks CTAs of a cooperative
 * grid each arrive once at a barrier that waits for n_expected arrivals; a CTA
 * gives up after timeout_ns, or-es FGS_DEV_TIMEOUT into *d_status and returns, so
 * a barrier that can never complete (n_expected > n_blocks: an arrival nothing
 * will make) ends in about timeout_ns and leaves the context usable.
 * out: *d_passed += the number of CTAs whose wait completed (n_blocks when
 *   n_expected == n_blocks, 0 when it is larger).
 * ws: 32 bytes of device scratch (cleared by the call).
 * err: INVALID_ARGUMENT unless 1 <= n_blocks <= the SM count, n_expected >=
 *   n_blocks and 1 us <= timeout_ns <= 5 s; NULLs. */
fgs_status fgs_grid_barrier_probe(int32_t n_blocks, int32_t n_expected, int64_t timeout_ns, void *ws,
                                  size_t ws_bytes, uint32_t *d_passed, int32_t *d_status, void *stream);

/* fgs_lookback_probe -- self-test of the bounded decoupled look-back that chains
 * the tiles of the binning's depth sort (the paper has no counterpart: this is the
 * failure detection of that wait).  n_tiles CTAs each take a tile by ticket, publish
 * a count of 1 for each of 256 digits and sum the counts of the earlier tiles, as a
 * sort pass does.  With skip_first the first tile publishes nothing, so every later
 * wait can only end by its limit: it gives up after timeout_ns, or-es
 * FGS_DEV_TIMEOUT into *d_status and returns, leaving the context usable.
 * out: sums [n_tiles][256] int32: tile t's sums (t everywhere when no wait gave
 *   up; the first tile's row is left unwritten with skip_first).
 * ws: fgs_lookback_probe_workspace_size(n_tiles) bytes, 256-byte aligned (cleared
 *   by the call).
 * err: INVALID_ARGUMENT unless 1 <= n_tiles <= 4096 and 1 us <= timeout_ns <= 5 s;
 *   NULLs; small workspace. */
fgs_status fgs_lookback_probe(int32_t n_tiles, int32_t skip_first, int64_t timeout_ns, void *ws,
                              size_t ws_bytes, int32_t *sums, int32_t *d_status, void *stream);
size_t fgs_lookback_probe_workspace_size(int32_t n_tiles);

/* ---------------------------------------------------------------------------------
 * fgs_prune -- Gaussian pruning (Sec. III-A, "Gaussian Pruning"): removes every
 * Gaussian that has grown too large in some dimension or whose opacity is below a
 * threshold, so that mapping can re-seed the region.  Decided in float32 on the
 * parameters themselves: Gaussian i is removed when
 *   opacity_logits[i] < p->min_logit   (opacity below sigmoid(min_logit)), or
 *   max_k log_scales[k][i] > p->max_log_scale   (largest scale above exp(max_log_scale)).
 * With K survivors, those below index K keep their slots; the removed slots
 * below K, lowest first, receive the survivors at index K and above, highest
 * first (only as many Gaussians move as were removed below K).  The same moves
 * are made in the Adam moments m and v when they are not NULL (same capacity as
 * g); slots from K on are left as they were.
 * Count: the live count is g->d_n ? *g->d_n : g->n; the new count is written to
 *   *d_num_kept and, when g->d_n is set, to *g->d_n (so a captured graph can
 *   replay it); the host g->n is not changed.
 * ws: fgs_prune_workspace_size(g->capacity) bytes, 256-byte aligned.
 * err: INVALID_ARGUMENT for NULLs, small workspace, m / v of another capacity. */
typedef struct {
  float min_logit;      /* remove when the opacity logit is below this             */
  float max_log_scale;  /* remove when the largest log-scale is above this         */
} fgs_prune_params;
fgs_status fgs_prune(fgs_gaussians *g, fgs_gaussians *m, fgs_gaussians *v, const fgs_prune_params *p,
                     void *ws, size_t ws_bytes, int64_t *d_num_kept, void *stream);
size_t fgs_prune_workspace_size(int64_t capacity);

/* ---------------------------------------------------------------------------------
 * fgs_covisibility -- co-visibility of keyframes with the current frame (Sec.
 * III-C, "Keyframe Selection"): the fraction of the current frame's observed
 * points that a keyframe also sees.  The current depth map is sampled every `step`
 * pixels in x and y from (0, 0); a sample with depth d > 0 is back-projected,
 *   p_c = (d (x - cx) / fx, d (y - cy) / fy, d),  p_w = R^T (p_c - t),
 * and counted as inside keyframe k when q = R_k p_w + t_k has q.z > znear_k and
 * projects to u = fx_k (q.x / q.z) + cx_k in [-0.5, W_k - 0.5), v likewise in
 * [-0.5, H_k - 0.5) -- every operation rounded to float32 in this order.
 * out: d_inside[k] (int64) samples inside keyframe k, *d_valid (int64) samples
 *   with depth > 0; co-visibility = d_inside[k] / *d_valid.
 * err: INVALID_ARGUMENT for NULLs, step < 1, n_keyframes outside 1..256. */
fgs_status fgs_covisibility(const float *depth, const fgs_camera *cam, const fgs_camera *keyframes,
                            int32_t n_keyframes, int32_t step, int64_t *d_inside, int64_t *d_valid,
                            void *stream);

/* fgs_select_keyframes -- the keyframe window of Sec. III-C: keyframes whose
 * co-visibility d_inside[k] / *d_valid exceeds `threshold` (0.7 in the paper) are
 * co-visible; of the others, the round(frac * count) (frac 0.3 in the paper) with
 * the smallest draws u[k] (ties by index) are the random keyframes.  The draws are
 * an input (uniform numbers, one per keyframe, on the device).
 * out: d_kind[k] = 1 co-visible, 2 random, 0 not selected; *d_count selected.
 *   With *d_valid == 0 no keyframe is co-visible.
 * err: INVALID_ARGUMENT for NULLs, n_keyframes outside 1..1024. */
fgs_status fgs_select_keyframes(const int64_t *d_inside, const int64_t *d_valid, const float *u,
                                int32_t n_keyframes, float threshold, float frac, int32_t *d_kind,
                                int32_t *d_count, void *stream);

/* ---------------------------------------------------------------------------------
 * GICP tracking on the sparse map (Sec. III-B, eq12-eq14).  Point clouds are
 * float32 [capacity][3] arrays with a count that lives on the device; per-point
 * covariances are symmetric 3x3 stored as [capacity][6] (xx, xy, xz, yy, yz, zz).
 * A uniform grid indexes a cloud for neighbour search: its cell edge bounds every
 * neighbourhood radius used with it (covariance radius, correspondence distance),
 * so 27 cells around a point hold every candidate. */
typedef struct {
  float origin[3];  /* corner of cell (0, 0, 0)                                 */
  float cell;       /* cell edge (world units)                                  */
  int32_t dims[3];  /* cells per axis (product <= 2^26); points outside are skipped */
} fgs_grid;

/* fgs_depth_points -- the observed points of a depth map in camera coordinates:
 * pixels with x % step == 0, y % step == 0, depth d > 0 and, when mask is not NULL,
 * (mask & mask_bits) != 0, as (d (x - cx) / fx, d (y - cy) / fy, d) in pixel order,
 * each operation rounded to float32 in that order.
 * out: xyz[capacity][3], *d_n; FGS_DEV_MAP_FULL and a truncated cloud when more
 * points than capacity.  ws: fgs_depth_points_workspace_size(W, H, step). */
fgs_status fgs_depth_points(const float *depth, const uint8_t *mask, uint8_t mask_bits, const fgs_camera *cam,
                            int32_t step, float *xyz, int64_t capacity, int64_t *d_n, void *ws, size_t ws_bytes,
                            int32_t *d_status, void *stream);
size_t fgs_depth_points_workspace_size(int32_t width, int32_t height, int32_t step);

/* fgs_transform_points -- xyz_out = R xyz_in + t for [R | t] = pose (row-major 3x4,
 * double on the device), and covariances C_out = R C_in R^T when both pointers
 * are set; in place is allowed. */
fgs_status fgs_transform_points(const float *xyz_in, const float *cov_in, const int64_t *d_n, int64_t n_max,
                                const double *d_pose, float *xyz_out, float *cov_out, void *stream);

/* fgs_voxel_downsample -- uniform downsampling in 3D: of every occupied grid cell
 * the point with the lowest index, appended in index order to out (the sparse
 * map's addition of Sec. III-B).  Points outside the grid are dropped.
 * out: out_xyz[out_capacity][3] from index *d_n_out on (then *d_n_out grows);
 *   FGS_DEV_MAP_FULL when it would exceed out_capacity.
 * ws: fgs_voxel_workspace_size(grid, n_max). */
fgs_status fgs_voxel_downsample(const float *xyz, const int64_t *d_n, int64_t n_max, const fgs_grid *grid,
                                void *ws, size_t ws_bytes, float *out_xyz, int64_t out_capacity,
                                int64_t *d_n_out, int32_t *d_status, void *stream);
size_t fgs_voxel_workspace_size(const fgs_grid *grid, int64_t n_max);

/* fgs_grid_build -- cell index of a cloud: order[cell_start[c] .. cell_start[c+1])
 * are the points in cell c (any order within a cell).  cell_start has
 * cells + 1 entries; ws: fgs_grid_workspace_size(grid, n_max). */
fgs_status fgs_grid_build(const float *xyz, const int64_t *d_n, int64_t n_max, const fgs_grid *grid,
                          int32_t *cell_start, int32_t *order, void *ws, size_t ws_bytes, void *stream);
size_t fgs_grid_workspace_size(const fgs_grid *grid, int64_t n_max);

/* fgs_point_covariances -- GICP surface covariances: the neighbourhood of a point
 * is its (up to) k nearest points within the grid's cell edge, itself included,
 * ordered by (squared distance, index); C = (1/m) sum (x - mean)(x - mean)^T over
 * them; with eigenvectors v1..v3 of C by increasing eigenvalue the covariance is
 * regularised to eps v1 v1^T + v2 v2^T + v3 v3^T (a plane); fewer than 3
 * neighbours give the identity.  k in 3..32. */
fgs_status fgs_point_covariances(const float *xyz, const int64_t *d_n, int64_t n_max, const fgs_grid *grid,
                                 const int32_t *cell_start, const int32_t *order, int32_t k, float eps,
                                 float *cov, void *stream);

/* fgs_gicp -- eq14 by Gauss-Newton: minimises sum_i d_i^T (C_q + R C_p R^T)^-1 d_i
 * over T = [R | t], d_i = q_i - T p_i (eq12), q_i the nearest target point to T p_i
 * within max_dist (ties by index; pairs without one are left out).  Increment
 * xi = (w, v) of T <- (Rodrigues(w), v) T from the normal equations of the
 * linearisation d + [[T p]_x, -I] xi; correspondences are renewed every iteration;
 * it stops early when |xi| < 1e-6 (a micro-radian and micrometre step), and
 * keeps the pose when fewer than 6 pairs or a singular system remain.  d_pose
 * (double [12], row-major [R | t], the world-from-source pose) holds the initial
 * guess and receives the result.
 * d_stats (double [4]): cost and correspondences at the last evaluated pose, the
 * fraction of source points with a target point within overlap_dist there (the
 * keyframe test of Sec. III-C), iterations run.  ws: fgs_gicp_workspace_size(n_src_max). */
typedef struct {
  int32_t iterations;  /* at most this many Gauss-Newton steps                 */
  float max_dist;      /* correspondence distance (<= the target grid's cell)  */
  float overlap_dist;  /* overlap distance (<= the target grid's cell)         */
} fgs_gicp_params;
fgs_status fgs_gicp(const float *src_xyz, const float *src_cov, const int64_t *d_n_src, int64_t n_src_max,
                    const float *tgt_xyz, const float *tgt_cov, const fgs_grid *grid, const int32_t *cell_start,
                    const int32_t *order, const fgs_gicp_params *p, double *d_pose, double *d_stats, void *ws,
                    size_t ws_bytes, void *stream);
size_t fgs_gicp_workspace_size(int64_t n_src_max);

/* ---------------------------------------------------------------------------------
 * fgs_fourier_seed -- adaptive densification of Sec. III-A for one frame.
 *   gray = 0.299 R + 0.587 G + 0.114 B of rgb_gt; F = DFT2(gray) (eq2);
 *   centred (eq3, read as the standard spectrum shift); high-pass H = 1 -
 *   exp(-D^2 / (2 D0^2)) with D in Nyquist units (eq5, eq7); inverse DFT (eq8);
 *   E = |I_h|.  256-bin histogram of E / max E, triangle threshold t (a frame
 *   whose max E is at most 1e-5 of its peak |gray| has no high-frequency region);
 *   M_h = bin > t, M_l = not M_h.  Missing region (eq9):
 *   M_m = (A < tau_alpha) | (D/A - D_gt > tau_depth_rel D_gt) | (sum|C - C_gt| > 3 tau_color),
 *   all pixels when r_alpha is NULL.  Seeds (eq10): M_h & M_m on the m-grid and
 *   M_l & M_m on the n-grid (x % s == 0 && y % s == 0), valid depth only, high
 *   seeds first then low, row-major, at most max_new.  New Gaussians (eq11):
 *   back-projected from depth_gt, log-scale log(alpha_{h|l} d / f) on all axes
 *   (f = (fx + fy)/2), identity rotation, rgb of the frame, logit init_logit;
 *   when `prior` is not NULL the learned prior (fgs_prior_infer) sets the logit of
 *   every high-frequency seed, and its log-scales unless one axis is further than
 *   prior_max_dev from eq11's; low-frequency seeds keep eq11.
 * Appends at g->d_n ? *g->d_n : g->n and increments *g->d_n when set.
 * out: mask (uint8 per pixel: bit0 M_h, bit1 M_l, bit2 M_m, bit3 seeded),
 *   energy (E, nullable), *d_num_new, *d_threshold (bin t), appended Gaussians,
 *   seed_xy (nullable, [max_new][2] int32: pixel of the i-th appended Gaussian).
 * ws: fgs_fourier_seed_workspace_size(W, H, max_new) bytes, 256-byte aligned.
 * err: UNSUPPORTED when W or H has a prime factor above 17 (the FFT's radices). */
typedef struct {
  float d0;          /* high-pass cutoff in Nyquist units (0.25)       */
  int32_t m, n;      /* sampling spacing in high / low frequency areas */
  float alpha_h, alpha_l;
  float tau_alpha, tau_depth_rel, tau_color;
  int32_t max_new;
  float init_logit;
  float prior_max_dev; /* natural-log distance for the learned prior's fallback */
} fgs_seed_params;

typedef struct {
  /* BF16 weights (uint16 bit patterns), row-major [out][in], and FP32 biases. */
  const uint16_t *w1; /* [128][272] (input: 256 log-magnitudes, depth, 15 zeros) */
  const float *b1;    /* [128]                                                   */
  const uint16_t *w2; /* [128][128] */
  const float *b2;    /* [128]      */
  const uint16_t *w3; /* [8][128]  rows 4..7 zero */
  const float *b3;    /* [8]        rows 4..7 zero */
} fgs_mlp;

fgs_status fgs_fourier_seed(const float *rgb_gt, const float *depth_gt, const float *r_color,
                            const float *r_depth, const float *r_alpha,
                            const fgs_camera *cam, const fgs_seed_params *params,
                            const fgs_mlp *prior, uint8_t *mask, float *energy,
                            fgs_gaussians *g, int32_t *d_num_new, int32_t *d_threshold,
                            int32_t *seed_xy, void *ws, size_t ws_bytes, int32_t *d_status,
                            void *stream);
size_t fgs_fourier_seed_workspace_size(int32_t width, int32_t height, int32_t max_new);

/* fgs_fourier_seed in two calls, for a caller that overlaps the first with other
 * work on a second stream: the first needs only the frame, the second the render.
 * fgs_fourier_energy -- eq2-eq8 and the threshold: E (into energy, or into ws when
 *   energy is NULL), its histogram and the triangle threshold *d_threshold.
 * fgs_fourier_seed_from_energy -- the rest of fgs_fourier_seed (eq9-eq11, the
 *   prior), with the same arguments, reading E, the threshold and the maxima that
 *   fgs_fourier_energy left in `energy` (or ws), *d_threshold and ws.
 * The pair gives fgs_fourier_seed's outputs bit for bit when both calls get the
 * same cam size, params, energy, d_threshold and ws, and the second runs after the
 * first has completed (same stream, or an event between the streams); nothing
 * checks that, and in between neither ws nor energy may be used by another call.
 * Errors as fgs_fourier_seed. */
fgs_status fgs_fourier_energy(const float *rgb_gt, const fgs_camera *cam, const fgs_seed_params *params,
                              float *energy, int32_t *d_threshold, void *ws, size_t ws_bytes,
                              void *stream);
fgs_status fgs_fourier_seed_from_energy(const float *rgb_gt, const float *depth_gt,
                                        const float *r_color, const float *r_depth,
                                        const float *r_alpha, const fgs_camera *cam,
                                        const fgs_seed_params *params, const fgs_mlp *prior,
                                        uint8_t *mask, const float *energy, fgs_gaussians *g,
                                        int32_t *d_num_new, int32_t *d_threshold, int32_t *seed_xy,
                                        void *ws, size_t ws_bytes, int32_t *d_status, void *stream);

/* ---------------------------------------------------------------------------------
 * fgs_render_window -- a keyframe window (the co-visible and random keyframes the
 * map is optimised over, Sec. III-C/D) rendered (eq1), scored (eq16 without eq15)
 * and differentiated in one persistent cooperative launch: every CTA of a grid
 * that fits on the GPU at once claims (view, tile) items and loss tiles from atomic
 * counters in three phases -- blend, loss, adjoint -- separated by grid barriers,
 * so views of mixed resolution balance across the SMs.
 *   Inputs as fgs_render_fwd / fgs_loss / fgs_render_bwd for the view set (the
 *   projection and the sorted lists of all views, from fgs_project and
 *   fgs_bin_sort).  Outputs: the render (color, depth, alpha, t_final, n_contrib),
 *   dL/dC and dL/dD, the loss ADDED to *d_loss, and the splat gradients ADDED to
 *   grad2d [n_views][stride][8] and grads->rgb (the caller zeroes both); chain them
 *   to the Gaussians with fgs_project_bwd.
 *   ws: fgs_render_window_workspace_size(cams, n_views) bytes, 256-byte aligned.
 *   tile_order: NULL or a permutation of the view set's tiles (fgs_tile_order of
 *   an earlier window's n_contrib): the blend and adjoint phases claim their
 *   (view, tile) items in that order, heaviest first; as for fgs_render_fwd, an
 *   entry outside the tiles is skipped and or-es FGS_DEV_BAD_ORDER into *d_status.
 *   Device errors: every barrier wait is bounded (2 s); a CTA that gives up sets
 *   FGS_DEV_TIMEOUT and returns, and the outputs are then invalid.
 *   err: UNSUPPORTED when the kernel cannot be made co-resident. */
fgs_status fgs_render_window(const fgs_gaussians *g, const fgs_projected *proj,
                             const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                             const int32_t *ids, const int32_t *tile_ranges,
                             const int32_t *tile_order, const float *color_gt, const float *depth_gt,
                             const fgs_loss_params *lp, float *color, float *depth, float *alpha,
                             float *t_final, int32_t *n_contrib, float *dL_dcolor,
                             float *dL_ddepth, float *grad2d, fgs_gaussians *grads, float *d_loss,
                             void *ws, size_t ws_bytes, int32_t *d_status, void *stream);
size_t fgs_render_window_workspace_size(const fgs_camera *cams, int32_t n_views);

/* fgs_autotune -- picks the tiling of the keyframe window above (the window of
 * Sec. III-C; the paper gives no kernel design, so the tile shape and batch depth
 * are measured rather than fixed): every supported tiling -- 8x8, 16x16 and 16x32
 * tiles (w x h) times batch depths 32, 64, 128, 256, FGS_AUTOTUNE_CONFIGS in the
 * order 8x8/32, 8x8/64, ..., 16x32/256 -- runs fgs_project, fgs_bin_sort,
 * fgs_render_window (in the heaviest-first tile order of the previous pass),
 * fgs_tile_order and fgs_project_bwd on the caller's map g, views cams and
 * targets (color_gt, depth_gt as for fgs_render_window, weights `loss`), once
 * untimed and `reps` times timed with CUDA events; the fastest is written to
 * *best and, when ms_out (host, FGS_AUTOTUNE_CONFIGS floats) is not NULL, the
 * milliseconds per pass of every tiling (FLT_MAX for a tiling whose pass set a
 * device status bit, e.g. more pairs than pair_capacity).
 *   g is only read (its gradients and every intermediate go to ws).
 *   ws: fgs_autotune_workspace_size(g, cams, n_views, pair_capacity) bytes,
 *   256-byte aligned, caller-owned.
 *   Unlike the other entry points this call synchronises the host with `stream`
 *   (it reads its timings back) and cannot be captured in a CUDA graph.
 * err: INVALID_ARGUMENT (bad views, NULLs, small workspace, reps outside
 *   1..1000), CAPACITY when every tiling overflowed, CUDA. */
#define FGS_AUTOTUNE_CONFIGS 12
fgs_status fgs_autotune(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views,
                        const float *color_gt, const float *depth_gt, const fgs_loss_params *loss,
                        int64_t pair_capacity, int32_t reps, void *ws, size_t ws_bytes,
                        fgs_tiling *best, float *ms_out, void *stream);
size_t fgs_autotune_workspace_size(const fgs_gaussians *g, const fgs_camera *cams,
                                   int32_t n_views, int64_t pair_capacity);

/* ---------------------------------------------------------------------------------
 * Learned seeding prior (not in the paper; an extension).  Features per seed
 * pixel (x, y): the 16x16 grayscale patch with top-left (x-8, y-8), clamped to the
 * image, its 2D DFT magnitude as log(1 + |F|) in natural frequency order (256),
 * then the depth, then 15 zeros -> BF16 row of 272.  MLP 272 -> 128 -> 128 -> 4,
 * GELU (erf form), BF16 operands, FP32 accumulation, activations rounded to BF16
 * before each product.  Output: log-scale x, y, z and opacity logit.
 *
 * fgs_prior_features: rgb [3][H][W] (gray = BT.601 luma), depth [H][W],
 *   seed_xy [n][2] int32 -> features [n][272] BF16.
 * fgs_prior_infer: features -> out [n][4] float, on the fifth-generation tensor
 *   cores: a persistent grid walks 128-row tiles; the three layers run as
 *   tcgen05.mma chains (M = 128; N = 128, 128, 16; K = 272, 128, 128) with the
 *   weights resident in shared memory and FP32 accumulators in tensor memory; the
 *   bias, GELU and BF16 rounding are applied when the accumulator is read back.
 *   features and out must be 16-byte aligned.  d_status (may be NULL): a tensor-core
 *   completion wait that gives up or-es FGS_DEV_TIMEOUT into it and the rows of
 *   that tile are left unwritten. */
#define FGS_PRIOR_IN 272
#define FGS_PRIOR_HID 128
#define FGS_PRIOR_OUT 4
fgs_status fgs_prior_features(const float *rgb, const float *depth, int32_t width,
                              int32_t height, const int32_t *seed_xy, int64_t n,
                              uint16_t *features, void *stream);
fgs_status fgs_prior_infer(const fgs_mlp *mlp, const uint16_t *features, int64_t n,
                           float *out, int32_t *d_status, void *stream);

/* fgs_prior_train -- one Adam step of the prior on a batch: mean squared error
 * over the batch's n x 4 outputs against `targets`, gradients through the MLP,
 * Adam on the FP32 master weights, BF16 copies refreshed.  *d_loss receives the
 * batch loss (before the step), ADDED.  After the call the first
 * fgs_prior_num_params() floats of ws hold the batch gradient in packed order
 * (w1 [128][272], b1, w2 [128][128], b2, w3 [8][128], b3 [8]); the Adam moments
 * in master->m / master->v use the same order. */
typedef struct {
  float *w1, *b1, *w2, *b2, *w3, *b3; /* FP32 masters, same shapes as fgs_mlp */
  float *m;                           /* Adam first moments, all params packed */
  float *v;                           /* Adam second moments                    */
} fgs_mlp_master;
typedef struct {
  float lr, beta1, beta2, eps;
  int32_t step; /* t >= 1 */
} fgs_train_params;
fgs_status fgs_prior_train(fgs_mlp *mlp_bf16_out, fgs_mlp_master *master,
                           const uint16_t *features, const float *targets, int64_t n,
                           const fgs_train_params *hp, float *d_loss, void *ws,
                           size_t ws_bytes, void *stream);
size_t fgs_prior_train_workspace_size(int64_t n);
int64_t fgs_prior_num_params(void);

/* ---------------------------------------------------------------------------------
 * Auxiliary. */
const char *fgs_last_error(void);
int32_t fgs_version(void);
/* Kernel launches issued by this library in this process (host counter). */
int64_t fgs_launch_count(void);
/* cudaMemsetAsync of `bytes` bytes at device pointer dst on the stream (used to
 * clear gradient planes and loss accumulators between mapping iterations). */
fgs_status fgs_memset_async(void *dst, int32_t value, size_t bytes, void *stream);
/* cudaMemcpyAsync of `bytes` bytes (any direction the pointers imply) on the stream. */
fgs_status fgs_memcpy_async(void *dst, const void *src, size_t bytes, void *stream);

/* Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount). */
int32_t fgs_num_sms(void);

/* fgs_peak_probe -- one launch of a microbenchmark of an on-chip rate that bounds
 * the blend kernels (measurement infrastructure; the paper has none): kind
 * FGS_PEAK_FFMA runs FP32 fused multiply-adds, FGS_PEAK_EX2 the ex2.approx MUFU
 * instruction, FGS_PEAK_LDS 16-byte shared-memory loads, each as 16 independent
 * chains per thread in fgs_num_sms() * blocks_per_sm blocks of 256 threads for
 * `iters` rounds.  *ops (host) receives the operation count of the launch:
 * floating-point operations (2 per FMA), ex2 evaluations, or bytes loaded.  The
 * caller times the launch on `stream` (CUDA events) and divides.  sink: a device
 * float per block that the kernels never write in practice (it keeps their
 * results live).  blocks_per_sm 1..32, iters 1..2^32. */
enum { FGS_PEAK_FFMA = 0, FGS_PEAK_EX2 = 1, FGS_PEAK_LDS = 2 };
fgs_status fgs_peak_probe(int32_t kind, int32_t blocks_per_sm, int64_t iters, float *sink,
                          int64_t *ops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FGS_H */
