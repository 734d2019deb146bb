// render.cu -- eq1 alpha blending (colour, depth and opacity readings) per tile,
// and its reverse-order adjoint.
//
// One CTA per (view, tile), one thread per pixel.  The tile's depth-ordered list
// is walked in batches of BATCH splats: each batch is gathered by id from the
// splat records (two float4 loads plus three colour planes per splat) into
// shared memory once and then evaluated by every pixel of the tile.  The walk
// stops when every pixel of the tile is saturated (T < 1e-4).
//
// The backward walks the same lists back to front from the tile's largest
// contributor count, recovering each pixel's transmittance by division by
// (1 - alpha) (alpha <= 0.99) instead of storing it.  Per-splat gradients are
// reduced across the warp with shuffles, accumulated per batch in shared memory
// and flushed with one global atomic per (CTA, splat, field).
#include "common.cuh"

namespace fgs {

struct RenderArgs {
  DevViews vs;
  const float4 *splat;  // [V][stride][2]
  int64_t stride;
  const float *rgb;     // [3][cap]
  int64_t cap;
  const int32_t *ids;
  const int2 *ranges;
  float *color, *depth, *alpha, *t_final;
  int32_t *n_contrib;
};

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW *TH) k_render_fwd(RenderArgs a) {
  constexpr int NT = TW * TH;
  __shared__ float4 s_g0[BATCH];  // mean2d x, y, conic a, b
  __shared__ float4 s_g1[BATCH];  // conic c, opacity, depth, -
  __shared__ float4 s_rgb[BATCH];
  const int t = blockIdx.x;
  const int v = view_of_tile(a.vs, t);
  const DevCam &cm = a.vs.cam[v];
  const int lt = t - cm.tile_base;
  const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
  const int px = tx * TW + (threadIdx.x % TW), py = ty * TH + (threadIdx.x / TW);
  const bool inside = px < cm.W && py < cm.H;
  const float fpx = (float)px, fpy = (float)py;
  const int2 range = a.ranges[t];
  const int n = range.y - range.x;
  const float4 *sp = a.splat + 2 * (int64_t)v * a.stride;
  bool done = !inside;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, A = 0.f;
  int last = 0;
  for (int base = 0; base < n; base += BATCH) {
    if (__syncthreads_count(done) == NT) break;
    for (int j = threadIdx.x; j < BATCH; j += NT) {
      if (base + j < n) {
        const int id = a.ids[range.x + base + j];
        s_g0[j] = sp[2 * (int64_t)id];
        s_g1[j] = sp[2 * (int64_t)id + 1];
        s_rgb[j] = make_float4(a.rgb[id], a.rgb[a.cap + id], a.rgb[2 * a.cap + id], 0.f);
      }
    }
    __syncthreads();
    if (!done) {
      const int cnt = min(BATCH, n - base);
      for (int k = 0; k < cnt; ++k) {
        const float4 g0 = s_g0[k], g1 = s_g1[k];
        float dx, dy;
        const float power = splat_power(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, fpy, dx, dy);
        if (power > 0.f) continue;
        const float alpha = fminf(kAlphaMax, __fmul_rn(g1.y, __expf(power)));
        if (alpha < kAlphaMin) continue;
        const float Tn = T * (1.f - alpha);
        if (Tn < kTMin) {
          done = true;
          break;
        }
        const float w = alpha * T;
        const float4 c = s_rgb[k];
        C0 += c.x * w;
        C1 += c.y * w;
        C2 += c.z * w;
        D += g1.z * w;
        A += w;
        T = Tn;
        last = base + k + 1;
      }
    }
  }
  if (inside) {
    const int64_t HW = (int64_t)cm.W * cm.H;
    const int64_t pix = (int64_t)py * cm.W + px;
    float *col = a.color + 3 * cm.pix_base;
    col[pix] = C0;
    col[HW + pix] = C1;
    col[2 * HW + pix] = C2;
    a.depth[cm.pix_base + pix] = D;
    a.alpha[cm.pix_base + pix] = A;
    a.t_final[cm.pix_base + pix] = T;
    a.n_contrib[cm.pix_base + pix] = last;
  }
}

struct RenderBwdArgs {
  DevViews vs;
  const float4 *splat;
  int64_t stride;
  const float *rgb;
  int64_t cap;
  const int32_t *ids;
  const int2 *ranges;
  const float *t_final;
  const int32_t *n_contrib;
  const float *dC, *dD, *dA;
  float *grad2d;     // [V][stride][8]
  float *grad_rgb;   // [3][cap]
};

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW *TH) k_render_bwd(RenderBwdArgs a) {
  constexpr int NT = TW * TH;
  constexpr int NF = 10;  // mean2d x, y, conic a, b, c, opacity, depth, r, g, b
  __shared__ float4 s_g0[BATCH];
  __shared__ float4 s_g1[BATCH];
  __shared__ float4 s_rgb[BATCH];
  __shared__ int s_id[BATCH];
  __shared__ float s_acc[BATCH][NF];
  __shared__ int s_max_last;
  const int t = blockIdx.x;
  const int v = view_of_tile(a.vs, t);
  const DevCam &cm = a.vs.cam[v];
  const int lt = t - cm.tile_base;
  const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
  const int px = tx * TW + (threadIdx.x % TW), py = ty * TH + (threadIdx.x / TW);
  const bool inside = px < cm.W && py < cm.H;
  const float fpx = (float)px, fpy = (float)py;
  const int2 range = a.ranges[t];
  const float4 *sp = a.splat + 2 * (int64_t)v * a.stride;
  const int64_t HW = (int64_t)cm.W * cm.H;
  const int64_t pix = (int64_t)py * cm.W + px;
  float T = 1.f;
  int last = 0;
  float g_c0 = 0.f, g_c1 = 0.f, g_c2 = 0.f, g_d = 0.f, g_a = 0.f;
  if (inside) {
    T = a.t_final[cm.pix_base + pix];
    last = a.n_contrib[cm.pix_base + pix];
    const float *dc = a.dC + 3 * cm.pix_base;
    g_c0 = dc[pix];
    g_c1 = dc[HW + pix];
    g_c2 = dc[2 * HW + pix];
    if (a.dD) g_d = a.dD[cm.pix_base + pix];
    if (a.dA) g_a = a.dA[cm.pix_base + pix];
  }
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  {
    int m = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&s_max_last, m);
  }
  __syncthreads();
  const int max_last = s_max_last;
  // suffix sums of gamma alpha T behind the current splat: r, g, b, depth, 1
  float S0 = 0.f, S1 = 0.f, S2 = 0.f, Sd = 0.f, Sa = 0.f;
  const int lane = threadIdx.x & 31;
  for (int end = max_last; end > 0; end -= BATCH) {
    const int start = max(0, end - BATCH);
    const int cnt = end - start;
    for (int j = threadIdx.x; j < BATCH; j += NT) {
      if (j < cnt) {
        const int id = a.ids[range.x + start + j];
        s_id[j] = id;
        s_g0[j] = sp[2 * (int64_t)id];
        s_g1[j] = sp[2 * (int64_t)id + 1];
        s_rgb[j] = make_float4(a.rgb[id], a.rgb[a.cap + id], a.rgb[2 * a.cap + id], 0.f);
      }
    }
    for (int e = threadIdx.x; e < BATCH * NF; e += NT) (&s_acc[0][0])[e] = 0.f;
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      const int j = start + k;
      float gr[NF];
      bool contrib = false;
      if (j < last) {
        const float4 g0 = s_g0[k], g1 = s_g1[k];
        float dx, dy;
        const float power = splat_power(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, fpy, dx, dy);
        if (power <= 0.f) {
          const float G = __expf(power);
          const float raw = __fmul_rn(g1.y, G);
          const float alpha = fminf(kAlphaMax, raw);
          if (alpha >= kAlphaMin) {
            contrib = true;
            const float om = 1.f - alpha;
            T = T / om;  // transmittance in front of this splat
            const float w = alpha * T;
            const float4 c = s_rgb[k];
            const float dot_gam = g_c0 * c.x + g_c1 * c.y + g_c2 * c.z + g_d * g1.z + g_a;
            const float dot_S = g_c0 * S0 + g_c1 * S1 + g_c2 * S2 + g_d * Sd + g_a * Sa;
            const float dalpha = T * dot_gam - dot_S / om;
            S0 += c.x * w;
            S1 += c.y * w;
            S2 += c.z * w;
            Sd += g1.z * w;
            Sa += w;
            gr[7] = g_c0 * w;
            gr[8] = g_c1 * w;
            gr[9] = g_c2 * w;
            gr[6] = g_d * w;
            if (raw < kAlphaMax) {
              const float dp = dalpha * alpha;  // d alpha / d power = alpha (unclamped)
              gr[0] = -dp * (g0.z * dx + g0.w * dy);
              gr[1] = -dp * (g0.w * dx + g1.x * dy);
              gr[2] = -0.5f * dp * dx * dx;
              gr[3] = -dp * dx * dy;
              gr[4] = -0.5f * dp * dy * dy;
              gr[5] = dalpha * G;
            } else {
              gr[0] = gr[1] = gr[2] = gr[3] = gr[4] = gr[5] = 0.f;
            }
          }
        }
      }
      const unsigned any = __ballot_sync(0xffffffffu, contrib);
      if (any) {
        if (!contrib) {
#pragma unroll
          for (int f = 0; f < NF; ++f) gr[f] = 0.f;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          float x = gr[f];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
          gr[f] = x;
        }
        if (lane < NF) {
          float mine = gr[0];
#pragma unroll
          for (int f = 1; f < NF; ++f) mine = lane == f ? gr[f] : mine;
          atomicAdd(&s_acc[k][lane], mine);
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * NF; e += NT) {
      const int k = e / NF, f = e - k * NF;
      const float val = s_acc[k][f];
      if (val != 0.f) {
        const int id = s_id[k];
        if (f < 7)
          atomicAdd(a.grad2d + 8 * ((int64_t)v * a.stride + id) + f, val);
        else
          atomicAdd(a.grad_rgb + (int64_t)(f - 7) * a.cap + id, val);
      }
    }
    __syncthreads();
  }
}

template <int TW, int TH, int BATCH>
static void launch_fwd(const RenderArgs &a, int blocks, cudaStream_t st) {
  k_render_fwd<TW, TH, BATCH><<<blocks, TW * TH, 0, st>>>(a);
}
template <int TW, int TH, int BATCH>
static void launch_bwd(const RenderBwdArgs &a, int blocks, cudaStream_t st) {
  k_render_bwd<TW, TH, BATCH><<<blocks, TW * TH, 0, st>>>(a);
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
                                     const int32_t *ids, const int32_t *tile_ranges, float *color,
                                     float *depth, float *alpha, float *t_final, int32_t *n_contrib,
                                     int32_t *d_status, void *stream) {
  (void)d_status;
  FGS_CHECK_ARG(proj && proj->splat, "fgs_render_fwd: NULL projection");
  if (!gaussians_ok(g, "g")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_render_fwd: unsupported tiling");
  FGS_CHECK_ARG(ids && tile_ranges && color && depth && alpha && t_final && n_contrib,
                "fgs_render_fwd: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(proj->splat) & 15) == 0, "fgs_render_fwd: splat alignment");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  RenderArgs a{vs, reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity, ids,
               reinterpret_cast<const int2 *>(tile_ranges), color, depth, alpha, t_final, n_contrib};
  FGS_DISPATCH_TILING(tiling, launch_fwd, a, vs.total_tiles, as_stream(stream));
  count_launch();
  FGS_CHECK_LAUNCH("fgs_render_fwd");
  return FGS_OK;
}

static fgs_status render_bwd_splats(const fgs_gaussians *g, const fgs_projected *proj, const DevViews &vs,
                                    fgs_tiling tiling, const int32_t *ids, const int32_t *tile_ranges,
                                    const float *t_final, const int32_t *n_contrib, const float *dL_dcolor,
                                    const float *dL_ddepth, const float *dL_dalpha, float *grad2d,
                                    fgs_gaussians *grads, cudaStream_t st) {
  RenderBwdArgs a{vs,      reinterpret_cast<const float4 *>(proj->splat), proj->stride, g->rgb, g->capacity,
                  ids,     reinterpret_cast<const int2 *>(tile_ranges), t_final, n_contrib, dL_dcolor,
                  dL_ddepth, dL_dalpha, grad2d, grads->rgb};
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
                                            const float *t_final, const int32_t *n_contrib,
                                            const float *dL_dcolor, const float *dL_ddepth,
                                            const float *dL_dalpha, float *grad2d, fgs_gaussians *grads,
                                            int32_t *d_status, void *stream) {
  (void)d_status;
  fgs_status s = check_bwd_args(g, proj, tiling, ids, tile_ranges, t_final, n_contrib, dL_dcolor, grad2d, grads);
  if (s != FGS_OK) return s;
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  return render_bwd_splats(g, proj, vs, tiling, ids, tile_ranges, t_final, n_contrib, dL_dcolor, dL_ddepth,
                           dL_dalpha, grad2d, grads, as_stream(stream));
}

extern "C" fgs_status fgs_render_bwd(const fgs_gaussians *g, const fgs_projected *proj,
                                     const fgs_camera *cams, int32_t n_views, fgs_tiling tiling,
                                     const int32_t *ids, const int32_t *tile_ranges,
                                     const float *t_final, const int32_t *n_contrib,
                                     const float *dL_dcolor, const float *dL_ddepth,
                                     const float *dL_dalpha, float *grad2d, fgs_gaussians *grads,
                                     int32_t *d_status, void *stream) {
  (void)d_status;
  fgs_status s = check_bwd_args(g, proj, tiling, ids, tile_ranges, t_final, n_contrib, dL_dcolor, grad2d, grads);
  if (s != FGS_OK) return s;
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = as_stream(stream);
  FGS_CUDA(cudaMemsetAsync(grad2d, 0, sizeof(float) * 8 * (size_t)n_views * (size_t)proj->stride, st),
           "memset grad2d");
  s = render_bwd_splats(g, proj, vs, tiling, ids, tile_ranges, t_final, n_contrib, dL_dcolor, dL_ddepth, dL_dalpha,
                        grad2d, grads, st);
  if (s != FGS_OK) return s;
  return launch_project_bwd(g, vs, proj->radius, grad2d, proj->stride, grads, st);
}
