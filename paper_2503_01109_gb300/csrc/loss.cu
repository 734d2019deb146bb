// loss.cu -- the mapping loss of eq16 (L1 colour, L1 depth, 1 - SSIM), the scale
// regulariser of eq15, and the Adam step of the map optimisation (Sec. III-D).
//
// The loss kernel runs one fused tile pass (loss_tile.cuh) per 32x32 output tile.
// Loss values are reduced per CTA into a workspace and summed in a fixed order by
// one CTA, so the value is reproducible bit for bit.
#include <cmath>
#include <mutex>

#include "loss_tile.cuh"

namespace fgs {

constexpr int kLT = 32;          // loss tile side
constexpr int kLThreads = 384;   // 12 warps: one pass of each 11-tap stage covers the tile
constexpr size_t kLossSmem = sizeof(float) * LossGeom<kLT>::SmemFloats;  // 88 KB: two CTAs per SM

__global__ void __launch_bounds__(kLThreads, 2) k_loss(LossArgs a) {
  pdl_enter();
  extern __shared__ float sm[];
  loss_tile<kLT>(a, blockIdx.x, sm);
}

// Raises k_loss's dynamic shared-memory limit (a host-side attribute of the
// current device's context; set on every call so that a new context gets it too).
static fgs_status loss_smem_attr() {
  FGS_CUDA(cudaFuncSetAttribute(k_loss, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLossSmem),
           "fgs_loss: shared-memory attribute");
  return FGS_OK;
}

// Sums `count` partials in a fixed order and adds the total to *d_loss.
__global__ void k_reduce_partials(const double *__restrict__ partials, int64_t count, float *d_loss) {
  pdl_enter();
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

// `who` names the entry point in the error message.
static bool loss_views(const fgs_camera *cams, int32_t n_views, LossViews *lv, int *blocks,
                       const char *who = "fgs_loss") {
  if (!cams || n_views < 1 || n_views > FGS_MAX_VIEWS) {
    set_error("%s: n_views must be 1..%d", who, FGS_MAX_VIEWS);
    return false;
  }
  lv->n = n_views;
  int tiles = 0;
  int64_t pix = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width <= 0 || cams[v].height <= 0) {
      set_error("%s: bad image size", who);
      return false;
    }
    lv->v[v].W = cams[v].width;
    lv->v[v].H = cams[v].height;
    lv->v[v].tiles_x = (cams[v].width + kLT - 1) / kLT;
    lv->v[v].tile_base = tiles;
    lv->v[v].pix_base = pix;
    tiles += lv->v[v].tiles_x * ((cams[v].height + kLT - 1) / kLT);
    pix += (int64_t)cams[v].width * cams[v].height;
  }
  *blocks = tiles;
  return true;
}

// ---------------------------------------------------------------------------------
// eq15: per Gaussian |s1 - m| + |s2 - m| + |s3|, m = (s1 + s2)/2, s = exp(log-scale),
// mean over the live Gaussians, times weight.
__global__ void k_scale_reg(const float *__restrict__ ls, int64_t cap, int64_t n, const int64_t *d_n,
                            float weight, float *__restrict__ gls, double *__restrict__ partials) {
  pdl_enter();
  __shared__ double red[8];
  const int64_t live = live_count(d_n, n);
  const float wn = live > 0 ? weight / (float)live : 0.f;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float val = 0.f;
  if (i < live) {
    const float s1 = expf(ls[i]), s2 = expf(ls[cap + i]), s3 = expf(ls[2 * cap + i]);
    const float m = 0.5f * (s1 + s2);
    val = fabsf(s1 - m) + fabsf(s2 - m) + fabsf(s3);
    const float g1 = 0.5f * sgnf(s1 - m) - 0.5f * sgnf(s2 - m);
    const float g2 = 0.5f * sgnf(s2 - m) - 0.5f * sgnf(s1 - m);
    gls[i] += wn * g1 * s1;
    gls[cap + i] += wn * g2 * s2;
    gls[2 * cap + i] += wn * (s3 > 0.f ? 1.f : 0.f) * s3;
  }
  float s = val * wn;  // warp sums in FP32, block and grid sums in FP64
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------------
// Adam over the 14 parameter planes: blockIdx.y selects the plane.
struct AdamPlanes {
  float *p[14];
  float *g[14];
  float *m[14];
  float *v[14];
  float lr[14];
};

// Adam's bias corrections at step t as reciprocals: 1 / (1 - beta1^t), 1 / (1 - beta2^t).
__device__ __forceinline__ float2 adam_bias(float b1, float b2, int t) {
  return make_float2(1.f / (1.f - powf(b1, (float)t)), 1.f / (1.f - powf(b2, (float)t)));
}

// One bias-corrected Adam step of one parameter (r = adam_bias(b1, b2, t)).  The
// square root and the quotient use the hardware approximations (a few ulp): the
// step is a heuristic whose size needs no correctly rounded arithmetic, and the
// IEEE sequences made the optimiser instruction-bound.
__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float b1, float b2, float eps,
                                         float lr, float2 r) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  const float vh = v * r.y;
  const float den = (vh > 0.f ? vh * rsqrtf(vh) : 0.f) + eps;
  p -= __fdividef(lr * (m * r.x), den);
}

__global__ void k_adam_step_incr(int32_t *d_step) { pdl_enter(); *d_step += 1; }

// VEC: four consecutive elements per thread with 16-byte loads (every plane
// 16-byte aligned); else one element per thread.
// Planes from zero_from on have their gradient cleared after it is read.
template <bool VEC>
__global__ void k_adam(AdamPlanes P, int64_t n, const int64_t *d_n, float b1, float b2, float eps, int32_t step,
                       const int32_t *d_step, int zero_from) {
  pdl_enter();
  const int plane = blockIdx.y;
  const int64_t live = live_count(d_n, n);
  const int t = d_step ? *d_step : step;
  const float2 r = adam_bias(b1, b2, t);
  const float lr = P.lr[plane];
  float *__restrict__ p = P.p[plane];
  float *__restrict__ g = P.g[plane];
  const bool zero = plane >= zero_from;
  float *__restrict__ m = P.m[plane];
  float *__restrict__ v = P.v[plane];
  const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * (VEC ? 4 : 1);
  if (i0 >= live) return;
  if (VEC && i0 + 4 <= live) {
    float4 pp = *reinterpret_cast<const float4 *>(p + i0), gg = *reinterpret_cast<const float4 *>(g + i0);
    float4 mm = *reinterpret_cast<const float4 *>(m + i0), vv = *reinterpret_cast<const float4 *>(v + i0);
    adam_one(pp.x, gg.x, mm.x, vv.x, b1, b2, eps, lr, r);
    adam_one(pp.y, gg.y, mm.y, vv.y, b1, b2, eps, lr, r);
    adam_one(pp.z, gg.z, mm.z, vv.z, b1, b2, eps, lr, r);
    adam_one(pp.w, gg.w, mm.w, vv.w, b1, b2, eps, lr, r);
    *reinterpret_cast<float4 *>(p + i0) = pp;
    *reinterpret_cast<float4 *>(m + i0) = mm;
    *reinterpret_cast<float4 *>(v + i0) = vv;
    if (zero) *reinterpret_cast<float4 *>(g + i0) = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int64_t i1 = VEC ? min(i0 + 4, live) : i0 + 1;
  for (int64_t i = i0; i < i1; ++i) {
    float pi = p[i], mi = m[i], vi = v[i];
    adam_one(pi, g[i], mi, vi, b1, b2, eps, lr, r);
    p[i] = pi;
    m[i] = mi;
    v[i] = vi;
    if (zero) g[i] = 0.f;
  }
}

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_loss_workspace_size(const fgs_camera *cams, int32_t n_views) {
  LossViews lv;
  int blocks = 0;
  if (!loss_views(cams, n_views, &lv, &blocks)) return 0;
  return align_up(sizeof(double) * (size_t)blocks);
}

extern "C" fgs_status fgs_loss(const fgs_camera *cams, int32_t n_views, const float *color, const float *depth,
                               const float *color_gt, const float *depth_gt, const fgs_loss_params *params,
                               float *dL_dcolor, float *dL_ddepth, float *d_loss, void *ws, size_t ws_bytes,
                               void *stream) {
  FGS_CHECK_ARG(color && depth && color_gt && depth_gt && params && dL_dcolor && dL_ddepth && d_loss,
                "fgs_loss: NULL argument");
  LossArgs a;
  int blocks = 0;
  if (!loss_views(cams, n_views, &a.lv, &blocks)) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(ws && ws_bytes >= sizeof(double) * (size_t)blocks, "fgs_loss: workspace too small");
  a.color = color;
  a.depth = depth;
  a.color_gt = color_gt;
  a.depth_gt = depth_gt;
  a.w_c = params->w_l1_color;
  a.w_d = params->w_l1_depth;
  a.w_s = params->w_ssim;
  a.dC = dL_dcolor;
  a.dD = dL_ddepth;
  a.partials = static_cast<double *>(ws);
  double g[11], gs = 0.0;
  for (int i = 0; i < 11; ++i) {
    g[i] = std::exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
    gs += g[i];
  }
  for (int i = 0; i < 11; ++i) a.g[i] = (float)(g[i] / gs);
  const fgs_status sa = loss_smem_attr();
  if (sa != FGS_OK) return sa;
  cudaStream_t st = as_stream(stream);
  pdl_launch(k_loss, blocks, kLThreads, kLossSmem, st, a);
  pdl_launch(k_reduce_partials, 1, 256, 0, st, a.partials, blocks, d_loss);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_loss");
  return FGS_OK;
}

extern "C" size_t fgs_scale_reg_workspace_size(int64_t n) {
  return align_up(sizeof(double) * (size_t)std::max<int64_t>((n + 255) / 256, 1));
}

extern "C" fgs_status fgs_scale_reg(const fgs_gaussians *g, float weight, fgs_gaussians *grads, float *d_loss,
                                    void *ws, size_t ws_bytes, void *stream) {
  if (!gaussians_ok(g, "g") || !gaussians_ok(grads, "grads")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(d_loss && ws && ws_bytes >= fgs_scale_reg_workspace_size(g->n), "fgs_scale_reg: workspace");
  if (g->n == 0) return FGS_OK;
  const int64_t blocks = (g->n + 255) / 256;
  cudaStream_t st = as_stream(stream);
  pdl_launch(k_scale_reg, (unsigned)blocks, 256, 0, st, g->log_scales, g->capacity, g->n, g->d_n, weight,
             grads->log_scales, static_cast<double *>(ws));
  pdl_launch(k_reduce_partials, 1, 256, 0, st, static_cast<double *>(ws), blocks, d_loss);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_scale_reg");
  return FGS_OK;
}

namespace fgs {
void launch_reduce_partials(const double *partials, int64_t count, float *d_loss, cudaStream_t st) {
  pdl_launch(k_reduce_partials, 1, 256, 0, st, partials, count, d_loss);
}

fgs_status launch_adam(fgs_gaussians *params, fgs_gaussians *grads, fgs_gaussians *m, fgs_gaussians *v,
                       const fgs_adam_params *hp, int32_t *d_step, int zero_from, cudaStream_t st) {
  if (params->n == 0) return FGS_OK;
  AdamPlanes P;
  auto fill = [&](int base, int cnt, float *pp, float *gp, float *mp, float *vp, int64_t pc, int64_t gc, int64_t mc,
                  int64_t vc, float lr) {
    for (int k = 0; k < cnt; ++k) {
      P.p[base + k] = pp + k * pc;
      P.g[base + k] = gp + k * gc;
      P.m[base + k] = mp + k * mc;
      P.v[base + k] = vp + k * vc;
      P.lr[base + k] = lr;
    }
  };
  const int64_t pc = params->capacity, gc = grads->capacity, mc = m->capacity, vc = v->capacity;
  fill(0, 3, params->means, grads->means, m->means, v->means, pc, gc, mc, vc, hp->lr[0]);
  fill(3, 3, params->log_scales, grads->log_scales, m->log_scales, v->log_scales, pc, gc, mc, vc, hp->lr[1]);
  fill(6, 4, params->quats, grads->quats, m->quats, v->quats, pc, gc, mc, vc, hp->lr[2]);
  fill(10, 1, params->opacity_logits, grads->opacity_logits, m->opacity_logits, v->opacity_logits, pc, gc, mc, vc,
       hp->lr[3]);
  fill(11, 3, params->rgb, grads->rgb, m->rgb, v->rgb, pc, gc, mc, vc, hp->lr[4]);
  if (d_step) {
    pdl_launch(k_adam_step_incr, 1, 1, 0, st, d_step);
    count_launch();
  }
  bool aligned = true;
  for (int k = 0; k < 14; ++k)
    aligned = aligned && ((reinterpret_cast<uintptr_t>(P.p[k]) | reinterpret_cast<uintptr_t>(P.g[k]) |
                           reinterpret_cast<uintptr_t>(P.m[k]) | reinterpret_cast<uintptr_t>(P.v[k])) & 15) == 0;
  const int64_t per_block = aligned ? 1024 : 256;
  const unsigned bx = (unsigned)std::max<int64_t>(1, (params->n + per_block - 1) / per_block);
  if (aligned)
    pdl_launch(k_adam<true>, dim3(bx, 14), 256, 0, st, P, params->n, params->d_n, hp->beta1, hp->beta2, hp->eps,
               hp->step, d_step, zero_from);
  else
    pdl_launch(k_adam<false>, dim3(bx, 14), 256, 0, st, P, params->n, params->d_n, hp->beta1, hp->beta2, hp->eps,
               hp->step, d_step, zero_from);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_adam");
  return FGS_OK;
}
}  // namespace fgs

extern "C" fgs_status fgs_adam(fgs_gaussians *params, const fgs_gaussians *grads, fgs_gaussians *m,
                               fgs_gaussians *v, const fgs_adam_params *hp, int32_t *d_step, void *stream) {
  if (!gaussians_ok(params, "params") || !gaussians_ok(grads, "grads") || !gaussians_ok(m, "m") ||
      !gaussians_ok(v, "v"))
    return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(hp, "fgs_adam: NULL hyper-parameters");
  FGS_CHECK_ARG(d_step || hp->step >= 1, "fgs_adam: step must be >= 1");
  // zero_from = 14: the gradient is only read (the struct is const to the caller)
  return launch_adam(params, const_cast<fgs_gaussians *>(grads), m, v, hp, d_step, 14, as_stream(stream));
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of fgs_loss.  Its per-CTA partial sums live in a
// file-scope device array instead of caller workspace, for callers that may not
// allocate device memory.  Host code must not pass the array's name to a kernel:
// on the host that name is only a stand-in, so the device address is looked up
// with cudaGetSymbolAddress once per device and cached (a cudaDeviceReset
// unloads the module, so the cached address is stale after one).
namespace fgs {

static __device__ __align__(256) double g_loss_scratch[FGS_LOSS_NOALLOC_MAX_TILES];

static std::mutex g_loss_scratch_mu;
static double *g_loss_scratch_dev[64] = {nullptr};

static fgs_status loss_scratch_address(double **out) {
  int dev = -1;
  FGS_CUDA(cudaGetDevice(&dev), "fgs_loss_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("fgs_loss_noalloc: device ordinal %d out of range", dev);
    return FGS_ERR_INVALID_ARGUMENT;
  }
  std::lock_guard<std::mutex> lock(g_loss_scratch_mu);
  if (g_loss_scratch_dev[dev] == nullptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_loss_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("fgs_loss_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FGS_ERR_CUDA;
    }
    g_loss_scratch_dev[dev] = static_cast<double *>(p);
  }
  *out = g_loss_scratch_dev[dev];
  return FGS_OK;
}

}  // namespace fgs

extern "C" fgs_status fgs_loss_noalloc(const fgs_camera *cams, int32_t n_views, const float *color,
                                       const float *depth, const float *color_gt, const float *depth_gt,
                                       const fgs_loss_params *params, float *dL_dcolor, float *dL_ddepth,
                                       float *d_loss, void *stream) {
  FGS_CHECK_ARG(color && depth && color_gt && depth_gt && params && dL_dcolor && dL_ddepth && d_loss,
                "fgs_loss_noalloc: NULL argument");
  LossArgs a;
  int blocks = 0;
  if (!loss_views(cams, n_views, &a.lv, &blocks, "fgs_loss_noalloc")) return FGS_ERR_INVALID_ARGUMENT;
  if (blocks > FGS_LOSS_NOALLOC_MAX_TILES) {
    set_error("fgs_loss_noalloc: %d loss tiles (32x32 px) exceed the built-in scratch of %d tiles; "
              "use fgs_loss with a workspace",
              blocks, FGS_LOSS_NOALLOC_MAX_TILES);
    return FGS_ERR_CAPACITY;
  }
  double *scratch = nullptr;
  const fgs_status s = loss_scratch_address(&scratch);
  if (s != FGS_OK) return s;
  a.color = color;
  a.depth = depth;
  a.color_gt = color_gt;
  a.depth_gt = depth_gt;
  a.w_c = params->w_l1_color;
  a.w_d = params->w_l1_depth;
  a.w_s = params->w_ssim;
  a.dC = dL_dcolor;
  a.dD = dL_ddepth;
  a.partials = scratch;
  double g[11], gs = 0.0;
  for (int i = 0; i < 11; ++i) {
    g[i] = std::exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
    gs += g[i];
  }
  for (int i = 0; i < 11; ++i) a.g[i] = (float)(g[i] / gs);
  const fgs_status sa = loss_smem_attr();
  if (sa != FGS_OK) return sa;
  cudaStream_t st = as_stream(stream);
  pdl_launch(k_loss, blocks, kLThreads, kLossSmem, st, a);
  pdl_launch(k_reduce_partials, 1, 256, 0, st, scratch, blocks, d_loss);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_loss_noalloc");
  return FGS_OK;
}
