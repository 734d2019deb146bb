// loss.cu -- the mapping loss of eq16 (L1 colour, L1 depth, 1 - SSIM), the scale
// regulariser of eq15, and the Adam step of the map optimisation (Sec. III-D).
//
// The loss kernel is one fused pass per 16x16 output tile: it stages the colour
// pair with a 10-pixel halo in shared memory, forms the five windowed moments
// (mu_x, mu_y, E[x^2], E[y^2], E[xy]) with separable 11-tap sums on the tile plus
// a 5-pixel halo, evaluates SSIM and its partial derivatives there, and applies
// the adjoint window to produce dL/dC on the tile -- no intermediate map touches
// HBM.  Loss values are reduced per CTA into a workspace and summed in a fixed
// order by one CTA, so the value is reproducible bit for bit.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace fgs {

constexpr int kLT = 16;              // output tile
constexpr int kLR = 5;               // window radius (11 taps)
constexpr int kLIn = kLT + 4 * kLR;  // 36: input with a 10-pixel halo
constexpr int kLMid = kLT + 2 * kLR; // 26: moment maps with a 5-pixel halo
constexpr int kLThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct LossViews {
  int n;
  struct V {
    int W, H, tiles_x, tile_base;
    int64_t pix_base;
  } v[FGS_MAX_VIEWS];
};

struct LossArgs {
  LossViews lv;
  const float *color, *depth, *color_gt, *depth_gt;
  float w_c, w_d, w_s;
  float *dC, *dD;
  double *partials;
  float g[11];
};

__device__ __forceinline__ float sgnf(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(kLThreads) k_loss(LossArgs a) {
  extern __shared__ float sm[];
  float *X = sm;                      // [kLIn][kLIn]
  float *Y = X + kLIn * kLIn;
  float *H5 = Y + kLIn * kLIn;        // [5][kLIn][kLMid]
  float *M5 = H5 + 5 * kLIn * kLMid;  // [5][kLMid][kLMid]; later [3] derivative maps
  float *H3 = H5;                     // [3][kLMid][kLT] (reuses H5)
  __shared__ double red[kLThreads / 32];
  const int b = blockIdx.x;
  int v = 0;
  while (v + 1 < a.lv.n && b >= a.lv.v[v + 1].tile_base) ++v;
  const auto &cv = a.lv.v[v];
  const int lt = b - cv.tile_base;
  const int ty = lt / cv.tiles_x, tx = lt - ty * cv.tiles_x;
  const int W = cv.W, H = cv.H;
  const int64_t HW = (int64_t)W * H;
  const int ox = tx * kLT - 2 * kLR, oy = ty * kLT - 2 * kLR;  // input origin
  const float inv3 = 1.0f / (3.0f * (float)HW), inv1 = 1.0f / (float)HW;
  const float dS = -a.w_s * inv3;  // dL / dSSIM(q)
  const float *C = a.color + 3 * cv.pix_base, *Cg = a.color_gt + 3 * cv.pix_base;
  float *dC = a.dC + 3 * cv.pix_base;
  float acc = 0.f;
  for (int ch = 0; ch < 3; ++ch) {
    const float *Xc = C + ch * HW, *Yc = Cg + ch * HW;
    if (a.w_s != 0.f) {
      for (int e = threadIdx.x; e < kLIn * kLIn; e += kLThreads) {
        const int iy = e / kLIn, ix = e - iy * kLIn;
        const int gx = ox + ix, gy = oy + iy;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        X[e] = in ? Xc[(int64_t)gy * W + gx] : 0.f;
        Y[e] = in ? Yc[(int64_t)gy * W + gx] : 0.f;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kLIn * kLMid; e += kLThreads) {
        const int r = e / kLMid, c = e - r * kLMid;
        float s1 = 0.f, s2 = 0.f, s11 = 0.f, s22 = 0.f, s12 = 0.f;
#pragma unroll
        for (int i = 0; i < 11; ++i) {
          const float x = X[r * kLIn + c + i], y = Y[r * kLIn + c + i], w = a.g[i];
          s1 += w * x;
          s2 += w * y;
          s11 += w * x * x;
          s22 += w * y * y;
          s12 += w * x * y;
        }
        const int o = r * kLMid + c;
        H5[o] = s1;
        H5[kLIn * kLMid + o] = s2;
        H5[2 * kLIn * kLMid + o] = s11;
        H5[3 * kLIn * kLMid + o] = s22;
        H5[4 * kLIn * kLMid + o] = s12;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kLMid * kLMid; e += kLThreads) {
        const int r = e / kLMid, c = e - r * kLMid;
        float m[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < 11; ++i) s += a.g[i] * H5[k * kLIn * kLMid + (r + i) * kLMid + c];
          m[k] = s;
        }
        const int qx = ox + kLR + c, qy = oy + kLR + r;
        float d1 = 0.f, d11 = 0.f, d12 = 0.f;
        if (qx >= 0 && qx < W && qy >= 0 && qy < H) {
          const float m1 = m[0], m2 = m[1];
          const float sx = m[2] - m1 * m1, sy = m[3] - m2 * m2, sxy = m[4] - m1 * m2;
          const float A1 = 2.f * m1 * m2 + kC1, A2 = 2.f * sxy + kC2;
          const float B1 = m1 * m1 + m2 * m2 + kC1, B2 = sx + sy + kC2;
          const float rB = 1.f / (B1 * B2);
          const float S = A1 * A2 * rB;
          d1 = dS * ((2.f * m2 * A2 - 2.f * m2 * A1) * rB - S * (2.f * m1 / B1 - 2.f * m1 / B2));
          d11 = dS * (-S / B2);
          d12 = dS * (2.f * A1 * rB);
          if (r >= kLR && r < kLR + kLT && c >= kLR && c < kLR + kLT) acc += a.w_s * (1.f - S) * inv3;
        }
        M5[e] = d1;
        M5[kLMid * kLMid + e] = d11;
        M5[2 * kLMid * kLMid + e] = d12;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kLMid * kLT; e += kLThreads) {
        const int r = e / kLT, c = e - r * kLT;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < 11; ++i) s += a.g[i] * M5[k * kLMid * kLMid + r * kLMid + c + i];
          H3[k * kLMid * kLT + e] = s;
        }
      }
      __syncthreads();
    }
    {
      const int r = threadIdx.x / kLT, c = threadIdx.x - r * kLT;
      const int gx = tx * kLT + c, gy = ty * kLT + r;
      if (gx < W && gy < H) {
        const int64_t p = (int64_t)gy * W + gx;
        const float xp = Xc[p], yp = Yc[p];
        float grad = 0.f;
        if (a.w_s != 0.f) {
          float vv[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 11; ++i) s += a.g[i] * H3[k * kLMid * kLT + (r + i) * kLT + c];
            vv[k] = s;
          }
          grad = vv[0] + 2.f * xp * vv[1] + yp * vv[2];
        }
        const float d = xp - yp;
        acc += a.w_c * fabsf(d) * inv3;
        grad += a.w_c * sgnf(d) * inv3;
        dC[ch * HW + p] = grad;
      }
    }
    __syncthreads();
  }
  {
    const int r = threadIdx.x / kLT, c = threadIdx.x - r * kLT;
    const int gx = tx * kLT + c, gy = ty * kLT + r;
    if (gx < W && gy < H) {
      const int64_t p = cv.pix_base + (int64_t)gy * W + gx;
      const float dg = a.depth_gt[p];
      float gd = 0.f;
      if (dg > 0.f) {
        const float d = a.depth[p] - dg;
        acc += a.w_d * fabsf(d) * inv1;
        gd = a.w_d * sgnf(d) * inv1;
      }
      a.dD[p] = gd;
    }
  }
  double s = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLThreads / 32; ++w) t += red[w];
    a.partials[blockIdx.x] = t;
  }
}

// Sums `count` partials in a fixed order and adds the total to *d_loss.
__global__ void k_reduce_partials(const double *__restrict__ partials, int64_t count, float *d_loss) {
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

static bool loss_views(const fgs_camera *cams, int32_t n_views, LossViews *lv, int *blocks) {
  if (!cams || n_views < 1 || n_views > FGS_MAX_VIEWS) {
    set_error("fgs_loss: n_views must be 1..%d", FGS_MAX_VIEWS);
    return false;
  }
  lv->n = n_views;
  int tiles = 0;
  int64_t pix = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width <= 0 || cams[v].height <= 0) {
      set_error("fgs_loss: bad image size");
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
  double s = (double)val * (double)wn;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
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
  const float *g[14];
  float *m[14];
  float *v[14];
  float lr[14];
};

__global__ void k_adam_step_incr(int32_t *d_step) { *d_step += 1; }

__global__ void k_adam(AdamPlanes P, int64_t n, const int64_t *d_n, float b1, float b2, float eps, int32_t step,
                       const int32_t *d_step) {
  const int plane = blockIdx.y;
  const int64_t live = live_count(d_n, n);
  const int t = d_step ? *d_step : step;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  const float lr = P.lr[plane];
  float *__restrict__ p = P.p[plane];
  const float *__restrict__ g = P.g[plane];
  float *__restrict__ m = P.m[plane];
  float *__restrict__ v = P.v[plane];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < live; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
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
  const size_t smem = sizeof(float) * (2 * kLIn * kLIn + 5 * kLIn * kLMid + 5 * kLMid * kLMid);
  static_assert(sizeof(float) * (2 * kLIn * kLIn + 5 * kLIn * kLMid + 5 * kLMid * kLMid) <= 48 * 1024,
                "loss tile must fit the default dynamic shared-memory limit");
  cudaStream_t st = as_stream(stream);
  k_loss<<<blocks, kLThreads, smem, st>>>(a);
  k_reduce_partials<<<1, 256, 0, st>>>(a.partials, blocks, d_loss);
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
  k_scale_reg<<<(unsigned)blocks, 256, 0, st>>>(g->log_scales, g->capacity, g->n, g->d_n, weight, grads->log_scales,
                                                static_cast<double *>(ws));
  k_reduce_partials<<<1, 256, 0, st>>>(static_cast<double *>(ws), blocks, d_loss);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_scale_reg");
  return FGS_OK;
}

extern "C" fgs_status fgs_adam(fgs_gaussians *params, const fgs_gaussians *grads, fgs_gaussians *m,
                               fgs_gaussians *v, const fgs_adam_params *hp, int32_t *d_step, void *stream) {
  if (!gaussians_ok(params, "params") || !gaussians_ok(grads, "grads") || !gaussians_ok(m, "m") ||
      !gaussians_ok(v, "v"))
    return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(hp, "fgs_adam: NULL hyper-parameters");
  FGS_CHECK_ARG(d_step || hp->step >= 1, "fgs_adam: step must be >= 1");
  if (params->n == 0) return FGS_OK;
  AdamPlanes P;
  auto fill = [&](int base, int cnt, float *pp, const float *gp, float *mp, float *vp, int64_t pc, int64_t gc,
                  int64_t mc, int64_t vc, float lr) {
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
  cudaStream_t st = as_stream(stream);
  if (d_step) {
    k_adam_step_incr<<<1, 1, 0, st>>>(d_step);
    count_launch();
  }
  const int64_t want = (params->n + 1023) / 1024;
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 2 * num_sms()));
  k_adam<<<dim3(bx, 14), 256, 0, st>>>(P, params->n, params->d_n, hp->beta1, hp->beta2, hp->eps, hp->step, d_step);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_adam");
  return FGS_OK;
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of fgs_loss.  Its per-CTA partial sums live in a
// file-scope device array instead of caller workspace, for callers that may not
// allocate device memory.  Host code must not pass the array's name to a kernel:
// on the host that name is only a stand-in, so the device address is looked up
// with cudaGetSymbolAddress once per device and cached.
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
  if (!loss_views(cams, n_views, &a.lv, &blocks)) return FGS_ERR_INVALID_ARGUMENT;
  if (blocks > FGS_LOSS_NOALLOC_MAX_TILES) {
    set_error("fgs_loss_noalloc: %d loss tiles (16x16 px) exceed the built-in scratch of %d tiles; "
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
  const size_t smem = sizeof(float) * (2 * kLIn * kLIn + 5 * kLIn * kLMid + 5 * kLMid * kLMid);
  cudaStream_t st = as_stream(stream);
  k_loss<<<blocks, kLThreads, smem, st>>>(a);
  k_reduce_partials<<<1, 256, 0, st>>>(scratch, blocks, d_loss);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_loss_noalloc");
  return FGS_OK;
}
