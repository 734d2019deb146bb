// common.cuh -- shared device/host helpers of libfgs (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/fgs.h"

namespace fgs {

// ---------------------------------------------------------------------------------
// Rasteriser constants.  The paper states only the blend (eq1); these are the
// standard values of the Gaussian-splatting rasteriser it cites.
constexpr float kDilation = 0.3f;       // px^2 added to the 2D covariance
constexpr float kAlphaMax = 0.99f;      // alpha clamp (keeps 1 - alpha >= 0.01)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;          // stop before T would fall below this
constexpr float kJacClamp = 1.3f;       // x/z, y/z clamp in units of tan(half FOV)
constexpr float kSupportSigma = 3.0f;   // support box half-width in sigmas

// ---------------------------------------------------------------------------------
// error reporting (thread-local message, host launch counter)
void set_error(const char *fmt, ...);
void count_launch(int n = 1);

#define FGS_CHECK_ARG(cond, ...)              \
  do {                                        \
    if (!(cond)) {                            \
      ::fgs::set_error(__VA_ARGS__);          \
      return FGS_ERR_INVALID_ARGUMENT;        \
    }                                         \
  } while (0)

#define FGS_CHECK_LAUNCH(what)                                                         \
  do {                                                                                 \
    cudaError_t e__ = cudaGetLastError();                                              \
    if (e__ != cudaSuccess) {                                                          \
      ::fgs::set_error("%s: %s", what, cudaGetErrorString(e__));                       \
      return FGS_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

#define FGS_CUDA(call, what)                                                           \
  do {                                                                                 \
    cudaError_t e__ = (call);                                                          \
    if (e__ != cudaSuccess) {                                                          \
      ::fgs::set_error("%s: %s", what, cudaGetErrorString(e__));                       \
      return FGS_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------------------------
// views as kernel parameters

struct DevCam {
  int W, H;
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  float znear;
  int tiles_x, tiles_y;
  int tile_base;    // first global tile of the view
  int64_t pix_base; // first pixel of the view in concatenated images
};

struct DevViews {
  int n;
  int total_tiles;
  int64_t total_pix;
  DevCam cam[FGS_MAX_VIEWS];
};

inline bool tiling_ok(const fgs_tiling &t) {
  bool shape = (t.tile_w == 8 && t.tile_h == 8) || (t.tile_w == 16 && t.tile_h == 16) ||
               (t.tile_w == 16 && t.tile_h == 32);
  bool depth = t.batch_depth == 32 || t.batch_depth == 64 || t.batch_depth == 128 ||
               t.batch_depth == 256;
  return shape && depth;
}

// Fills a DevViews from host cameras; returns false (with the error set) on bad input.
bool make_views(const fgs_camera *cams, int32_t n_views, int tile_w, int tile_h, DevViews *out);

struct GaussPtrs {
  const float *means, *log_scales, *quats, *logits, *rgb;
  int64_t cap;
};
struct GaussGrads {
  float *means, *log_scales, *quats, *logits, *rgb;
  int64_t cap;
};

inline GaussPtrs gauss_ptrs(const fgs_gaussians *g) {
  return GaussPtrs{g->means, g->log_scales, g->quats, g->opacity_logits, g->rgb, g->capacity};
}
inline GaussGrads gauss_grads(const fgs_gaussians *g) {
  return GaussGrads{g->means, g->log_scales, g->quats, g->opacity_logits, g->rgb, g->capacity};
}
bool gaussians_ok(const fgs_gaussians *g, const char *name);

__device__ __forceinline__ int64_t live_count(const int64_t *d_n, int64_t n) {
  if (d_n == nullptr) return n;
  int64_t v = *d_n;
  return v < n ? v : n;
}

__device__ __forceinline__ int view_of_tile(const DevViews &vs, int t) {
  int v = 0;
#pragma unroll 1
  while (v + 1 < vs.n && t >= vs.cam[v + 1].tile_base) ++v;
  return v;
}

// Alpha of one (pixel, splat) evaluation, written with explicit rounding
// intrinsics so that the forward and the backward kernels take bit-identical
// skip / stop decisions.  Returns power; sets G = exp(power), alpha.
__device__ __forceinline__ float splat_power(float mx, float my, float ca, float cb, float cc,
                                             float px, float py, float &dx, float &dy) {
  dx = __fsub_rn(mx, px);
  dy = __fsub_rn(my, py);
  float q = __fmaf_rn(ca, __fmul_rn(dx, dx), __fmul_rn(cc, __fmul_rn(dy, dy)));
  return __fmaf_rn(-0.5f, q, -__fmul_rn(__fmul_rn(cb, dx), dy));
}

// Round-to-nearest float -> bf16 bits (ties to even), finite inputs.
__device__ __forceinline__ uint16_t f2bf(float x) {
  uint32_t b = __float_as_uint(x);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

int num_sms();

}  // namespace fgs
