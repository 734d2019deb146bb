// common.cuh -- shared device/host helpers of libfgs (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <utility>

#include "../../include/fgs.h"

namespace fgs {

// ---------------------------------------------------------------------------------
// Programmatic dependent launch (griddepcontrol).  The library's kernels follow
// one another on one stream, many of them short (binning, scans, reductions), so
// the gap between two dependent launches is a visible share of a step.  A kernel
// launched by pdl_launch may be scheduled while the kernel before it drains; its
// first statement is pdl_enter(), which waits until that kernel has completed and
// its writes are visible (griddepcontrol.wait), then lets the next kernel be
// scheduled in turn (griddepcontrol.launch_dependents).  Nothing before
// pdl_enter() touches memory, so the order of every read and write is the plain
// stream order.  FGS_PDL=0 in the environment launches without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

inline bool pdl_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("FGS_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

// kernel<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialisation; launch errors surface through cudaGetLastError as for <<<>>>.
template <typename... P, typename... A>
inline void pdl_launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

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

// The blend evaluates each (pixel, splat) pair in the base-2 domain: the
// staged copy of a splat carries its conic scaled by -log2(e)/2 (a, c) and
// -log2(e) (b), so that power * log2(e) is one quadratic form and G = exp(power)
// is one ex2.  Explicit rounding intrinsics make the forward and the adjoint
// kernels take bit-identical skip decisions and alphas.
constexpr float kLog2e = 1.44269504088896341f;
constexpr float kLn2 = 0.693147180559945309f;

__device__ __forceinline__ float4 stage_g0(float4 r0) {  // (mx, my, a, b) -> (mx, my, A, B)
  return make_float4(r0.x, r0.y, __fmul_rn(-0.5f * kLog2e, r0.z), __fmul_rn(-kLog2e, r0.w));
}
// (c, o, z, thr) -> (C, o, z, P) with P = -log2(255 o): alpha = o 2^power2 falls
// below 1/255 exactly where power2 < P, so the blend skips those pairs before
// the ex2 (the forward and the adjoint share the test, hence the decisions).
__device__ __forceinline__ float4 stage_g1(float4 r1) {
  return make_float4(__fmul_rn(-0.5f * kLog2e, r1.x), r1.y, r1.z, -log2f(__fmul_rn(255.f, r1.y)));
}

// power * log2(e) at pixel (px, py) for a staged conic (A, B, C); dx = mx - px, dy = my - py.
__device__ __forceinline__ float splat_power2(float mx, float my, float A, float B, float C, float px, float py,
                                              float &dx, float &dy) {
  dx = __fsub_rn(mx, px);
  dy = __fsub_rn(my, py);
  const float t = __fmul_rn(__fmul_rn(B, dx), dy);
  return __fmaf_rn(A, __fmul_rn(dx, dx), __fmaf_rn(C, __fmul_rn(dy, dy), t));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Margin added to the opacity-aware support threshold 2 ln(255 o): it exceeds
// every float32 rounding of the blend's alpha test, so a tile the binning culls
// (kept_columns() in binsort.cu) can hold no pixel whose alpha reaches 1/255.
constexpr float kSupportMargin = 0.01f;

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
