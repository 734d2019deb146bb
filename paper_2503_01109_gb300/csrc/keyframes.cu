// keyframes.cu -- keyframe co-visibility and the keyframe window of Sec. III-C
// ("Keyframe Selection"): keyframes that see more than a threshold of the current
// frame's points are co-visible, and a random share of the others joins them.
//
//   k_covisibility       one thread per sampled pixel: back-projection into the
//                        world, projection into every keyframe (cameras in the
//                        kernel parameters), warp-aggregated counts per keyframe
//   k_select_keyframes   one CTA: co-visible flags, then the random keyframes as
//                        the smallest draws among the rest (rank by comparison)
//
// Every operation of the geometry is rounded to float32 in a fixed order with
// explicit intrinsics, so the inside / outside decisions can be reproduced
// exactly elsewhere.
#include <cmath>

#include "common.cuh"

namespace fgs {

constexpr int kMaxKeyframes = 256;
constexpr int kMaxSelect = 1024;

struct KfCam {
  float R[9], t[3];
  float fx, fy, cx, cy, znear, umax, vmax;  // umax = W - 0.5, vmax = H - 0.5
};

struct KfArgs {
  int n;
  KfCam k[kMaxKeyframes];
};

// ((x a + y b) + z c), each operation rounded once
__device__ __forceinline__ float dot3v(float x, float y, float z, float a, float b, float c) {
  return __fadd_rn(__fadd_rn(__fmul_rn(x, a), __fmul_rn(y, b)), __fmul_rn(z, c));
}

__global__ void __launch_bounds__(256) k_covisibility(const float *__restrict__ depth, int W, int H, int step,
                                                      KfCam cur, KfArgs kf,
                                                      unsigned long long *__restrict__ d_inside,
                                                      unsigned long long *__restrict__ d_valid) {
  pdl_enter();
  const int sx = (W + step - 1) / step, sy = (H + step - 1) / step;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  float pw0 = 0.f, pw1 = 0.f, pw2 = 0.f;
  bool valid = false;
  if (s < (int64_t)sx * sy) {
    const int yy = (int)(s / sx), xx = (int)(s - (int64_t)yy * sx);
    const int x = xx * step, y = yy * step;
    const float d = depth[(int64_t)y * W + x];
    if (d > 0.f) {
      valid = true;
      const float xn = __fdiv_rn(__fsub_rn((float)x, cur.cx), cur.fx);
      const float yn = __fdiv_rn(__fsub_rn((float)y, cur.cy), cur.fy);
      const float q0 = __fsub_rn(__fmul_rn(xn, d), cur.t[0]);
      const float q1 = __fsub_rn(__fmul_rn(yn, d), cur.t[1]);
      const float q2 = __fsub_rn(d, cur.t[2]);
      // R^T (p_c - t): column i of R
      pw0 = dot3v(cur.R[0], cur.R[3], cur.R[6], q0, q1, q2);
      pw1 = dot3v(cur.R[1], cur.R[4], cur.R[7], q0, q1, q2);
      pw2 = dot3v(cur.R[2], cur.R[5], cur.R[8], q0, q1, q2);
    }
  }
  const uint32_t vb = __ballot_sync(0xffffffffu, valid);
  if (lane == 0 && vb) atomicAdd(d_valid, (unsigned long long)__popc(vb));
  for (int k = 0; k < kf.n; ++k) {
    // values, not references: the cameras stay in the parameter space
    const float r0 = kf.k[k].R[0], r1 = kf.k[k].R[1], r2 = kf.k[k].R[2];
    const float r3 = kf.k[k].R[3], r4 = kf.k[k].R[4], r5 = kf.k[k].R[5];
    const float r6 = kf.k[k].R[6], r7 = kf.k[k].R[7], r8 = kf.k[k].R[8];
    bool in = false;
    if (valid) {
      const float qx = __fadd_rn(dot3v(r0, r1, r2, pw0, pw1, pw2), kf.k[k].t[0]);
      const float qy = __fadd_rn(dot3v(r3, r4, r5, pw0, pw1, pw2), kf.k[k].t[1]);
      const float qz = __fadd_rn(dot3v(r6, r7, r8, pw0, pw1, pw2), kf.k[k].t[2]);
      if (qz > kf.k[k].znear) {
        const float u = __fadd_rn(__fmul_rn(kf.k[k].fx, __fdiv_rn(qx, qz)), kf.k[k].cx);
        const float v = __fadd_rn(__fmul_rn(kf.k[k].fy, __fdiv_rn(qy, qz)), kf.k[k].cy);
        in = u >= -0.5f && u < kf.k[k].umax && v >= -0.5f && v < kf.k[k].vmax;
      }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, in);
    if (lane == 0 && b) atomicAdd(d_inside + k, (unsigned long long)__popc(b));
  }
}

__global__ void k_covis_zero(unsigned long long *inside, int n, unsigned long long *valid) {
  pdl_enter();
  for (int k = threadIdx.x; k < n; k += blockDim.x) inside[k] = 0ull;
  if (threadIdx.x == 0) *valid = 0ull;
}

__global__ void __launch_bounds__(kMaxSelect) k_select_keyframes(const int64_t *__restrict__ d_inside,
                                                                 const int64_t *__restrict__ d_valid,
                                                                 const float *__restrict__ u, int n,
                                                                 float threshold, float frac,
                                                                 int32_t *__restrict__ d_kind,
                                                                 int32_t *__restrict__ d_count) {
  pdl_enter();
  __shared__ int s_rest[kMaxSelect];  // 1 where keyframe k is not co-visible
  __shared__ float s_u[kMaxSelect];
  __shared__ int s_nrest, s_count;
  const int k = threadIdx.x;
  if (k == 0) {
    s_nrest = 0;
    s_count = 0;
  }
  __syncthreads();
  const int64_t valid = *d_valid;
  bool covis = false;
  if (k < n) {
    // inside / valid > threshold, compared in double (exact for counts below 2^53)
    covis = valid > 0 && (double)d_inside[k] > (double)threshold * (double)valid;
    s_rest[k] = covis ? 0 : 1;
    s_u[k] = u[k];
    if (!covis) atomicAdd(&s_nrest, 1);
  }
  __syncthreads();
  const int want = (int)floorf(__fadd_rn(__fmul_rn(frac, (float)s_nrest), 0.5f));  // round(frac * rest)
  int kind = 0;
  if (k < n) {
    if (covis) {
      kind = 1;
    } else {
      int rank = 0;  // rest keyframes with a smaller draw, ties by index
      for (int j = 0; j < n; ++j)
        if (s_rest[j] && (s_u[j] < s_u[k] || (s_u[j] == s_u[k] && j < k))) ++rank;
      kind = rank < want ? 2 : 0;
    }
    d_kind[k] = kind;
    if (kind) atomicAdd(&s_count, 1);
  }
  __syncthreads();
  if (k == 0) *d_count = s_count;
}

static void fill_kf(const fgs_camera &c, KfCam &k) {
  for (int r = 0; r < 3; ++r) {
    for (int j = 0; j < 3; ++j) k.R[3 * r + j] = c.world_to_cam[4 * r + j];
    k.t[r] = c.world_to_cam[4 * r + 3];
  }
  k.fx = c.fx;
  k.fy = c.fy;
  k.cx = c.cx;
  k.cy = c.cy;
  k.znear = c.znear;
  k.umax = (float)c.width - 0.5f;
  k.vmax = (float)c.height - 0.5f;
}

}  // namespace fgs

using namespace fgs;

extern "C" fgs_status fgs_covisibility(const float *depth, const fgs_camera *cam, const fgs_camera *keyframes,
                                       int32_t n_keyframes, int32_t step, int64_t *d_inside, int64_t *d_valid,
                                       void *stream) {
  FGS_CHECK_ARG(depth && cam && keyframes && d_inside && d_valid, "fgs_covisibility: NULL argument");
  FGS_CHECK_ARG(step >= 1, "fgs_covisibility: step must be >= 1");
  FGS_CHECK_ARG(n_keyframes >= 1 && n_keyframes <= kMaxKeyframes, "fgs_covisibility: 1..%d keyframes",
                kMaxKeyframes);
  FGS_CHECK_ARG(cam->width > 0 && cam->height > 0 && cam->fx > 0 && cam->fy > 0, "fgs_covisibility: camera");
  KfCam cur;
  fill_kf(*cam, cur);
  KfArgs kf;
  kf.n = n_keyframes;
  for (int k = 0; k < n_keyframes; ++k) {
    FGS_CHECK_ARG(keyframes[k].fx > 0 && keyframes[k].fy > 0 && keyframes[k].width > 0 && keyframes[k].height > 0,
                  "fgs_covisibility: keyframe %d camera", k);
    fill_kf(keyframes[k], kf.k[k]);
  }
  cudaStream_t st = as_stream(stream);
  auto *inside = reinterpret_cast<unsigned long long *>(d_inside);
  auto *valid = reinterpret_cast<unsigned long long *>(d_valid);
  pdl_launch(k_covis_zero, 1, 256, 0, st, inside, n_keyframes, valid);
  const int64_t samples = (int64_t)((cam->width + step - 1) / step) * ((cam->height + step - 1) / step);
  const unsigned blocks = (unsigned)((samples + 255) / 256);
  pdl_launch(k_covisibility, blocks, 256, 0, st, depth, cam->width, cam->height, step, cur, kf, inside, valid);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_covisibility");
  return FGS_OK;
}

extern "C" fgs_status fgs_select_keyframes(const int64_t *d_inside, const int64_t *d_valid, const float *u,
                                           int32_t n_keyframes, float threshold, float frac, int32_t *d_kind,
                                           int32_t *d_count, void *stream) {
  FGS_CHECK_ARG(d_inside && d_valid && u && d_kind && d_count, "fgs_select_keyframes: NULL argument");
  FGS_CHECK_ARG(n_keyframes >= 1 && n_keyframes <= kMaxSelect, "fgs_select_keyframes: 1..%d keyframes",
                kMaxSelect);
  pdl_launch(k_select_keyframes, 1, kMaxSelect, 0, as_stream(stream), d_inside, d_valid, u, n_keyframes, threshold,
             frac, d_kind, d_count);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_select_keyframes");
  return FGS_OK;
}
