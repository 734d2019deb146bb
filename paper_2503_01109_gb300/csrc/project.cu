// project.cu -- EWA projection of the Gaussians (Sec. III: C = R S S^T R^T and its
// 2D projection) and its adjoint.
//
// One thread per Gaussian handles every view: the parameters are read once with
// coalesced structure-of-arrays loads and each view's 32-byte splat record is
// written with two float4 stores (consecutive threads, consecutive records).
#include "common.cuh"

namespace fgs {

struct GaussLocal {
  float mu[3], s[3], qn[4], qinv, R[9], o;
};

__device__ __forceinline__ void load_gaussian(const GaussPtrs &g, int64_t i, GaussLocal &L) {
  const int64_t c = g.cap;
  L.mu[0] = g.means[i];
  L.mu[1] = g.means[c + i];
  L.mu[2] = g.means[2 * c + i];
  float q0 = g.quats[i], q1 = g.quats[c + i], q2 = g.quats[2 * c + i], q3 = g.quats[3 * c + i];
  float len = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  L.qinv = 1.0f / len;
  float w = q0 * L.qinv, x = q1 * L.qinv, y = q2 * L.qinv, z = q3 * L.qinv;
  L.qn[0] = w; L.qn[1] = x; L.qn[2] = y; L.qn[3] = z;
  L.R[0] = 1.f - 2.f * (y * y + z * z); L.R[1] = 2.f * (x * y - w * z); L.R[2] = 2.f * (x * z + w * y);
  L.R[3] = 2.f * (x * y + w * z); L.R[4] = 1.f - 2.f * (x * x + z * z); L.R[5] = 2.f * (y * z - w * x);
  L.R[6] = 2.f * (x * z - w * y); L.R[7] = 2.f * (y * z + w * x); L.R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int k = 0; k < 3; ++k) L.s[k] = expf(g.log_scales[k * c + i]);
  L.o = 1.0f / (1.0f + expf(-g.logits[i]));
}

// a d - b c with one rounding error of each product compensated (the FMA recovers
// the exact error of b c), so that a small difference of two large products keeps
// its relative accuracy.
__device__ __forceinline__ float diff_of_products(float a, float d, float b, float c) {
  const float bc = b * c;
  const float err = fmaf(-b, c, bc);
  return fmaf(a, d, -bc) + err;
}

struct ViewLocal {
  float p[3];
  float uc, vc;
  bool clamp_u, clamp_v;
  float T[6];   // J R_cam, 2x3
  float TR[6];  // J R_cam R, 2x3: the Gaussian's axes in the image plane (per unit scale)
  float N[6];   // TR diag(s): Sigma' = N N^T + 0.3 I
  float a, b, c, det;
};

// Returns false when culled (behind the near plane or degenerate covariance).
// The 2D covariance is formed as N N^T (N = J R_cam R diag(s), 2x3) rather than
// through the 3D covariance, and its determinant by the Cauchy-Binet sum of the
// squared 2x2 minors of N plus the dilation's terms -- all positive, so that a
// needle-like Gaussian (one long axis) keeps an accurate determinant and conic
// in float32, where a c - b^2 would cancel.
__device__ __forceinline__ bool project_view(const GaussLocal &L, const DevCam &cm, ViewLocal &V) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    V.p[r] = cm.R[3 * r] * L.mu[0] + cm.R[3 * r + 1] * L.mu[1] + cm.R[3 * r + 2] * L.mu[2] + cm.t[r];
  const float z = V.p[2];
  if (!(z >= cm.znear)) return false;
  const float rz = 1.0f / z;
  const float limx = kJacClamp * (0.5f * (float)cm.W / cm.fx);
  const float limy = kJacClamp * (0.5f * (float)cm.H / cm.fy);
  const float u = V.p[0] * rz, v = V.p[1] * rz;
  V.uc = fminf(fmaxf(u, -limx), limx);
  V.vc = fminf(fmaxf(v, -limy), limy);
  V.clamp_u = V.uc != u;
  V.clamp_v = V.vc != v;
  const float jx = cm.fx * rz, jy = cm.fy * rz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    V.T[k] = jx * (cm.R[k] - V.uc * cm.R[6 + k]);
    V.T[3 + k] = jy * (cm.R[3 + k] - V.vc * cm.R[6 + k]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      V.TR[3 * r + k] = V.T[3 * r] * L.R[k] + V.T[3 * r + 1] * L.R[3 + k] + V.T[3 * r + 2] * L.R[6 + k];
      V.N[3 * r + k] = V.TR[3 * r + k] * L.s[k];
    }
  const float *N = V.N;
  const float aa = N[0] * N[0] + N[1] * N[1] + N[2] * N[2];
  const float cc = N[3] * N[3] + N[4] * N[4] + N[5] * N[5];
  V.a = aa + kDilation;
  V.b = N[0] * N[3] + N[1] * N[4] + N[2] * N[5];
  V.c = cc + kDilation;
  const float m01 = diff_of_products(N[0], N[4], N[1], N[3]);
  const float m02 = diff_of_products(N[0], N[5], N[2], N[3]);
  const float m12 = diff_of_products(N[1], N[5], N[2], N[4]);
  V.det = (m01 * m01 + m02 * m02 + m12 * m12) + kDilation * (aa + cc) + kDilation * kDilation;
  return V.det > 0.0f;
}

// A Gaussian whose position, scales, normalised quaternion, opacity or colour is
// not finite (a diverged optimisation, a zero quaternion) is culled from every
// view, and FGS_DEV_NONFINITE is set in *d_status (when given), once per warp.
__device__ __forceinline__ bool gaussian_finite(const GaussPtrs &g, int64_t i, const GaussLocal &L) {
  float s = L.o;
#pragma unroll
  for (int k = 0; k < 3; ++k) s += L.mu[k] + L.s[k] + g.rgb[k * g.cap + i];
#pragma unroll
  for (int k = 0; k < 4; ++k) s += L.qn[k];
  return isfinite(s);
}

__global__ void k_project(GaussPtrs g, int64_t n, const int64_t *__restrict__ d_n, DevViews vs,
                          int tw, int th, float4 *__restrict__ splat, int32_t *__restrict__ radius,
                          uint2 *__restrict__ rect, int64_t stride, int32_t *d_status) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i >= live_count(d_n, n)) {  // a slot past the live count: culled, its record otherwise untouched
#pragma unroll 1
    for (int v = 0; v < vs.n; ++v) radius[v * stride + i] = 0;
    return;
  }
  bool alive = true;
  GaussLocal L;
  {
    load_gaussian(g, i, L);
    const bool bad = !gaussian_finite(g, i, L);
    const unsigned m = __ballot_sync(__activemask(), bad);
    if (m && d_status && (int)(threadIdx.x & 31) == __ffs(m) - 1) atomicOr(d_status, FGS_DEV_NONFINITE);
    alive = !bad;
  }
#pragma unroll 1
  for (int v = 0; v < vs.n; ++v) {
    const DevCam &cm = vs.cam[v];
    const int64_t r = v * stride + i;
    ViewLocal V;
    if (!alive || !project_view(L, cm, V)) {
      splat[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
      splat[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      radius[r] = 0;
      rect[r] = make_uint2(1u | (1u << 16), 0u);
      continue;
    }
    const float rdet = 1.0f / V.det;
    const float ca = V.c * rdet, cb = -V.b * rdet, cc = V.a * rdet;
    const float rz = 1.0f / V.p[2];
    const float mx = cm.fx * V.p[0] * rz + cm.cx;
    const float my = cm.fy * V.p[1] * rz + cm.cy;
    const float mid = 0.5f * (V.a + V.c);
    const float lam = mid + sqrtf(fmaxf(0.0f, mid * mid - V.det));
    const int rad = (int)ceilf(kSupportSigma * sqrtf(lam));
    // opacity-aware support: alpha = o exp(-q/2) >= 1/255 needs q <= 2 ln(255 o);
    // a splat with o <= 1/255 can blend nowhere.  The box is the 3-sigma box cut
    // to the bounding box of that ellipse (half-widths sqrt(thr Sigma'_xx), ...).
    const float lo = 255.0f * L.o;
    const float thr = lo > 1.0f ? 2.0f * logf(lo) + kSupportMargin : -1.0f;
    const float k = fminf(kSupportSigma, sqrtf(fmaxf(thr, 0.f)));
    const float ex = k * sqrtf(V.a), ey = k * sqrtf(V.c);
    float x0 = ceilf((mx - ex - (float)(tw - 1)) / (float)tw);
    float x1 = floorf((mx + ex) / (float)tw);
    float y0 = ceilf((my - ey - (float)(th - 1)) / (float)th);
    float y1 = floorf((my + ey) / (float)th);
    x0 = fmaxf(x0, 0.f);
    y0 = fmaxf(y0, 0.f);
    x1 = fminf(x1, (float)(cm.tiles_x - 1));
    y1 = fminf(y1, (float)(cm.tiles_y - 1));
    uint2 rc = make_uint2(1u | (1u << 16), 0u);
    if (x0 <= x1 && y0 <= y1 && thr >= 0.f)
      rc = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
    splat[2 * r] = make_float4(mx, my, ca, cb);
    splat[2 * r + 1] = make_float4(cc, L.o, V.p[2], thr);
    radius[r] = rad;
    rect[r] = rc;
  }
}

// ---------------------------------------------------------------------------------
// Adjoint.  grad2d[v][stride] records: mean2d x, y, conic a, b, c, opacity, depth, -.
// Gradients are added to grads' planes; the thread owns its Gaussian, so no atomics.
// The chain rule of the projection for Gaussian i over every view: the gradients
// of its means (g[0..2]), log-scales (g[3..5]), quaternion (g[6..9]) and opacity
// logit (g[10]) from its splat records' gradients in grad2d.  Returns the mask of
// the views whose record it read (0 when no view projects it; then only g[10] may
// be non-zero).
__device__ __forceinline__ uint32_t chain_rule(const GaussLocal &L, int64_t i, const DevViews &vs,
                                               const int32_t *__restrict__ radius, const float4 *grad2d,
                                               int64_t stride, float *g) {
#pragma unroll
  for (int k = 0; k < 11; ++k) g[k] = 0.f;
  // Accumulated over views: dL/dlog s_k (gls) and the gradient of a rotation of
  // the Gaussian about its own axes (gth, the tangent space of the quaternion).
  float gls[3] = {0.f, 0.f, 0.f}, gth[3] = {0.f, 0.f, 0.f};
  const float s2[3] = {L.s[0] * L.s[0], L.s[1] * L.s[1], L.s[2] * L.s[2]};
  float go = 0.f;
  uint32_t read = 0u;
#pragma unroll 1
  for (int v = 0; v < vs.n; ++v) {
    const int64_t r = v * stride + i;
    if (radius[r] <= 0) continue;
    const DevCam &cm = vs.cam[v];
    ViewLocal V;
    if (!project_view(L, cm, V)) continue;
    read |= 1u << v;
    const float4 gA4 = grad2d[2 * r], gB4 = grad2d[2 * r + 1];
    const float rdet = 1.0f / V.det;
    const float A = V.c * rdet, B = -V.b * rdet, C = V.a * rdet;
    // dL/dSigma' = -Sigma'^-1 G Sigma'^-1 in terms of the conic (A, B, C)
    const float gA = gA4.z, gB = gA4.w, gC = gB4.x;
    const float ga = -(gA * A * A + gB * A * B + gC * B * B);
    const float gb = -(2.f * gA * A * B + gB * (A * C + B * B) + 2.f * gC * B * C);
    const float gc = -(gA * B * B + gB * B * C + gC * C * C);
    go += gB4.y;
    // G' = dL/dSigma' (2x2 symmetric, off-diagonal gb/2); Q = G' TR (2x3).  With
    // Sigma' = N N^T, N = TR diag(s):
    //   dL/dlog s_k = 2 N_k^T G' N_k = 2 s_k^2 (TR_k^T Q_k)          (N_k, TR_k: column k)
    //   K = TR^T G' TR, and a rotation R -> R (I + [theta]x) of the Gaussian about
    //   its own axes changes L by 2 K_12 (s_1^2 - s_2^2) theta_x
    //   + 2 K_02 (s_2^2 - s_0^2) theta_y + 2 K_01 (s_0^2 - s_1^2) theta_z;
    //   dL/dT = 2 G' T Sigma = 2 Q diag(s^2) R^T.
    const float G00 = ga, G01 = 0.5f * gb, G11 = gc;
    float Q[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Q[k] = G00 * V.TR[k] + G01 * V.TR[3 + k];
      Q[3 + k] = G01 * V.TR[k] + G11 * V.TR[3 + k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) gls[k] += 2.f * s2[k] * (V.TR[k] * Q[k] + V.TR[3 + k] * Q[3 + k]);
    const float K01 = V.TR[0] * Q[1] + V.TR[3] * Q[4];
    const float K02 = V.TR[0] * Q[2] + V.TR[3] * Q[5];
    const float K12 = V.TR[1] * Q[2] + V.TR[4] * Q[5];
    gth[0] += 2.f * K12 * (s2[1] - s2[2]);
    gth[1] += 2.f * K02 * (s2[2] - s2[0]);
    gth[2] += 2.f * K01 * (s2[0] - s2[1]);
    float QS[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      QS[k] = Q[k] * s2[k];
      QS[3 + k] = Q[3 + k] * s2[k];
    }
    float GT[6];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        GT[3 * rr + j] =
            2.f * (QS[3 * rr] * L.R[3 * j] + QS[3 * rr + 1] * L.R[3 * j + 1] + QS[3 * rr + 2] * L.R[3 * j + 2]);
    // T = J R_cam: dL/dJ = dL/dT R_cam^T (only J00, J02, J11, J12 are non-zero)
    const float *Rc = cm.R;
    const float GJ00 = GT[0] * Rc[0] + GT[1] * Rc[1] + GT[2] * Rc[2];
    const float GJ02 = GT[0] * Rc[6] + GT[1] * Rc[7] + GT[2] * Rc[8];
    const float GJ11 = GT[3] * Rc[3] + GT[4] * Rc[4] + GT[5] * Rc[5];
    const float GJ12 = GT[3] * Rc[6] + GT[4] * Rc[7] + GT[5] * Rc[8];
    const float x = V.p[0], y = V.p[1], z = V.p[2];
    const float rz = 1.0f / z, rz2 = rz * rz;
    float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f;
    gp2 += -(GJ00 * cm.fx + GJ11 * cm.fy) * rz2;
    if (V.clamp_u) {
      gp2 += GJ02 * cm.fx * V.uc * rz2;
    } else {  // J02 = -fx x / z^2
      gp0 += -GJ02 * cm.fx * rz2;
      gp2 += GJ02 * 2.f * cm.fx * x * rz2 * rz;
    }
    if (V.clamp_v) {
      gp2 += GJ12 * cm.fy * V.vc * rz2;
    } else {
      gp1 += -GJ12 * cm.fy * rz2;
      gp2 += GJ12 * 2.f * cm.fy * y * rz2 * rz;
    }
    // mean2d = (fx x/z + cx, fy y/z + cy); depth gamma = z
    gp0 += gA4.x * cm.fx * rz;
    gp1 += gA4.y * cm.fy * rz;
    gp2 += -(gA4.x * cm.fx * x + gA4.y * cm.fy * y) * rz2 + gB4.z;
    // p = R_cam mu + t
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] += Rc[k] * gp0 + Rc[3 + k] * gp1 + Rc[6 + k] * gp2;
  }
  g[10] = go * L.o * (1.f - L.o);
  if (!read) return 0u;
#pragma unroll
  for (int k = 0; k < 3; ++k) g[3 + k] = gls[k];
  // q_hat -> q_hat (x) (1, theta / 2) is the rotation R (I + [theta]x), so the
  // gradient with respect to the raw quaternion (through its normalisation) is
  // 2 (q_hat (x) (0, gth)) / |q| = (2 / |q|) (-v . gth, w gth + v x gth), already
  // orthogonal to q: no projection that would cancel.
  const float w = L.qn[0], qx = L.qn[1], qy = L.qn[2], qz = L.qn[3];
  const float f2 = 2.f * L.qinv;
  g[6] = -f2 * (qx * gth[0] + qy * gth[1] + qz * gth[2]);
  g[7] = f2 * (w * gth[0] + (qy * gth[2] - qz * gth[1]));
  g[8] = f2 * (w * gth[1] + (qz * gth[0] - qx * gth[2]));
  g[9] = f2 * (w * gth[2] + (qx * gth[1] - qy * gth[0]));
  return read;
}

__global__ void __launch_bounds__(256, 3)
    k_project_bwd(GaussPtrs g, int64_t n, const int64_t *__restrict__ d_n, DevViews vs,
                  const int32_t *__restrict__ radius, const float4 *__restrict__ grad2d, int64_t stride,
                  GaussGrads out) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || i >= live_count(d_n, n)) return;
  GaussLocal L;
  load_gaussian(g, i, L);
  // The kernel only adds to the gradient planes: their old values are loaded
  // here, together, so that their latencies overlap instead of each
  // read-modify-write waiting for the one before it.
  const int64_t c = out.cap;
  const float old_logit = out.logits[i];
  float old_mu[3], old_ls[3], old_q[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    old_mu[k] = out.means[k * c + i];
    old_ls[k] = out.log_scales[k * c + i];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) old_q[k] = out.quats[k * c + i];
  float gr[11];
  const bool any = chain_rule(L, i, vs, radius, grad2d, stride, gr) != 0u;
  out.logits[i] = old_logit + gr[10];
  if (!any) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out.means[k * c + i] = old_mu[k] + gr[k];
    out.log_scales[k * c + i] = old_ls[k] + gr[3 + k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) out.quats[k * c + i] = old_q[k] + gr[6 + k];
}

constexpr int FUSED_THREADS = 256;

// The first half of the end of a mapping iteration, per Gaussian: the chain rule
// of the projection plus the eq15 regulariser's gradient (as fgs_scale_reg),
// STORED into the 11 geometric gradient planes (nothing is read from them); the
// grad2d records read are cleared; per-block FP64 partial sums of the eq15 loss.
// The Adam pass that follows reads these planes and the RGB gradient.
__global__ void __launch_bounds__(FUSED_THREADS, 3)
    k_project_bwd_reg(GaussPtrs gp, int64_t n, const int64_t *__restrict__ d_n, DevViews vs,
                      const int32_t *__restrict__ radius, float4 *__restrict__ grad2d, int64_t stride,
                      GaussGrads out, float reg_weight, double *__restrict__ partials) {
  pdl_enter();
  __shared__ double red[FUSED_THREADS / 32];
  const int64_t live = live_count(d_n, n);
  const int tid = threadIdx.x;
  const int64_t i = blockIdx.x * (int64_t)FUSED_THREADS + tid;
  float reg_val = 0.f;
  const float wn = live > 0 ? reg_weight / (float)live : 0.f;
  if (i < live) {
    GaussLocal L;
    load_gaussian(gp, i, L);
    float gq[11];
    const uint32_t read = chain_rule(L, i, vs, radius, grad2d, stride, gq);
    if (reg_weight != 0.f) {  // eq15, as fgs_scale_reg
      const float s1 = L.s[0], s2 = L.s[1], s3 = L.s[2];
      const float mm = 0.5f * (s1 + s2);
      reg_val = fabsf(s1 - mm) + fabsf(s2 - mm) + fabsf(s3);
      const float sg1 = s1 - mm > 0.f ? 1.f : (s1 - mm < 0.f ? -1.f : 0.f);
      const float sg2 = s2 - mm > 0.f ? 1.f : (s2 - mm < 0.f ? -1.f : 0.f);
      gq[3] += wn * (0.5f * sg1 - 0.5f * sg2) * s1;
      gq[4] += wn * (0.5f * sg2 - 0.5f * sg1) * s2;
      gq[5] += wn * (s3 > 0.f ? 1.f : 0.f) * s3;
    }
    const int64_t c = out.cap;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      out.means[k * c + i] = gq[k];
      out.log_scales[k * c + i] = gq[3 + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out.quats[k * c + i] = gq[6 + k];
    out.logits[i] = gq[10];
    // The records read are cleared only now, after their values were used: a
    // store issued right behind the load of the same address waits for that
    // load in the memory pipeline and holds up the loads queued after it.
    for (uint32_t b = read; b; b &= b - 1) {
      const int64_t r = (int64_t)(__ffs(b) - 1) * stride + i;
      grad2d[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
      grad2d[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  float s = reg_val * wn;  // warp sums in FP32, block and grid sums in FP64 (as fgs_scale_reg)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) red[tid >> 5] = (double)s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < FUSED_THREADS / 32; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// *d_loss += the sum of `count` FP64 partials, in a fixed order (loss.cu).
void launch_reduce_partials(const double *partials, int64_t count, float *d_loss, cudaStream_t st);

// Adam over the 14 planes (loss.cu); planes from zero_from on have their gradient
// cleared after it is read.
fgs_status launch_adam(fgs_gaussians *params, fgs_gaussians *grads, fgs_gaussians *m, fgs_gaussians *v,
                       const fgs_adam_params *hp, int32_t *d_step, int zero_from, cudaStream_t st);

fgs_status launch_project_bwd(const fgs_gaussians *g, const DevViews &vs, const int32_t *radius,
                              const float *grad2d, int64_t stride, fgs_gaussians *grads,
                              cudaStream_t st) {
  if (g->n == 0) return FGS_OK;
  const int threads = 256;
  const int64_t blocks = (g->n + threads - 1) / threads;
  pdl_launch(k_project_bwd, (unsigned)blocks, threads, 0, st, gauss_ptrs(g), g->n, g->d_n, vs, radius,
             reinterpret_cast<const float4 *>(grad2d), stride, gauss_grads(grads));
  count_launch();
  FGS_CHECK_LAUNCH("project_bwd");
  return FGS_OK;
}

}  // namespace fgs

using namespace fgs;

extern "C" fgs_status fgs_project(const fgs_gaussians *g, const fgs_camera *cams, int32_t n_views,
                                  fgs_tiling tiling, fgs_projected *out, int32_t *d_status,
                                  void *stream) {
  if (!gaussians_ok(g, "g")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(tiling_ok(tiling), "fgs_project: unsupported tiling %dx%d/%d", tiling.tile_w,
                tiling.tile_h, tiling.batch_depth);
  FGS_CHECK_ARG(out && out->splat && out->radius && out->rect, "fgs_project: NULL output");
  FGS_CHECK_ARG(out->stride >= g->n, "fgs_project: stride < n");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(out->splat) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(out->rect) & 7) == 0,
                "fgs_project: splat must be 16-byte and rect 8-byte aligned");
  DevViews vs;
  if (!make_views(cams, n_views, tiling.tile_w, tiling.tile_h, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  if (g->n == 0) return FGS_OK;
  const int threads = 256;
  const int64_t blocks = (g->n + threads - 1) / threads;
  pdl_launch(k_project, (unsigned)blocks, threads, 0, as_stream(stream), gauss_ptrs(g), g->n, g->d_n, vs,
             tiling.tile_w, tiling.tile_h, reinterpret_cast<float4 *>(out->splat), out->radius,
             reinterpret_cast<uint2 *>(out->rect), out->stride, d_status);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_project");
  return FGS_OK;
}

extern "C" fgs_status fgs_project_bwd(const fgs_gaussians *g, const fgs_projected *proj, const fgs_camera *cams,
                                      int32_t n_views, const float *grad2d, fgs_gaussians *grads, void *stream) {
  if (!gaussians_ok(g, "g") || !gaussians_ok(grads, "grads")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(grads->n >= g->n, "fgs_project_bwd: grads->n < g->n");
  FGS_CHECK_ARG(proj && proj->radius && proj->stride >= g->n && grad2d, "fgs_project_bwd: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(grad2d) & 15) == 0, "fgs_project_bwd: grad2d alignment");
  DevViews vs;
  if (!make_views(cams, n_views, 16, 16, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  return launch_project_bwd(g, vs, proj->radius, grad2d, proj->stride, grads, as_stream(stream));
}

extern "C" size_t fgs_project_bwd_adam_workspace_size(int64_t n) {
  return align_up(sizeof(double) * (size_t)std::max<int64_t>((n + FUSED_THREADS - 1) / FUSED_THREADS, 1));
}

extern "C" fgs_status fgs_project_bwd_adam(fgs_gaussians *params, const fgs_projected *proj, const fgs_camera *cams,
                                           int32_t n_views, float *grad2d, fgs_gaussians *grads, float reg_weight,
                                           float *d_loss, fgs_gaussians *m, fgs_gaussians *v,
                                           const fgs_adam_params *hp, int32_t *d_step, void *ws, size_t ws_bytes,
                                           void *stream) {
  if (!gaussians_ok(params, "params") || !gaussians_ok(grads, "grads") || !gaussians_ok(m, "m") ||
      !gaussians_ok(v, "v"))
    return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(proj && proj->radius && proj->stride >= params->n && grad2d && hp && d_loss,
                "fgs_project_bwd_adam: NULL argument");
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(grad2d) & 15) == 0, "fgs_project_bwd_adam: grad2d alignment");
  FGS_CHECK_ARG(grads->n >= params->n && m->n >= params->n && v->n >= params->n,
                "fgs_project_bwd_adam: grads, m and v must cover params");
  FGS_CHECK_ARG(d_step || hp->step >= 1, "fgs_project_bwd_adam: step must be >= 1");
  FGS_CHECK_ARG(ws && ws_bytes >= fgs_project_bwd_adam_workspace_size(params->n),
                "fgs_project_bwd_adam: workspace");
  DevViews vs;
  if (!make_views(cams, n_views, 16, 16, &vs)) return FGS_ERR_INVALID_ARGUMENT;
  if (params->n == 0) return FGS_OK;
  cudaStream_t st = as_stream(stream);
  const int64_t blocks = (params->n + FUSED_THREADS - 1) / FUSED_THREADS;
  pdl_launch(k_project_bwd_reg, (unsigned)blocks, FUSED_THREADS, 0, st, gauss_ptrs(params), params->n, params->d_n,
             vs, proj->radius, reinterpret_cast<float4 *>(grad2d), proj->stride, gauss_grads(grads), reg_weight,
             static_cast<double *>(ws));
  launch_reduce_partials(static_cast<double *>(ws), blocks, d_loss, st);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_project_bwd_adam");
  // Adam over all 14 planes; it clears the RGB gradient planes after reading them
  return launch_adam(params, grads, m, v, hp, d_step, /*zero_from=*/11, st);
}
