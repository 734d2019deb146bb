// loss_tile.cuh -- one T x T tile of the fused eq16 loss (L1 colour, L1 depth,
// 1 - SSIM) and its gradient, shared by the loss kernel (loss.cu, T = 32) and the
// persistent window (window.cu, T = 16).
//
// The tile stages the colour pair with a 10-pixel halo in shared memory, forms
// the five windowed moments (mu_x, mu_y, E[x^2], E[y^2], E[xy]) with separable
// 11-tap sums on the tile plus a 5-pixel halo, evaluates SSIM and its partial
// derivatives there, and applies the adjoint window to produce dL/dC on the tile
// -- no intermediate map touches HBM.
//
// Each of the four 11-tap passes is register-blocked: a work item produces a run
// of consecutive outputs along the pass direction from one sliding read of its
// inputs (run + 10 loads instead of 11 per output), and the squares and cross
// product of the first pass are formed once per input.  Shared-memory rows have
// odd strides, so the lanes of a warp (consecutive rows in the horizontal passes,
// consecutive columns in the vertical ones) hit distinct banks.
#pragma once

#include "common.cuh"

namespace fgs {

constexpr int kLR = 5;  // window radius (11 taps)
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// Tile geometry for output side T.
template <int T>
struct LossGeom {
  static constexpr int In = T + 4 * kLR;    // input side (10-pixel halo)
  static constexpr int Mid = T + 2 * kLR;   // moment maps (5-pixel halo)
  static constexpr int RM = T == 32 ? 6 : 2;  // outputs per item of the two moment passes (divides Mid)
  static constexpr int RA = 4;              // outputs per item of the two adjoint passes (divides T)
  static constexpr int InS = In | 1, MidS = Mid | 1, TS = T | 1;  // odd row strides
  static constexpr int OffY = In * InS;
  static constexpr int OffH5 = 2 * In * InS;            // [5][In][MidS]; later H3 [3][Mid][TS]
  static constexpr int OffM3 = OffH5 + 5 * In * MidS;   // [3][Mid][MidS]
  static constexpr int SmemFloats = OffM3 + 3 * Mid * MidS;
  static_assert(Mid % RM == 0 && T % RA == 0, "runs must tile the maps");
  static_assert(3 * Mid * TS <= 5 * In * MidS, "H3 must fit in the H5 area");
};

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

// Loss tile b (a T x T output tile of one view) by the whole CTA (any multiple of
// 32 threads); `sm` holds LossGeom<T>::SmemFloats floats.  Writes dL/dC, dL/dD of
// the tile and the tile's loss contribution to a.partials[b].
template <int T>
__device__ __forceinline__ void loss_tile(const LossArgs &a, int b, float *sm) {
  using G = LossGeom<T>;
  constexpr int In = G::In, Mid = G::Mid, RM = G::RM, RA = G::RA;
  constexpr int InS = G::InS, MidS = G::MidS, TS = G::TS;
  float *X = sm;             // [In][InS]
  float *Y = sm + G::OffY;   // [In][InS]
  float *H5 = sm + G::OffH5; // [5][In][MidS]
  float *M3 = sm + G::OffM3; // [3][Mid][MidS]
  float *H3 = H5;            // [3][Mid][TS]
  __shared__ double red[32];
  const int nthr = blockDim.x;
  __syncthreads();  // the previous user of the shared buffer is done
  int v = 0;
  while (v + 1 < a.lv.n && b >= a.lv.v[v + 1].tile_base) ++v;
  const auto &cv = a.lv.v[v];
  const int lt = b - cv.tile_base;
  const int ty = lt / cv.tiles_x, tx = lt - ty * cv.tiles_x;
  const int W = cv.W, H = cv.H;
  const int64_t HW = (int64_t)W * H;
  const int ox = tx * T - 2 * kLR, oy = ty * T - 2 * kLR;  // input origin
  const float inv3 = 1.0f / (3.0f * (float)HW), inv1 = 1.0f / (float)HW;
  const float dS = -a.w_s * inv3;  // dL / dSSIM(q)
  const float *C = a.color + 3 * cv.pix_base, *Cg = a.color_gt + 3 * cv.pix_base;
  float *dC = a.dC + 3 * cv.pix_base;
  float acc = 0.f;
  for (int ch = 0; ch < 3; ++ch) {
    const float *Xc = C + ch * HW, *Yc = Cg + ch * HW;
    if (a.w_s != 0.f) {
      for (int e = threadIdx.x; e < In * In; e += nthr) {
        const int iy = e / In, ix = e - iy * In;
        const int gx = ox + ix, gy = oy + iy;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        X[iy * InS + ix] = in ? Xc[(int64_t)gy * W + gx] : 0.f;
        Y[iy * InS + ix] = in ? Yc[(int64_t)gy * W + gx] : 0.f;
      }
      __syncthreads();
      // horizontal moment sums: H5[k][r][c] over inputs (r, c .. c + 10), runs of RM columns
      for (int item = threadIdx.x; item < In * (Mid / RM); item += nthr) {
        const int r = item % In, c0 = (item / In) * RM;
        float s1[RM], s2[RM], s11[RM], s22[RM], s12[RM];
#pragma unroll
        for (int o = 0; o < RM; ++o) s1[o] = s2[o] = s11[o] = s22[o] = s12[o] = 0.f;
        const float *xr = X + r * InS + c0, *yr = Y + r * InS + c0;
#pragma unroll
        for (int i = 0; i < RM + 2 * kLR; ++i) {
          const float x = xr[i], y = yr[i];
          const float xx = x * x, yy = y * y, xy = x * y;
#pragma unroll
          for (int o = 0; o < RM; ++o) {
            const int t = i - o;
            if (t >= 0 && t <= 2 * kLR) {
              const float w = a.g[t];
              s1[o] = fmaf(w, x, s1[o]);
              s2[o] = fmaf(w, y, s2[o]);
              s11[o] = fmaf(w, xx, s11[o]);
              s22[o] = fmaf(w, yy, s22[o]);
              s12[o] = fmaf(w, xy, s12[o]);
            }
          }
        }
#pragma unroll
        for (int o = 0; o < RM; ++o) {
          const int q = r * MidS + c0 + o;
          H5[q] = s1[o];
          H5[In * MidS + q] = s2[o];
          H5[2 * In * MidS + q] = s11[o];
          H5[3 * In * MidS + q] = s22[o];
          H5[4 * In * MidS + q] = s12[o];
        }
      }
      __syncthreads();
      // vertical moment sums, SSIM and its partial derivatives at (r, c), runs of RM rows
      for (int item = threadIdx.x; item < Mid * (Mid / RM); item += nthr) {
        const int c = item % Mid, r0 = (item / Mid) * RM;
        float m[5][RM];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
          for (int o = 0; o < RM; ++o) m[k][o] = 0.f;
          const float *col = H5 + k * In * MidS + r0 * MidS + c;
#pragma unroll
          for (int i = 0; i < RM + 2 * kLR; ++i) {
            const float h = col[i * MidS];
#pragma unroll
            for (int o = 0; o < RM; ++o) {
              const int t = i - o;
              if (t >= 0 && t <= 2 * kLR) m[k][o] = fmaf(a.g[t], h, m[k][o]);
            }
          }
        }
        const int qx = ox + kLR + c;
#pragma unroll
        for (int o = 0; o < RM; ++o) {
          const int r = r0 + o;
          const int qy = oy + kLR + r;
          float d1 = 0.f, d11 = 0.f, d12 = 0.f;
          if (qx >= 0 && qx < W && qy >= 0 && qy < H) {
            const float m1 = m[0][o], m2 = m[1][o];
            const float sx = m[2][o] - m1 * m1, sy = m[3][o] - m2 * m2, sxy = m[4][o] - m1 * m2;
            const float A1 = 2.f * m1 * m2 + kC1, A2 = 2.f * sxy + kC2;
            const float B1 = m1 * m1 + m2 * m2 + kC1, B2 = sx + sy + kC2;
            const float rB = 1.f / (B1 * B2);
            const float S = A1 * A2 * rB;
            d1 = dS * ((2.f * m2 * A2 - 2.f * m2 * A1) * rB - S * (2.f * m1 / B1 - 2.f * m1 / B2));
            d11 = dS * (-S / B2);
            d12 = dS * (2.f * A1 * rB);
            if (r >= kLR && r < kLR + T && c >= kLR && c < kLR + T) acc += a.w_s * (1.f - S) * inv3;
          }
          const int q = r * MidS + c;
          M3[q] = d1;
          M3[Mid * MidS + q] = d11;
          M3[2 * Mid * MidS + q] = d12;
        }
      }
      __syncthreads();
      // adjoint window, horizontal: H3[k][r][c] over M3 (r, c .. c + 10), runs of RA columns
      for (int item = threadIdx.x; item < Mid * (T / RA); item += nthr) {
        const int r = item % Mid, c0 = (item / Mid) * RA;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float s[RA];
#pragma unroll
          for (int o = 0; o < RA; ++o) s[o] = 0.f;
          const float *row = M3 + k * Mid * MidS + r * MidS + c0;
#pragma unroll
          for (int i = 0; i < RA + 2 * kLR; ++i) {
            const float h = row[i];
#pragma unroll
            for (int o = 0; o < RA; ++o) {
              const int t = i - o;
              if (t >= 0 && t <= 2 * kLR) s[o] = fmaf(a.g[t], h, s[o]);
            }
          }
#pragma unroll
          for (int o = 0; o < RA; ++o) H3[k * Mid * TS + r * TS + c0 + o] = s[o];
        }
      }
      __syncthreads();
    }
    // adjoint window, vertical, and the gradient: runs of RA rows of column c
    for (int item = threadIdx.x; item < T * (T / RA); item += nthr) {
      const int c = item % T, r0 = (item / T) * RA;
      float vv[3][RA];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 0; o < RA; ++o) vv[k][o] = 0.f;
      if (a.w_s != 0.f) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float *col = H3 + k * Mid * TS + r0 * TS + c;
#pragma unroll
          for (int i = 0; i < RA + 2 * kLR; ++i) {
            const float h = col[i * TS];
#pragma unroll
            for (int o = 0; o < RA; ++o) {
              const int t = i - o;
              if (t >= 0 && t <= 2 * kLR) vv[k][o] = fmaf(a.g[t], h, vv[k][o]);
            }
          }
        }
      }
      const int gx = tx * T + c;
#pragma unroll
      for (int o = 0; o < RA; ++o) {
        const int gy = ty * T + r0 + o;
        if (gx < W && gy < H) {
          const int64_t p = (int64_t)gy * W + gx;
          float xp, yp;
          if (a.w_s != 0.f) {
            const int s = (r0 + o + 2 * kLR) * InS + c + 2 * kLR;
            xp = X[s];
            yp = Y[s];
          } else {
            xp = Xc[p];
            yp = Yc[p];
          }
          float grad = vv[0][o] + 2.f * xp * vv[1][o] + yp * vv[2][o];
          const float d = xp - yp;
          acc += a.w_c * fabsf(d) * inv3;
          grad += a.w_c * sgnf(d) * inv3;
          dC[ch * HW + p] = grad;
        }
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < T * T; e += nthr) {
    const int r = e / T, c = e - r * T;
    const int gx = tx * T + c, gy = ty * T + r;
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
    for (int w = 0; w < nthr / 32; ++w) t += red[w];
    a.partials[b] = t;
  }
}

}  // namespace fgs
