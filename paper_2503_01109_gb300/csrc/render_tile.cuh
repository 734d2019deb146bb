// render_tile.cuh -- per-tile bodies of the eq1 blend and its adjoint, shared by
// the one-CTA-per-tile kernels (render.cu) and the persistent window (window.cu).
#pragma once

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

// Pixels per thread: a thread owns PX vertically adjacent pixels of its tile
// column, so every splat staged in shared memory is read once per PX pixels and,
// in the adjoint, its gradients are summed over PX pixels in registers before
// the warp reduction.
// Measured at 1200x680 with a 1M-Gaussian map (ms per mapping iteration, 16x16
// tiles): forward 1 px/thread 0.82 vs 2 px 0.84 vs 4 px 1.02; adjoint 2 px 1.77
// vs 4 px 1.92 vs 8 px 2.52.
#ifndef FGS_FWD_PX
#define FGS_FWD_PX 1
#endif
#ifndef FGS_BWD_PX
#define FGS_BWD_PX 2
#endif
template <int TW, int TH>
struct PxPerThread {
  static constexpr int fwd = (TW * TH >= 256) ? FGS_FWD_PX : 1;
  static constexpr int bwd = (TW * TH >= 256) ? FGS_BWD_PX : 2;
};

// Shared memory of one tile pass (bytes): forward / adjoint.
template <int BATCH>
struct TileSmem {
  static constexpr int fwd = 48 * BATCH;
  static constexpr int bwd = 48 * BATCH + 4 * BATCH + 40 * BATCH + 16;
};

// Forward of global tile t by the whole CTA (TW * TH / PX threads); `smem` holds
// TileSmem<BATCH>::fwd bytes, 16-byte aligned.
template <int TW, int TH, int BATCH, int PX>
__device__ __forceinline__ void render_fwd_tile(const RenderArgs &a, int t, char *smem) {
  constexpr int NT = TW * TH / PX;
  float4 *s_g0 = reinterpret_cast<float4 *>(smem);  // mean2d x, y, conic a, b
  float4 *s_g1 = s_g0 + BATCH;                       // conic c, opacity, depth, -
  float4 *s_rgb = s_g1 + BATCH;
  const int v = view_of_tile(a.vs, t);
  const DevCam &cm = a.vs.cam[v];
  const int lt = t - cm.tile_base;
  const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
  const int px = tx * TW + (threadIdx.x % TW);
  const int py0 = ty * TH + (threadIdx.x / TW) * PX;
  const float fpx = (float)px;
  const int2 range = a.ranges[t];
  const int n = range.y - range.x;
  const float4 *sp = a.splat + 2 * (int64_t)v * a.stride;
  float T[PX], C0[PX], C1[PX], C2[PX], D[PX], A[PX];
  int last[PX];
  bool done[PX];
  bool all_done = true;
  __syncthreads();  // the previous user of the shared buffer is done
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    T[q] = 1.f;
    C0[q] = C1[q] = C2[q] = D[q] = A[q] = 0.f;
    last[q] = 0;
    done[q] = !(px < cm.W && py0 + q < cm.H);
    all_done = all_done && done[q];
  }
  for (int base = 0; base < n; base += BATCH) {
    if (__syncthreads_count(all_done) == NT) break;
    for (int j = threadIdx.x; j < BATCH; j += NT) {
      if (base + j < n) {
        const int id = a.ids[range.x + base + j];
        s_g0[j] = sp[2 * (int64_t)id];
        s_g1[j] = sp[2 * (int64_t)id + 1];
        s_rgb[j] = make_float4(a.rgb[id], a.rgb[a.cap + id], a.rgb[2 * a.cap + id], 0.f);
      }
    }
    __syncthreads();
    if (!all_done) {
      const int cnt = min(BATCH, n - base);
      for (int k = 0; k < cnt; ++k) {
        const float4 g0 = s_g0[k], g1 = s_g1[k];
        bool any_live = false;
#pragma unroll
        for (int q = 0; q < PX; ++q) {
          if (done[q]) continue;
          any_live = true;
          float dx, dy;
          const float power = splat_power(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, (float)(py0 + q), dx, dy);
          if (power > 0.f) continue;
          const float alpha = fminf(kAlphaMax, __fmul_rn(g1.y, __expf(power)));
          if (alpha < kAlphaMin) continue;
          const float Tn = T[q] * (1.f - alpha);
          if (Tn < kTMin) {
            done[q] = true;
            continue;
          }
          const float w = alpha * T[q];
          const float4 c = s_rgb[k];
          C0[q] += c.x * w;
          C1[q] += c.y * w;
          C2[q] += c.z * w;
          D[q] += g1.z * w;
          A[q] += w;
          T[q] = Tn;
          last[q] = base + k + 1;
        }
        if (!any_live) break;
      }
      all_done = true;
#pragma unroll
      for (int q = 0; q < PX; ++q) all_done = all_done && done[q];
    }
  }
  const int64_t HW = (int64_t)cm.W * cm.H;
  float *col = a.color + 3 * cm.pix_base;
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    const int py = py0 + q;
    if (px < cm.W && py < cm.H) {
      const int64_t pix = (int64_t)py * cm.W + px;
      col[pix] = C0[q];
      col[HW + pix] = C1[q];
      col[2 * HW + pix] = C2[q];
      a.depth[cm.pix_base + pix] = D[q];
      a.alpha[cm.pix_base + pix] = A[q];
      a.t_final[cm.pix_base + pix] = T[q];
      a.n_contrib[cm.pix_base + pix] = last[q];
    }
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

// Sum of 16 per-lane values over the warp by recursive halving: at each of the
// five butterfly steps a lane keeps half of its values and adds the partner's
// copies of them, so all 16 totals take 16 shuffles.  On return v[0] holds the
// total of field (lane >> 1) (lanes 2f and 2f+1 hold the same total).
__device__ __forceinline__ void warp_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool up = lane & bit;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Adjoint of global tile t by the whole CTA; `smem` holds TileSmem<BATCH>::bwd bytes.
template <int TW, int TH, int BATCH, int PX>
__device__ __forceinline__ void render_bwd_tile(const RenderBwdArgs &a, int t, char *smem) {
  constexpr int NT = TW * TH / PX;
  constexpr int NF = 10;  // mean2d x, y, conic a, b, c, opacity, depth, r, g, b
  float4 *s_g0 = reinterpret_cast<float4 *>(smem);
  float4 *s_g1 = s_g0 + BATCH;
  float4 *s_rgb = s_g1 + BATCH;
  float (*s_acc)[NF] = reinterpret_cast<float (*)[NF]>(s_rgb + BATCH);
  int *s_id = reinterpret_cast<int *>(s_acc + BATCH);
  int &s_max_last = s_id[BATCH];
  const int v = view_of_tile(a.vs, t);
  const DevCam &cm = a.vs.cam[v];
  const int lt = t - cm.tile_base;
  const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
  const int px = tx * TW + (threadIdx.x % TW);
  const int py0 = ty * TH + (threadIdx.x / TW) * PX;
  const float fpx = (float)px;
  const int2 range = a.ranges[t];
  const float4 *sp = a.splat + 2 * (int64_t)v * a.stride;
  const int64_t HW = (int64_t)cm.W * cm.H;
  const float *dc = a.dC + 3 * cm.pix_base;
  float T[PX], gc0[PX], gc1[PX], gc2[PX], gd[PX], ga[PX];
  float S0[PX], S1[PX], S2[PX], Sd[PX], Sa[PX];  // sums of gamma alpha T behind the current splat
  int last[PX];
  int my_max = 0;
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    const int py = py0 + q;
    T[q] = 1.f;
    last[q] = 0;
    gc0[q] = gc1[q] = gc2[q] = gd[q] = ga[q] = 0.f;
    S0[q] = S1[q] = S2[q] = Sd[q] = Sa[q] = 0.f;
    if (px < cm.W && py < cm.H) {
      const int64_t pix = (int64_t)py * cm.W + px;
      T[q] = a.t_final[cm.pix_base + pix];
      last[q] = a.n_contrib[cm.pix_base + pix];
      gc0[q] = dc[pix];
      gc1[q] = dc[HW + pix];
      gc2[q] = dc[2 * HW + pix];
      if (a.dD) gd[q] = a.dD[cm.pix_base + pix];
      if (a.dA) ga[q] = a.dA[cm.pix_base + pix];
      my_max = max(my_max, last[q]);
    }
  }
  __syncthreads();  // the previous user of the shared buffer is done
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
  const int lane = threadIdx.x & 31;
  if (lane == 0 && my_max > 0) atomicMax(&s_max_last, my_max);
  __syncthreads();
  const int max_last = s_max_last;
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
      const float4 g0 = s_g0[k], g1 = s_g1[k];
      const float4 c = s_rgb[k];
      float acc[16];
#pragma unroll
      for (int f = 0; f < 16; ++f) acc[f] = 0.f;
      bool contrib = false;
#pragma unroll
      for (int q = 0; q < PX; ++q) {
        if (j >= last[q]) continue;
        float dx, dy;
        const float power = splat_power(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, (float)(py0 + q), dx, dy);
        if (power > 0.f) continue;
        const float G = __expf(power);
        const float raw = __fmul_rn(g1.y, G);
        const float alpha = fminf(kAlphaMax, raw);
        if (alpha < kAlphaMin) continue;
        contrib = true;
        const float rom = __fdividef(1.f, 1.f - alpha);
        T[q] *= rom;  // transmittance in front of this splat
        const float w = alpha * T[q];
        const float dot_gam = gc0[q] * c.x + gc1[q] * c.y + gc2[q] * c.z + gd[q] * g1.z + ga[q];
        const float dot_S = gc0[q] * S0[q] + gc1[q] * S1[q] + gc2[q] * S2[q] + gd[q] * Sd[q] + ga[q] * Sa[q];
        const float dalpha = T[q] * dot_gam - dot_S * rom;
        S0[q] += c.x * w;
        S1[q] += c.y * w;
        S2[q] += c.z * w;
        Sd[q] += g1.z * w;
        Sa[q] += w;
        acc[6] += gd[q] * w;
        acc[7] += gc0[q] * w;
        acc[8] += gc1[q] * w;
        acc[9] += gc2[q] * w;
        if (raw < kAlphaMax) {
          const float dp = dalpha * alpha;  // d alpha / d power = alpha (unclamped)
          acc[0] -= dp * (g0.z * dx + g0.w * dy);
          acc[1] -= dp * (g0.w * dx + g1.x * dy);
          acc[2] -= 0.5f * dp * dx * dx;
          acc[3] -= dp * dx * dy;
          acc[4] -= 0.5f * dp * dy * dy;
          acc[5] += dalpha * G;
        }
      }
      if (__ballot_sync(0xffffffffu, contrib)) {
        warp_sum16(acc, lane);
        const int f = lane >> 1;
        if ((lane & 1) == 0 && f < NF) atomicAdd(&s_acc[k][f], acc[0]);
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

}  // namespace fgs
