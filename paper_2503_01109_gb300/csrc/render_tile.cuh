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
  const int32_t *order = nullptr;  // launch order of the tiles (NULL: CTA i takes tile i)
  int32_t *d_status = nullptr;
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

// Pixel owned by a thread: each warp covers a block kWarpW pixels wide and
// (32 / kWarpW) * PX rows high, so that the 32 lanes' pixels are close together
// and stop blending after similar numbers of splats; the blocks tile the tile
// row by row.  Writes the thread's column and first row (tile coordinates).
#ifndef FGS_WARP_W
#define FGS_WARP_W 8
#endif
template <int TW, int TH, int PX>
__device__ __forceinline__ void thread_pixel(int &x, int &y0) {
  constexpr int WW = TW < FGS_WARP_W ? TW : FGS_WARP_W;
  constexpr int WH = (32 / WW) * PX;
  static_assert(TW % WW == 0 && TH % WH == 0 && (TW / WW) * (TH / WH) * 32 * PX == TW * TH,
                "warp blocks must tile the tile");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  x = (warp % (TW / WW)) * WW + lane % WW;
  y0 = (warp / (TW / WW)) * WH + (lane / WW) * PX;
}

// Shared memory of one tile pass (bytes): forward / adjoint.
template <int BATCH>
struct TileSmem {
  static constexpr int fwd = 48 * BATCH;
  static constexpr int bwd = 48 * BATCH + 4 * BATCH + 40 * BATCH + 16;
};

// Forward of global tile t by the whole CTA ((TW / S) * (TH / S) / PX threads);
// `smem` holds TileSmem<BATCH>::fwd bytes, 16-byte aligned.  S > 1 blends only the
// pixels with x % S == 0 and y % S == 0 (the same arithmetic per pixel, so the
// same values there) and writes the background (colour, depth and alpha 0,
// t_final 1, n_contrib 0) to the other pixels of the tile.
template <int TW, int TH, int BATCH, int PX, int S = 1>
__device__ __forceinline__ void render_fwd_tile(const RenderArgs &a, int t, char *smem) {
  static_assert(TW % S == 0 && TH % S == 0, "the sample grid must tile the tile");
  constexpr int NT = (TW / S) * (TH / S) / PX;
  float4 *s_g0 = reinterpret_cast<float4 *>(smem);  // mean2d x, y, conic a, b
  float4 *s_g1 = s_g0 + BATCH;                       // conic c, opacity, depth, -
  float4 *s_rgb = s_g1 + BATCH;
  const int v = view_of_tile(a.vs, t);
  const DevCam &cm = a.vs.cam[v];
  const int lt = t - cm.tile_base;
  const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
  int lx, ly0;
  thread_pixel<TW / S, TH / S, PX>(lx, ly0);
  const int px = tx * TW + S * lx;
  const int py0 = ty * TH + S * ly0;  // the thread's rows: py0 + S q
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
    done[q] = !(px < cm.W && py0 + S * q < cm.H);
    all_done = all_done && done[q];
  }
  for (int base = 0; base < n; base += BATCH) {
    if (__syncthreads_count(all_done) == NT) break;
    for (int j = threadIdx.x; j < BATCH; j += NT) {
      if (base + j < n) {
        const int id = a.ids[range.x + base + j];
        s_g0[j] = stage_g0(sp[2 * (int64_t)id]);
        s_g1[j] = stage_g1(sp[2 * (int64_t)id + 1]);
        s_rgb[j] = make_float4(a.rgb[id], a.rgb[a.cap + id], a.rgb[2 * a.cap + id], 0.f);
      }
    }
    __syncthreads();
    if (!all_done) {
      const int cnt = min(BATCH, n - base);
      if constexpr (PX == 1) {
        // one pixel per thread: the thread leaves the batch when its pixel stops
        const float fpy = (float)py0;
        for (int k = 0; k < cnt; ++k) {
          const float4 g0 = s_g0[k], g1 = s_g1[k];
          float dx, dy;
          const float power2 = splat_power2(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, fpy, dx, dy);
          if (power2 > 0.f || power2 < g1.w) continue;  // g1.w: alpha < 1/255 below it
          const float alpha = fminf(kAlphaMax, __fmul_rn(g1.y, ex2_approx(power2)));
          const float Tn = T[0] * (1.f - alpha);
          if (Tn < kTMin) {
            done[0] = true;
            break;
          }
          const float w = alpha * T[0];
          const float4 c = s_rgb[k];
          C0[0] += c.x * w;
          C1[0] += c.y * w;
          C2[0] += c.z * w;
          D[0] += g1.z * w;
          A[0] += w;
          T[0] = Tn;
          last[0] = base + k + 1;
        }
        all_done = done[0];
      } else {
        for (int k = 0; k < cnt; ++k) {
          const float4 g0 = s_g0[k], g1 = s_g1[k];
          bool any_live = false;
#pragma unroll
          for (int q = 0; q < PX; ++q) {
            if (done[q]) continue;
            any_live = true;
            float dx, dy;
            const float power2 = splat_power2(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, (float)(py0 + S * q), dx, dy);
            if (power2 > 0.f || power2 < g1.w) continue;
            const float alpha = fminf(kAlphaMax, __fmul_rn(g1.y, ex2_approx(power2)));
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
  }
  const int64_t HW = (int64_t)cm.W * cm.H;
  float *col = a.color + 3 * cm.pix_base;
#pragma unroll
  for (int q = 0; q < PX; ++q) {
#pragma unroll
    for (int sy = 0; sy < S; ++sy) {
#pragma unroll
      for (int sx = 0; sx < S; ++sx) {
        const bool sample = sx == 0 && sy == 0;
        const int x = px + sx, py = py0 + S * q + sy;
        if (x < cm.W && py < cm.H) {
          const int64_t pix = (int64_t)py * cm.W + x;
          col[pix] = sample ? C0[q] : 0.f;
          col[HW + pix] = sample ? C1[q] : 0.f;
          col[2 * HW + pix] = sample ? C2[q] : 0.f;
          a.depth[cm.pix_base + pix] = sample ? D[q] : 0.f;
          a.alpha[cm.pix_base + pix] = sample ? A[q] : 0.f;
          a.t_final[cm.pix_base + pix] = sample ? T[q] : 1.f;
          a.n_contrib[cm.pix_base + pix] = sample ? last[q] : 0;
        }
      }
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
  const int32_t *order = nullptr;  // launch order of the tiles (NULL: CTA i takes tile i)
  int32_t *d_status = nullptr;
};

// Sum of 10 per-lane values over the warp by recursive halving: at each
// butterfly step a lane keeps half of its values (the list padded to an even
// length with a zero) and adds the partner's copies of them, 10 -> 5 -> 3 -> 2 -> 1,
// twelve shuffles in all.  On return v[0] holds the warp total of field
// warp_sum10_field(lane), or of a padding slot where that is negative.
__device__ __forceinline__ void warp_sum10(float (&v)[10], int lane) {
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float send = u16 ? v[i] : v[i + 5];
    const float keep = u16 ? v[i + 5] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  v[5] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float send = u8 ? v[i] : v[i + 3];
    const float keep = u8 ? v[i + 3] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  v[3] = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = u4 ? v[i] : v[i + 2];
    const float keep = u4 ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const float send = u2 ? v[0] : v[1];
    const float keep = u2 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Field whose warp total warp_sum10() leaves in `lane`, or -1 for a padding slot.
__host__ __device__ __forceinline__ int warp_sum10_field(int lane) {
  const int lc = (lane >> 1) & 1;
  const int lb = ((lane >> 2) & 1) * 2 + lc;
  const int la = ((lane >> 3) & 1) * 3 + lb;
  if (lb >= 3 || la >= 5) return -1;
  return ((lane >> 4) & 1) * 5 + la;
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
  int lx, ly0;
  thread_pixel<TW, TH, PX>(lx, ly0);
  const int px = tx * TW + lx;
  const int py0 = ty * TH + ly0;
  const float fpx = (float)px;
  const int2 range = a.ranges[t];
  const float4 *sp = a.splat + 2 * (int64_t)v * a.stride;
  const int64_t HW = (int64_t)cm.W * cm.H;
  const float *dc = a.dC + 3 * cm.pix_base;
  // Per pixel: T (recovered front to back from T_final), the upstream gradient
  // g = (dL/dC, dL/dD, dL/dA), and U = sum over the splats behind the current one
  // of w_j (g . gamma_j), gamma_j = (colour_j, depth_j, 1): the term of dL/dalpha
  // that the splats behind contribute, carried as one scalar.
  float T[PX], gc0[PX], gc1[PX], gc2[PX], gd[PX], ga[PX], U[PX];
  int last[PX];
  int my_max = 0;
#pragma unroll
  for (int q = 0; q < PX; ++q) {
    const int py = py0 + q;
    T[q] = 1.f;
    last[q] = 0;
    gc0[q] = gc1[q] = gc2[q] = gd[q] = ga[q] = U[q] = 0.f;
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
  const int my_field = (lane & 1) ? -1 : warp_sum10_field(lane);
  const int warp_last = my_max;  // no pixel of this warp blends a splat at or past it
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
        s_g0[j] = stage_g0(sp[2 * (int64_t)id]);
        s_g1[j] = stage_g1(sp[2 * (int64_t)id + 1]);
        s_rgb[j] = make_float4(a.rgb[id], a.rgb[a.cap + id], a.rgb[2 * a.cap + id], 0.f);
      }
    }
    for (int e = threadIdx.x; e < BATCH * NF; e += NT) (&s_acc[0][0])[e] = 0.f;
    __syncthreads();
    for (int k = min(cnt, warp_last - start) - 1; k >= 0; --k) {
      const int j = start + k;
      const float4 g0 = s_g0[k], g1 = s_g1[k];
      float dx, dy[PX], power2[PX];
      bool hit[PX], any_hit = false;
#pragma unroll
      for (int q = 0; q < PX; ++q) {
        power2[q] = splat_power2(g0.x, g0.y, g0.z, g0.w, g1.x, fpx, (float)(py0 + q), dx, dy[q]);
        hit[q] = j < last[q] && !(power2[q] > 0.f || power2[q] < g1.w);
        any_hit = any_hit || hit[q];
      }
      if (!__ballot_sync(0xffffffffu, any_hit)) continue;  // the splat reaches no pixel of this warp
      const float4 c = s_rgb[k];
      // Sums over this thread's pixels.  The power's derivatives are linear in
      // e = dL/dalpha * G with coefficients (dx, dy, dx^2, dx dy, dy^2) and the
      // splat's conic and opacity, so the pixels accumulate those moments and the
      // flush below applies the per-splat factors once:
      //   0..4: sum e dx, e dy, e dx^2, e dx dy, e dy^2;  5: sum e (= dL/dopacity);
      //   6: sum dL/dD w;  7..9: sum dL/dC w.
      // The body has no branch: a pixel the splat does not reach (past its last
      // contributor, or alpha below 1/255) takes G = 0, so alpha = w = e = 0 and
      // rom = 1, and every update below leaves its value unchanged exactly.
      float acc[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[f] = 0.f;
#pragma unroll
      for (int q = 0; q < PX; ++q) {
        const float G = hit[q] ? ex2_approx(power2[q]) : 0.f;
        const float raw = __fmul_rn(g1.y, G);
        const float alpha = fminf(kAlphaMax, raw);
        const float rom = hit[q] ? __fdividef(1.f, 1.f - alpha) : 1.f;
        T[q] *= rom;  // transmittance in front of this splat
        const float w = alpha * T[q];
        const float dot_gam = gc0[q] * c.x + gc1[q] * c.y + gc2[q] * c.z + gd[q] * g1.z + ga[q];
        const float dalpha = T[q] * dot_gam - U[q] * rom;
        U[q] += w * dot_gam;
        acc[6] += gd[q] * w;
        acc[7] += gc0[q] * w;
        acc[8] += gc1[q] * w;
        acc[9] += gc2[q] * w;
        const float e = raw < kAlphaMax ? dalpha * G : 0.f;  // d alpha / d power = alpha (unclamped)
        const float ex = e * dx, ey = e * dy[q];
        acc[0] += ex;
        acc[1] += ey;
        acc[2] += ex * dx;
        acc[3] += ex * dy[q];
        acc[4] += ey * dy[q];
        acc[5] += e;
      }
      warp_sum10(acc, lane);
      if (my_field >= 0) atomicAdd(&s_acc[k][my_field], acc[0]);
    }
    __syncthreads();
    // dL/dmean = -o (Q m), dL/d(a, b, c) = -o (m_xx / 2, m_xy, m_yy / 2) with Q the
    // conic [[a, b], [b, c]] and m the moments above; dL/dopacity = sum e.  The
    // staged conic is (A, B, C) = -log2(e) (a/2, b, c/2), so -o Q m =
    // o ln2 (2A m_x + B m_y, B m_x + 2C m_y).
    // One thread per splat: its seven splat-record fields as two float4 atomics
    // (each field still receives one add per tile), the colour as three.
    for (int k = threadIdx.x; k < cnt; k += NT) {
      const float *m = s_acc[k];
      const float4 g0 = s_g0[k];
      const float cC = s_g1[k].x, o = s_g1[k].y;
      const float4 lo = make_float4(o * kLn2 * (2.f * g0.z * m[0] + g0.w * m[1]),
                                    o * kLn2 * (g0.w * m[0] + 2.f * cC * m[1]), -0.5f * o * m[2], -o * m[3]);
      const float4 hi = make_float4(-0.5f * o * m[4], m[5], m[6], 0.f);
      const int id = s_id[k];
      float4 *rec = reinterpret_cast<float4 *>(a.grad2d + 8 * ((int64_t)v * a.stride + id));
      if (lo.x != 0.f || lo.y != 0.f || lo.z != 0.f || lo.w != 0.f) atomicAdd(rec, lo);
      if (hi.x != 0.f || hi.y != 0.f || hi.z != 0.f) atomicAdd(rec + 1, hi);
#pragma unroll
      for (int f = 7; f < NF; ++f)
        if (m[f] != 0.f) atomicAdd(a.grad_rgb + (int64_t)(f - 7) * a.cap + id, m[f]);
    }
    __syncthreads();
  }
}

}  // namespace fgs
