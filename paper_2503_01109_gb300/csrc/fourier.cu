// fourier.cu -- adaptive densification of Sec. III-A (eq2-eq11) for one frame.
//
//   k_fft_rows      gray = BT.601 luma of the frame, eq2's DFT along x for every row
//   k_fft_cols      per group of columns of the spectrum's left half (the right
//                   half is its conjugate mirror): DFT along y, the Gaussian high-pass of
//                   eq5/eq7 evaluated at the shifted frequency (eq3), inverse DFT
//                   along y -- forward, filter and inverse fused in shared memory
//   k_ifft_rows     inverse DFT along x, E = |I_h| / (H W) (eq8), running max of E
//   k_hist          256-bin histogram of E / max E (float32 decision per pixel); a
//                   frame whose max E is at most 1e-5 of its peak gray has no
//                   high-frequency region (E is rounding noise there)
//   k_triangle      triangle threshold t in exact integer arithmetic (one thread
//                   per bin, block reductions)
//   k_seed_count    masks M_h / M_l / M_m (eq9, eq10) and the equidistant samples,
//                   kept per pixel in the mask byte; per-CTA counts of high / low seeds
//   k_seed_scan     scan of the CTA counts, capped seed count, append base
//   k_seed_write    from the mask bytes: ordered compaction (high seeds then low,
//                   row-major), the seeded bit, and eq11:
//                   back-projected mean, log-scale log(alpha d / f), identity
//                   rotation, frame colour, initial logit
//
// The FFT is a mixed-radix Stockham autosort transform with the twiddle factors
// of its length tabulated in shared memory once per CTA: each stage of radix p
// combines p interleaved sub-transforms of length L into one of length L p with
// twiddles exp(-+2 pi i r k / (L p)) and a direct p-point DFT, ping-ponging between
// two shared-memory buffers; the output is in natural order.  Radices: 8, 4, 2
// and the odd primes up to 17 (so 64, 640, 1200, 48, 480 and 680 = 8 * 5 * 17
// are all exact transforms; sizes with a larger prime factor are rejected).
#include <cmath>

#include "common.cuh"

namespace fgs {

constexpr int kFftMaxStages = 16;
constexpr int kFftThreads = 256;
constexpr int kColGroup = 1;    // columns per CTA in the column pass
constexpr int kColThreads = 128;  // six column CTAs per SM hide the stages' latency
constexpr size_t kSmemMax = 227 * 1024;

struct FftPlan {
  int n, stages;
  int radix[kFftMaxStages];
};

static bool make_plan(int n, FftPlan *p) {
  static const int primes[] = {3, 5, 7, 11, 13, 17};
  p->n = n;
  p->stages = 0;
  int m = n;
  while (m > 1) {
    int r = 0;
    if (m % 8 == 0) r = 8;
    else if (m % 4 == 0) r = 4;
    else if (m % 2 == 0) r = 2;
    else
      for (int q : primes)
        if (m % q == 0) {
          r = q;
          break;
        }
    if (r == 0 || p->stages == kFftMaxStages) return false;
    p->radix[p->stages++] = r;
    m /= r;
  }
  return true;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One radix-P stage for butterfly `b` of a length-N transform whose finished
// sub-transforms have length L.  sign = -1 forward, +1 inverse.  tw[j] holds
// (cos, sin)(2 pi j / N); a twiddle exp(sign 2 pi i e / M) for M dividing N is
// tw[e N / M] with the sine's sign set by `sign`.
// Not inlined: each radix gets its own register allocation instead of the
// union of all radices' arrays inside the calling kernel.
template <int P>
__device__ __noinline__ void fft_butterfly(const float2 *__restrict__ src, float2 *__restrict__ dst, int N,
                                              int L, int b, float sign, int sstride, const float2 *__restrict__ tw) {
  const int s = b / L, k = b - s * L;
  const int Lp = L * P;
  const int NP = N / P;
  const int tstep = N / Lp;
  float2 v[P];
#pragma unroll
  for (int r = 0; r < P; ++r) {
    float2 x = src[(b + r * NP) * sstride];
    if (r > 0 && k > 0) {
      float2 t = tw[r * k * tstep];  // r k < P L: no reduction needed
      t.y *= sign;
      x = cmul(x, t);
    }
    v[r] = x;
  }
  // the P-point DFT's roots of unity: in registers for the small radices, read
  // from the table for the large odd primes (fewer live registers)
  constexpr bool kRegRoots = P <= 8;
  float2 w[kRegRoots ? P : 1];
  if constexpr (kRegRoots) {
#pragma unroll
    for (int m = 0; m < P; ++m) {
      w[m] = tw[m * NP];
      w[m].y *= sign;
    }
  }
  if constexpr (kRegRoots) {
#pragma unroll
    for (int q = 0; q < P; ++q) {
      float2 acc = v[0];
#pragma unroll
      for (int r = 1; r < P; ++r) {
        const float2 t = cmul(v[r], w[(r * q) % P]);
        acc.x += t.x;
        acc.y += t.y;
      }
      dst[(s * Lp + k + L * q) * sstride] = acc;
    }
  } else {
    // the large odd primes: one output per iteration, so the code stays small (a
    // fully unrolled P x P product overflowed the instruction cache); j = r q mod P
#pragma unroll 1
    for (int q = 0; q < P; ++q) {
      float2 acc = v[0];
      int j = 0;
#pragma unroll
      for (int r = 1; r < P; ++r) {
        j += q;
        if (j >= P) j -= P;
        float2 root = tw[j * NP];
        root.y *= sign;
        const float2 t = cmul(v[r], root);
        acc.x += t.x;
        acc.y += t.y;
      }
      dst[(s * Lp + k + L * q) * sstride] = acc;
    }
  }
}

__device__ __forceinline__ void fft_stage(int P, const float2 *src, float2 *dst, int N, int L, int b, float sign,
                                          int sstride, const float2 *tw) {
  switch (P) {
    case 2: fft_butterfly<2>(src, dst, N, L, b, sign, sstride, tw); break;
    case 3: fft_butterfly<3>(src, dst, N, L, b, sign, sstride, tw); break;
    case 4: fft_butterfly<4>(src, dst, N, L, b, sign, sstride, tw); break;
    case 5: fft_butterfly<5>(src, dst, N, L, b, sign, sstride, tw); break;
    case 7: fft_butterfly<7>(src, dst, N, L, b, sign, sstride, tw); break;
    case 8: fft_butterfly<8>(src, dst, N, L, b, sign, sstride, tw); break;
    case 11: fft_butterfly<11>(src, dst, N, L, b, sign, sstride, tw); break;
    case 13: fft_butterfly<13>(src, dst, N, L, b, sign, sstride, tw); break;
    default: fft_butterfly<17>(src, dst, N, L, b, sign, sstride, tw); break;
  }
}

// The table tw[j] = (cos, sin)(2 pi j / N), j < N, by the whole CTA; the caller
// synchronises before it is read.
__device__ __forceinline__ void fft_twiddles(float2 *tw, int N) {
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    float sn, cs;
    sincospif(2.0f * (float)j / (float)N, &sn, &cs);
    tw[j] = make_float2(cs, sn);
  }
}

// Transforms `lanes` independent sequences stored interleaved in shared memory
// (element i of sequence c at (i * lanes + c)); all threads of the CTA take part.
// tw: fft_twiddles(tw, plan.n).  Returns the buffer that holds the result.
__device__ float2 *fft_smem(float2 *a, float2 *b, const FftPlan &plan, int lanes, float sign, const float2 *tw) {
  const int N = plan.n;
  float2 *src = a, *dst = b;
  int L = 1;
  for (int st = 0; st < plan.stages; ++st) {
    const int P = plan.radix[st];
    const int nb = N / P;
    for (int e = threadIdx.x; e < nb * lanes; e += blockDim.x) {
      const int c = e % lanes, bf = e / lanes;
      fft_stage(P, src + c, dst + c, N, L, bf, sign, lanes, tw);
    }
    __syncthreads();
    float2 *t = src;
    src = dst;
    dst = t;
    L *= P;
  }
  return src;
}

// Max E at or below this fraction of the frame's peak |gray| is rounding noise:
// the frame has no high-frequency region (E is exactly 0 in exact arithmetic).
constexpr float kNoiseFloor = 1e-5f;

__device__ __forceinline__ void block_max_to(float v, uint32_t *dst) {
  __shared__ float red[kFftThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(dst, __float_as_uint(m));  // non-negative floats order like their bits
  }
}

// eq2 along x for every row of the gray frame; running max of |gray|.
__global__ void __launch_bounds__(kFftThreads) k_fft_rows(const float *__restrict__ rgb, int W, int H, FftPlan plan,
                                                          float2 *__restrict__ spec, uint32_t *__restrict__ gray_max) {
  pdl_enter();
  extern __shared__ float2 sm2[];
  float2 *a = sm2, *b = sm2 + W, *tw = sm2 + 2 * W;
  const int y = blockIdx.x;
  const int64_t HW = (int64_t)W * H;
  fft_twiddles(tw, W);
  float gm = 0.f;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    const int64_t p = (int64_t)y * W + x;
    const float gray = __fadd_rn(__fadd_rn(__fmul_rn(0.299f, rgb[p]), __fmul_rn(0.587f, rgb[HW + p])),
                                 __fmul_rn(0.114f, rgb[2 * HW + p]));
    a[x] = make_float2(gray, 0.f);
    gm = fmaxf(gm, fabsf(gray));
  }
  block_max_to(gm, gray_max);
  __syncthreads();
  const float2 *r = fft_smem(a, b, plan, 1, -1.f, tw);
  for (int x = threadIdx.x; x < W; x += blockDim.x) spec[(int64_t)y * W + x] = r[x];
}

// Along y for cg columns: forward DFT, eq5/eq7 high-pass at the centred
// frequency (eq3 read as the spectrum shift), inverse DFT.  Only columns
// u = 0 .. W/2 are transformed: the frame is real, so its spectrum is Hermitian,
// F(W - u, H - v) = conj F(u, v), and so is the filtered one (the high-pass is
// even in u and v); after the inverse along y, column W - u is then the complex
// conjugate of column u, and it is written from it.
__global__ void __launch_bounds__(kColThreads, 6) k_fft_cols(float2 *__restrict__ spec, int W, int H, FftPlan plan,
                                                          float d0, int cg) {
  pdl_enter();
  extern __shared__ float2 sm2[];
  float2 *a = sm2, *b = sm2 + H * cg, *tw = sm2 + 2 * H * cg;
  const int x0 = blockIdx.x * cg;
  const int ncol = min(cg, W / 2 + 1 - x0);
  fft_twiddles(tw, H);
  for (int e = threadIdx.x; e < H * cg; e += blockDim.x) {
    const int y = e / cg, c = e - y * cg;
    a[e] = c < ncol ? spec[(int64_t)y * W + x0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 *f = fft_smem(a, b, plan, cg, -1.f, tw);
  const float inv2d2 = 1.0f / (2.0f * d0 * d0);
  const float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
  for (int e = threadIdx.x; e < H * cg; e += blockDim.x) {
    const int v = e / cg, c = e - v * cg;
    const int u = x0 + c;
    // centred coordinates of frequency (u, v): ((u + W/2) mod W) - W/2
    const float du = (float)((u + W / 2) % W - W / 2) / hw;
    const float dv = (float)((v + H / 2) % H - H / 2) / hh;
    const float hp = 1.0f - expf(-(du * du + dv * dv) * inv2d2);
    f[e].x *= hp;
    f[e].y *= hp;
  }
  __syncthreads();
  float2 *other = (f == a) ? b : a;
  float2 *g = fft_smem(f, other, plan, cg, 1.f, tw);
  for (int e = threadIdx.x; e < H * cg; e += blockDim.x) {
    const int y = e / cg, c = e - y * cg;
    if (c < ncol) {
      const int u = x0 + c, m = W - u;  // m: the mirror column
      spec[(int64_t)y * W + u] = g[e];
      if (u > 0 && m > u) spec[(int64_t)y * W + m] = make_float2(g[e].x, -g[e].y);
    }
  }
}

// eq8 along x, E = |I_h| / (H W), and the running maximum of E (E >= 0, so its
// float bits order like unsigned integers).
__global__ void __launch_bounds__(kFftThreads) k_ifft_rows(const float2 *__restrict__ spec, int W, int H,
                                                           FftPlan plan, float *__restrict__ energy,
                                                           uint32_t *__restrict__ max_bits) {
  pdl_enter();
  extern __shared__ float2 sm2[];
  float2 *a = sm2, *b = sm2 + W, *tw = sm2 + 2 * W;
  const int y = blockIdx.x;
  fft_twiddles(tw, W);
  for (int x = threadIdx.x; x < W; x += blockDim.x) a[x] = spec[(int64_t)y * W + x];
  __syncthreads();
  const float2 *r = fft_smem(a, b, plan, 1, 1.f, tw);
  const float scale = 1.0f / ((float)W * (float)H);
  float mx = 0.f;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    const float e = hypotf(r[x].x, r[x].y) * scale;
    energy[(int64_t)y * W + x] = e;
    mx = fmaxf(mx, e);
  }
  block_max_to(mx, max_bits);
}

// max_bits[0] = max E, max_bits[1] = max |gray| (float bits)
__device__ __forceinline__ float energy_floor(const uint32_t *max_bits) {
  return __fmul_rn(kNoiseFloor, __uint_as_float(max_bits[1]));
}

__device__ __forceinline__ int energy_bin(float e, float maxE, float floorE) {
  if (!(maxE > floorE)) return 0;
  const float q = __fdiv_rn(__fmul_rn(256.0f, e), maxE);
  const float f = floorf(q);
  return f >= 255.f ? 255 : (int)f;
}

__global__ void k_hist(const float *__restrict__ energy, int64_t HW, const uint32_t *__restrict__ max_bits,
                       uint32_t *__restrict__ hist) {
  pdl_enter();
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const float maxE = __uint_as_float(*max_bits), floorE = energy_floor(max_bits);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[energy_bin(energy[p], maxE, floorE)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Maximum of a 64-bit key over the 256-thread CTA (every thread gets it).
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long k, unsigned long long *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, k, o);
    k = t > k ? t : k;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
  __syncthreads();
  unsigned long long m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = red[w] > m ? red[w] : m;
  __syncthreads();
  return m;
}

// Triangle method between the peak and the far non-empty end; exact integers.
// One thread per bin: the peak is the first bin of maximal count, lo / hi the
// first and last non-empty bins, e the end further from the peak (hi on a tie);
// t is the first bin, walking from the peak towards e, of maximal distance
// |(e - p)(h[k] - h[p]) - (k - p)(h[e] - h[p])| to the line from (p, h[p]) to
// (e, h[e]) (255 for an empty histogram).
__global__ void __launch_bounds__(256) k_triangle(const uint32_t *__restrict__ hist, int32_t *__restrict__ d_threshold) {
  pdl_enter();
  __shared__ unsigned long long red[8];
  __shared__ uint32_t hv[256];
  __shared__ int s_lo, s_hi;
  const int i = threadIdx.x;
  const uint32_t h = hist[i];
  hv[i] = h;
  if (i == 0) {
    s_lo = 256;
    s_hi = -1;
  }
  __syncthreads();
  if (h > 0) {
    atomicMin(&s_lo, i);
    atomicMax(&s_hi, i);
  }
  // peak: maximal count, then the smallest index
  const unsigned long long pk = block_max_u64(((unsigned long long)h << 8) | (unsigned)(255 - i), red);
  const int p = 255 - (int)(pk & 255u), lo = s_lo, hi = s_hi;
  if (hi < 0) {  // empty histogram
    if (i == 0) *d_threshold = 255;
    return;
  }
  const int e = (hi - p) >= (p - lo) ? hi : lo;
  if (e == p) {
    if (i == 0) *d_threshold = p;
    return;
  }
  const int step = e > p ? 1 : -1;
  const bool on_walk = step > 0 ? (i >= p && i <= e) : (i <= p && i >= e);
  unsigned long long key = 0;
  if (on_walk) {
    const int64_t hp = hv[p], he = hv[e];
    int64_t d = (int64_t)(e - p) * ((int64_t)h - hp) - (int64_t)(i - p) * (he - hp);
    if (d < 0) d = -d;
    // +1 keeps the peak's own d = 0 above the threads off the walk; ties go to the
    // bin nearest the peak
    key = (((unsigned long long)d + 1ull) << 8) | (unsigned)(step > 0 ? 255 - i : i);
  }
  const unsigned long long best = block_max_u64(key, red);
  if (i == 0) {
    const int r = (int)(best & 255u);
    *d_threshold = step > 0 ? 255 - r : r;
  }
}

struct SeedArgs {
  const float *rgb, *depth_gt, *r_color, *r_depth, *r_alpha, *energy;
  int W, H;
  int m, n;
  float tau_alpha, tau_depth_rel, tau_color, alpha_h, alpha_l, init_logit;
  int32_t max_new;
  float fx, fy, cx, cy, R[9], t[3];
  const uint32_t *max_bits;
  const int32_t *threshold;
  uint8_t *mask;
  uint32_t *bsum_hi, *bsum_lo;  // per-CTA counts, scanned in place
  int64_t *base;                // [0] append index, [1] seeds written
  int32_t *seed_xy;             // [max_new][2]
  uint8_t *seed_hi;             // [max_new]
};

constexpr int kSeedBlock = 1024;

// Flags of pixel p: bit0 M_h, bit1 M_l, bit2 M_m, bit4 high seed, bit5 low seed.
__device__ __forceinline__ uint32_t pixel_flags(const SeedArgs &a, int64_t p, int t, float maxE, float floorE) {
  const int64_t HW = (int64_t)a.W * a.H;
  const int x = (int)(p % a.W), y = (int)(p / a.W);
  const bool mh = energy_bin(a.energy[p], maxE, floorE) > t;
  bool mm = true;
  const float dg = a.depth_gt[p];
  if (a.r_alpha) {
    const float A = a.r_alpha[p];
    const bool mi = A < a.tau_alpha;
    bool md = false;
    if (dg > 0.f && A > 0.f) {
      const float diff = __fsub_rn(__fdiv_rn(a.r_depth[p], A), dg);
      md = diff > __fmul_rn(a.tau_depth_rel, dg);
    }
    const float s = __fadd_rn(__fadd_rn(fabsf(__fsub_rn(a.r_color[p], a.rgb[p])),
                                        fabsf(__fsub_rn(a.r_color[HW + p], a.rgb[HW + p]))),
                              fabsf(__fsub_rn(a.r_color[2 * HW + p], a.rgb[2 * HW + p])));
    const bool mc = s > __fmul_rn(3.0f, a.tau_color);
    mm = mi || md || mc;
  }
  const bool valid = dg > 0.f;
  const bool hs = mh && mm && valid && (x % a.m == 0) && (y % a.m == 0);
  const bool ls = !mh && mm && valid && (x % a.n == 0) && (y % a.n == 0);
  return (mh ? 1u : 0u) | (mh ? 0u : 2u) | (mm ? 4u : 0u) | (hs ? 16u : 0u) | (ls ? 32u : 0u);
}

__global__ void __launch_bounds__(kSeedBlock) k_seed_count(SeedArgs a) {
  pdl_enter();
  __shared__ uint32_t red_h[kSeedBlock / 32], red_l[kSeedBlock / 32];
  const int64_t HW = (int64_t)a.W * a.H;
  const int64_t p = blockIdx.x * (int64_t)kSeedBlock + threadIdx.x;
  uint32_t f = 0;
  if (p < HW) {
    f = pixel_flags(a, p, *a.threshold, __uint_as_float(a.max_bits[0]), energy_floor(a.max_bits));
    a.mask[p] = (uint8_t)f;  // the seed bits 4 and 5 stay until k_seed_write replaces them by bit 3
  }
  const uint32_t bh = __ballot_sync(0xffffffffu, f & 16u), bl = __ballot_sync(0xffffffffu, f & 32u);
  if ((threadIdx.x & 31) == 0) {
    red_h[threadIdx.x >> 5] = __popc(bh);
    red_l[threadIdx.x >> 5] = __popc(bl);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t h = 0, l = 0;
    for (int w = 0; w < kSeedBlock / 32; ++w) {
      h += red_h[w];
      l += red_l[w];
    }
    a.bsum_hi[blockIdx.x] = h;
    a.bsum_lo[blockIdx.x] = l;
  }
}

// Exclusive scans of the CTA counts, the capped seed count, the append base.
__global__ void __launch_bounds__(1024) k_seed_scan(SeedArgs a, int nb, int64_t *d_n, int64_t host_n, int64_t cap,
                                                    int32_t *d_num_new, int32_t *d_status) {
  pdl_enter();
  __shared__ uint32_t part_h[1024], part_l[1024];
  const int per = (nb + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  uint32_t sh = 0, sl = 0;
  for (int i = lo; i < hi; ++i) {
    sh += a.bsum_hi[i];
    sl += a.bsum_lo[i];
  }
  part_h[threadIdx.x] = sh;
  part_l[threadIdx.x] = sl;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t vh = threadIdx.x >= off ? part_h[threadIdx.x - off] : 0u;
    const uint32_t vl = threadIdx.x >= off ? part_l[threadIdx.x - off] : 0u;
    __syncthreads();
    part_h[threadIdx.x] += vh;
    part_l[threadIdx.x] += vl;
    __syncthreads();
  }
  uint32_t rh = part_h[threadIdx.x] - sh, rl = part_l[threadIdx.x] - sl;
  for (int i = lo; i < hi; ++i) {
    const uint32_t vh = a.bsum_hi[i], vl = a.bsum_lo[i];
    a.bsum_hi[i] = rh;
    a.bsum_lo[i] = rl;
    rh += vh;
    rl += vl;
  }
  if (threadIdx.x == 1023) {
    const int64_t total_hi = part_h[1023], total = total_hi + part_l[1023];
    int64_t want = total < a.max_new ? total : a.max_new;
    const int64_t base = d_n ? *d_n : host_n;
    int64_t room = cap - base;
    if (room < 0) room = 0;
    if (want > room) {
      want = room;
      if (d_status) atomicOr(d_status, FGS_DEV_MAP_FULL);
    }
    a.base[0] = base;
    a.base[1] = want;
    a.base[2] = total_hi;
    *d_num_new = (int32_t)want;
    if (d_n) *d_n = base + want;
  }
}

__global__ void __launch_bounds__(kSeedBlock) k_seed_write(SeedArgs a, GaussGrads g) {
  pdl_enter();
  __shared__ uint32_t wh[kSeedBlock / 32], wl[kSeedBlock / 32];
  const int64_t HW = (int64_t)a.W * a.H;
  const int64_t p = blockIdx.x * (int64_t)kSeedBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t f = 0;
  if (p < HW) f = a.mask[p];  // k_seed_count's flags
  const bool hs = f & 16u, ls = f & 32u;
  const uint32_t bh = __ballot_sync(0xffffffffu, hs), bl = __ballot_sync(0xffffffffu, ls);
  if (lane == 0) {
    wh[warp] = __popc(bh);
    wl[warp] = __popc(bl);
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t h = wh[lane], l = wl[lane];
    uint32_t ih = h, il = l;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t th = __shfl_up_sync(0xffffffffu, ih, o), tl = __shfl_up_sync(0xffffffffu, il, o);
      if (lane >= o) {
        ih += th;
        il += tl;
      }
    }
    wh[lane] = ih - h;
    wl[lane] = il - l;
  }
  __syncthreads();
  if (!(hs || ls)) return;
  const uint32_t lt = (1u << lane) - 1u;
  int64_t idx;
  if (hs)
    idx = (int64_t)a.bsum_hi[blockIdx.x] + wh[warp] + __popc(bh & lt);
  else
    idx = a.base[2] + (int64_t)a.bsum_lo[blockIdx.x] + wl[warp] + __popc(bl & lt);
  const bool kept = idx < a.base[1];  // else beyond the cap (or the map's room)
  a.mask[p] = (uint8_t)((f & 7u) | (kept ? 8u : 0u));
  if (!kept) return;
  const int x = (int)(p % a.W), y = (int)(p / a.W);
  a.seed_xy[2 * idx] = x;
  a.seed_xy[2 * idx + 1] = y;
  a.seed_hi[idx] = hs ? 1 : 0;
  // eq11: back-projection with the frame's depth, radius alpha d / f
  const float d = a.depth_gt[p];
  const float pcx = ((float)x - a.cx) * d / a.fx, pcy = ((float)y - a.cy) * d / a.fy, pcz = d;
  const float qx = pcx - a.t[0], qy = pcy - a.t[1], qz = pcz - a.t[2];
  const int64_t i = a.base[0] + idx, c = g.cap;
  g.means[i] = a.R[0] * qx + a.R[3] * qy + a.R[6] * qz;
  g.means[c + i] = a.R[1] * qx + a.R[4] * qy + a.R[7] * qz;
  g.means[2 * c + i] = a.R[2] * qx + a.R[5] * qy + a.R[8] * qz;
  const float f_ = 0.5f * (a.fx + a.fy);
  const float ls_ = logf((hs ? a.alpha_h : a.alpha_l) * d / f_);
  g.log_scales[i] = ls_;
  g.log_scales[c + i] = ls_;
  g.log_scales[2 * c + i] = ls_;
  g.quats[i] = 1.f;
  g.quats[c + i] = 0.f;
  g.quats[2 * c + i] = 0.f;
  g.quats[3 * c + i] = 0.f;
  g.logits[i] = a.init_logit;
  g.rgb[i] = a.rgb[p];
  g.rgb[c + i] = a.rgb[HW + p];
  g.rgb[2 * c + i] = a.rgb[2 * HW + p];
}

// Learned prior applied to the seeds just written (prior.cu).
fgs_status prior_apply_to_seeds(const fgs_mlp *mlp, const float *rgb, const float *depth, int W, int H,
                                const int32_t *seed_xy, const uint8_t *seed_hi, const int64_t *base, int64_t max_new,
                                float alpha_h, float alpha_l, float fx, float fy, float max_dev, void *ws,
                                size_t ws_bytes, GaussGrads g, int32_t *d_status, cudaStream_t st);
size_t prior_apply_workspace_size(int64_t max_new);

struct SeedWs {
  float2 *spec;
  float *energy;
  uint32_t *hist, *max_bits;
  uint32_t *bsum_hi, *bsum_lo;
  int64_t *base;
  int32_t *seed_xy;
  uint8_t *seed_hi;
  void *prior;
  size_t prior_bytes, bytes;
};

static SeedWs carve_seed(void *p, int W, int H, int64_t max_new) {
  SeedWs w;
  char *b = static_cast<char *>(p);
  size_t off = 0;
  auto take = [&](size_t n) {
    char *q = b ? b + off : nullptr;
    off += align_up(n);
    return q;
  };
  const size_t HW = (size_t)W * H;
  const size_t nb = (HW + kSeedBlock - 1) / kSeedBlock;
  w.spec = (float2 *)take(HW * sizeof(float2));
  w.energy = (float *)take(HW * sizeof(float));
  w.hist = (uint32_t *)take(258 * 4);
  w.max_bits = w.hist ? w.hist + 256 : nullptr;  // [0] max E, [1] max |gray|
  w.bsum_hi = (uint32_t *)take(nb * 4);
  w.bsum_lo = (uint32_t *)take(nb * 4);
  w.base = (int64_t *)take(4 * 8);
  w.seed_xy = (int32_t *)take((size_t)max_new * 8);
  w.seed_hi = (uint8_t *)take((size_t)max_new);
  w.prior_bytes = prior_apply_workspace_size(max_new);
  w.prior = take(w.prior_bytes);
  w.bytes = off;
  return w;
}

constexpr int64_t kMaxNewLimit = 1 << 22;

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_fourier_seed_workspace_size(int32_t width, int32_t height, int32_t max_new) {
  if (width <= 0 || height <= 0 || max_new < 0 || max_new > kMaxNewLimit) return 0;
  return carve_seed(nullptr, width, height, max_new).bytes;
}

namespace fgs {

// The two halves of fgs_fourier_seed.  Both check the frame size and the
// parameters the same way and carve the same workspace, so the energy map, the
// threshold and the running maximum that the first leaves in the workspace are
// where the second looks for them.
static fgs_status seed_setup(const char *what, const fgs_camera *cam, const fgs_seed_params *prm, void *ws,
                             size_t ws_bytes, FftPlan *px, FftPlan *py, SeedWs *w) {
  FGS_CHECK_ARG(cam && prm, "%s: NULL argument", what);
  const int W = cam->width, H = cam->height;
  FGS_CHECK_ARG(W > 0 && H > 0 && W <= 8192 && H <= 8192, "%s: image size", what);
  FGS_CHECK_ARG(prm->m >= 1 && prm->n >= 1 && prm->max_new >= 0 && prm->max_new <= kMaxNewLimit && prm->d0 > 0,
                "%s: bad parameters", what);
  FGS_CHECK_ARG(ws && (reinterpret_cast<uintptr_t>(ws) & 255) == 0, "%s: workspace alignment", what);
  if (!make_plan(W, px) || !make_plan(H, py)) {
    set_error("%s: %dx%d has a prime factor above 17", what, W, H);
    return FGS_ERR_UNSUPPORTED;
  }
  *w = carve_seed(ws, W, H, prm->max_new);
  FGS_CHECK_ARG(ws_bytes >= w->bytes, "%s: workspace %zu < %zu bytes", what, ws_bytes, w->bytes);
  return FGS_OK;
}

// eq2-eq8 and the threshold: the frame's high-frequency energy E, its histogram
// over E / max E and the triangle threshold.
static fgs_status launch_energy(const float *rgb_gt, const fgs_camera *cam, const fgs_seed_params *prm,
                                const FftPlan &px, const FftPlan &py, const SeedWs &w, float *E,
                                int32_t *d_threshold, cudaStream_t st) {
  const int W = cam->width, H = cam->height;
  const int64_t HW = (int64_t)W * H;
  FGS_CUDA(cudaMemsetAsync(w.hist, 0, 258 * 4, st), "memset hist");
  const size_t smem_row = 3 * (size_t)W * sizeof(float2);  // two buffers + twiddles
  int cg = kColGroup;
  while (cg > 1 && (2 * (size_t)H * cg + H) * sizeof(float2) > kSmemMax) cg >>= 1;
  const size_t smem_col = (2 * (size_t)H * cg + H) * sizeof(float2);
  if (smem_row > 48 * 1024) {
    FGS_CUDA(cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row), "attr");
    FGS_CUDA(cudaFuncSetAttribute(k_ifft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row), "attr");
  }
  if (smem_col > 48 * 1024)
    FGS_CUDA(cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col), "attr");
  pdl_launch(k_fft_rows, H, kFftThreads, smem_row, st, rgb_gt, W, H, px, w.spec, w.max_bits + 1);
  pdl_launch(k_fft_cols, (W / 2 + 1 + cg - 1) / cg, kColThreads, smem_col, st, w.spec, W, H, py, prm->d0, cg);
  pdl_launch(k_ifft_rows, H, kFftThreads, smem_row, st, w.spec, W, H, px, E, w.max_bits);
  pdl_launch(k_hist, 4 * num_sms(), 256, 0, st, E, HW, w.max_bits, w.hist);
  pdl_launch(k_triangle, 1, 256, 0, st, w.hist, d_threshold);
  count_launch(5);
  FGS_CHECK_LAUNCH("fgs_fourier_energy");
  return FGS_OK;
}

// eq9-eq11 (and the learned prior) from E and the threshold.
static fgs_status launch_seeds(const float *rgb_gt, const float *depth_gt, const float *r_color,
                               const float *r_depth, const float *r_alpha, const fgs_camera *cam,
                               const fgs_seed_params *prm, const fgs_mlp *prior, uint8_t *mask, const float *E,
                               fgs_gaussians *g, int32_t *d_num_new, int32_t *d_threshold, int32_t *seed_xy,
                               const SeedWs &w, int32_t *d_status, cudaStream_t st) {
  const int W = cam->width, H = cam->height;
  const int64_t HW = (int64_t)W * H;
  SeedArgs a;
  a.rgb = rgb_gt;
  a.depth_gt = depth_gt;
  a.r_color = r_color;
  a.r_depth = r_depth;
  a.r_alpha = r_alpha;
  a.energy = E;
  a.W = W;
  a.H = H;
  a.m = prm->m;
  a.n = prm->n;
  a.tau_alpha = prm->tau_alpha;
  a.tau_depth_rel = prm->tau_depth_rel;
  a.tau_color = prm->tau_color;
  a.alpha_h = prm->alpha_h;
  a.alpha_l = prm->alpha_l;
  a.init_logit = prm->init_logit;
  a.max_new = prm->max_new;
  a.fx = cam->fx;
  a.fy = cam->fy;
  a.cx = cam->cx;
  a.cy = cam->cy;
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) a.R[3 * r + k] = cam->world_to_cam[4 * r + k];
    a.t[r] = cam->world_to_cam[4 * r + 3];
  }
  a.max_bits = w.max_bits;
  a.threshold = d_threshold;
  a.mask = mask;
  a.bsum_hi = w.bsum_hi;
  a.bsum_lo = w.bsum_lo;
  a.base = w.base;
  a.seed_xy = seed_xy ? seed_xy : w.seed_xy;
  a.seed_hi = w.seed_hi;
  const int nb = (int)((HW + kSeedBlock - 1) / kSeedBlock);
  pdl_launch(k_seed_count, nb, kSeedBlock, 0, st, a);
  pdl_launch(k_seed_scan, 1, 1024, 0, st, a, nb, g->d_n, g->n, g->capacity, d_num_new, d_status);
  pdl_launch(k_seed_write, nb, kSeedBlock, 0, st, a, gauss_grads(g));
  count_launch(3);
  FGS_CHECK_LAUNCH("fgs_fourier_seed seeds");
  if (prior) {
    return prior_apply_to_seeds(prior, rgb_gt, depth_gt, W, H, a.seed_xy, w.seed_hi, w.base, prm->max_new,
                                prm->alpha_h, prm->alpha_l, cam->fx, cam->fy, prm->prior_max_dev, w.prior,
                                w.prior_bytes, gauss_grads(g), d_status, st);
  }
  return FGS_OK;
}

static fgs_status seed_args_ok(const char *what, const float *rgb_gt, const float *depth_gt, const float *r_color,
                               const float *r_depth, const float *r_alpha, uint8_t *mask, const fgs_gaussians *g,
                               int32_t *d_num_new, int32_t *d_threshold) {
  FGS_CHECK_ARG(rgb_gt && depth_gt && mask && d_num_new && d_threshold, "%s: NULL argument", what);
  FGS_CHECK_ARG(!r_alpha || (r_color && r_depth), "%s: r_alpha needs r_color and r_depth", what);
  if (!gaussians_ok(g, "g")) return FGS_ERR_INVALID_ARGUMENT;
  return FGS_OK;
}

}  // namespace fgs

using namespace fgs;

extern "C" fgs_status fgs_fourier_seed(const float *rgb_gt, const float *depth_gt, const float *r_color,
                                       const float *r_depth, const float *r_alpha, const fgs_camera *cam,
                                       const fgs_seed_params *prm, const fgs_mlp *prior, uint8_t *mask,
                                       float *energy, fgs_gaussians *g, int32_t *d_num_new, int32_t *d_threshold,
                                       int32_t *seed_xy, void *ws, size_t ws_bytes, int32_t *d_status,
                                       void *stream) {
  const char *what = "fgs_fourier_seed";
  fgs_status s = seed_args_ok(what, rgb_gt, depth_gt, r_color, r_depth, r_alpha, mask, g, d_num_new, d_threshold);
  if (s != FGS_OK) return s;
  FftPlan px, py;
  SeedWs w;
  if ((s = seed_setup(what, cam, prm, ws, ws_bytes, &px, &py, &w)) != FGS_OK) return s;
  cudaStream_t st = as_stream(stream);
  float *E = energy ? energy : w.energy;
  if ((s = launch_energy(rgb_gt, cam, prm, px, py, w, E, d_threshold, st)) != FGS_OK) return s;
  return launch_seeds(rgb_gt, depth_gt, r_color, r_depth, r_alpha, cam, prm, prior, mask, E, g, d_num_new,
                      d_threshold, seed_xy, w, d_status, st);
}

extern "C" fgs_status fgs_fourier_energy(const float *rgb_gt, const fgs_camera *cam, const fgs_seed_params *prm,
                                         float *energy, int32_t *d_threshold, void *ws, size_t ws_bytes,
                                         void *stream) {
  const char *what = "fgs_fourier_energy";
  FGS_CHECK_ARG(rgb_gt && d_threshold, "%s: NULL argument", what);
  FftPlan px, py;
  SeedWs w;
  fgs_status s = seed_setup(what, cam, prm, ws, ws_bytes, &px, &py, &w);
  if (s != FGS_OK) return s;
  return launch_energy(rgb_gt, cam, prm, px, py, w, energy ? energy : w.energy, d_threshold, as_stream(stream));
}

extern "C" fgs_status fgs_fourier_seed_from_energy(const float *rgb_gt, const float *depth_gt, const float *r_color,
                                                   const float *r_depth, const float *r_alpha,
                                                   const fgs_camera *cam, const fgs_seed_params *prm,
                                                   const fgs_mlp *prior, uint8_t *mask, const float *energy,
                                                   fgs_gaussians *g, int32_t *d_num_new, int32_t *d_threshold,
                                                   int32_t *seed_xy, void *ws, size_t ws_bytes, int32_t *d_status,
                                                   void *stream) {
  const char *what = "fgs_fourier_seed_from_energy";
  fgs_status s = seed_args_ok(what, rgb_gt, depth_gt, r_color, r_depth, r_alpha, mask, g, d_num_new, d_threshold);
  if (s != FGS_OK) return s;
  FftPlan px, py;
  SeedWs w;
  if ((s = seed_setup(what, cam, prm, ws, ws_bytes, &px, &py, &w)) != FGS_OK) return s;
  return launch_seeds(rgb_gt, depth_gt, r_color, r_depth, r_alpha, cam, prm, prior, mask, energy ? energy : w.energy,
                      g, d_num_new, d_threshold, seed_xy, w, d_status, as_stream(stream));
}
