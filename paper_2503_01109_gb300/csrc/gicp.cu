// gicp.cu -- tracking on the sparse map by GICP (Sec. III-B, eq12-eq14).
//
//   k_dp_count / k_dp_scatter     observed points of a depth map (ordered
//                                 compaction of the sampled pixels)
//   k_transform                   R p + t and R C R^T for a device pose
//   k_grid_count / k_grid_fill    counting sort of a cloud into a uniform grid
//   k_voxel_first / k_voxel_*     one point per occupied cell (the lowest index)
//   k_covariances                 k nearest neighbours in the 27 cells around a
//                                 point, sample covariance, Jacobi eigenvectors,
//                                 plane regularisation
//   k_gicp_step                   per source point: nearest target point, eq13's
//                                 combined covariance, the point's share of the
//                                 Gauss-Newton normal equations of eq14 (warp and
//                                 block sums)
//   k_gicp_solve                  one CTA: the 6x6 system in double, the pose
//                                 update, the stop test
//
// Every selection (nearest point, k nearest) orders candidates by (squared
// distance, index), so it does not depend on the order of points inside a cell.
#include <cmath>

#include "common.cuh"

namespace fgs {

constexpr int kGBlock = 256;
constexpr int kMaxK = 32;
constexpr int kSums = 30;  // 21 (J^T M J) + 6 (J^T M d) + cost + correspondences + overlap

// ---------------------------------------------------------------------------------
// helpers

struct GridDev {
  float ox, oy, oz, cell;
  int dx, dy, dz;
};

inline GridDev grid_dev(const fgs_grid &g) {
  return GridDev{g.origin[0], g.origin[1], g.origin[2], g.cell, g.dims[0], g.dims[1], g.dims[2]};
}

inline bool grid_ok(const fgs_grid *g) {
  if (!g || !(g->cell > 0.f) || g->dims[0] < 1 || g->dims[1] < 1 || g->dims[2] < 1) return false;
  const int64_t cells = (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
  return cells <= (int64_t(1) << 26);
}

inline int64_t grid_cells(const fgs_grid &g) { return (int64_t)g.dims[0] * g.dims[1] * g.dims[2]; }

__device__ __forceinline__ bool cell_of(const GridDev &G, float x, float y, float z, int &cx, int &cy, int &cz) {
  const float fx = floorf(__fdiv_rn(__fsub_rn(x, G.ox), G.cell));
  const float fy = floorf(__fdiv_rn(__fsub_rn(y, G.oy), G.cell));
  const float fz = floorf(__fdiv_rn(__fsub_rn(z, G.oz), G.cell));
  // range test in float first: a huge or non-finite coordinate never reaches an int cast
  if (!(fx >= 0.f && fx < (float)G.dx && fy >= 0.f && fy < (float)G.dy && fz >= 0.f && fz < (float)G.dz))
    return false;
  cx = (int)fx;
  cy = (int)fy;
  cz = (int)fz;
  return cx < G.dx && cy < G.dy && cz < G.dz;
}

__device__ __forceinline__ int cell_index(const GridDev &G, int cx, int cy, int cz) {
  return (cz * G.dy + cy) * G.dx + cx;
}

// squared distance, ((dx^2 + dy^2) + dz^2), each operation rounded once
__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ bool before(float d1, int i1, float d2, int i2) { return d1 < d2 || (d1 == d2 && i1 < i2); }

// ---------------------------------------------------------------------------------
// exclusive scan of a uint32 array: block sums, one CTA over the sums, apply

constexpr int kScanChunk = 4096;  // entries per block of the scan (1024 threads x 4)

__global__ void __launch_bounds__(1024) k_scan_sums(const uint32_t *__restrict__ a, int64_t n,
                                                    unsigned long long *__restrict__ sums) {
  pdl_enter();
  __shared__ unsigned long long red[32];
  const int64_t base = blockIdx.x * (int64_t)kScanChunk;
  unsigned long long s = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += 1024)
    if (base + i < n) s += a[base + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 32; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// one CTA: exclusive scan of nb block sums in place, total to *total
__global__ void __launch_bounds__(1024) k_scan_top(unsigned long long *__restrict__ sums, int nb,
                                                   unsigned long long *__restrict__ total) {
  pdl_enter();
  __shared__ unsigned long long part[1024];
  const int per = (nb + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += sums[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    const unsigned long long v = sums[i];
    sums[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) *total = part[1023];
}

// out[i] = exclusive prefix of a (n entries), out[n] = total (out and a distinct)
__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t *__restrict__ a, int64_t n,
                                                     const unsigned long long *__restrict__ sums,
                                                     const unsigned long long *__restrict__ total,
                                                     int32_t *__restrict__ out) {
  pdl_enter();
  __shared__ uint32_t s_val[kScanChunk];
  __shared__ uint32_t s_warp[32];
  const int64_t base = blockIdx.x * (int64_t)kScanChunk;
  for (int i = threadIdx.x; i < kScanChunk; i += 1024) s_val[i] = base + i < n ? a[base + i] : 0u;
  __syncthreads();
  uint32_t v[4], t = 0;  // 4 consecutive entries per thread, then a block scan of the thread sums
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = s_val[4 * threadIdx.x + j];
    t += v[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = s_warp[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    s_warp[lane] = wi - w;
  }
  __syncthreads();
  uint32_t run = (uint32_t)sums[blockIdx.x] + s_warp[warp] + incl - t;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t i = base + 4 * threadIdx.x + j;
    if (i < n) out[i] = (int32_t)run;
    run += v[j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)*total;
}

static fgs_status exclusive_scan(const uint32_t *a, int64_t n, unsigned long long *sums, unsigned long long *total,
                                 int32_t *out, cudaStream_t st) {
  const int64_t nb = std::max<int64_t>(1, (n + kScanChunk - 1) / kScanChunk);
  pdl_launch(k_scan_sums, (unsigned)nb, 1024, 0, st, a, n, sums);
  pdl_launch(k_scan_top, 1, 1024, 0, st, sums, (int)nb, total);
  pdl_launch(k_scan_apply, (unsigned)nb, 1024, 0, st, a, n, sums, total, out);
  count_launch(3);
  FGS_CHECK_LAUNCH("exclusive_scan");
  return FGS_OK;
}

// scratch of an ordered compaction over nb blocks: block counts, their exclusive
// scan (nb + 1 entries) and the scan's block sums
struct CompactWs {
  uint32_t *cnt;
  int32_t *off;
  unsigned long long *sums, *total;
  size_t bytes;
};

static CompactWs compact_carve(void *base, int64_t nb) {
  CompactWs w;
  char *p = static_cast<char *>(base);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char *q = p ? p + o : nullptr;
    o += align_up(std::max<size_t>(bytes, 1));
    return q;
  };
  w.cnt = (uint32_t *)take((size_t)(nb + 1) * 4);
  w.off = (int32_t *)take((size_t)(nb + 1) * 4);
  w.sums = (unsigned long long *)take((size_t)((nb + kScanChunk - 1) / kScanChunk + 1) * 8);
  w.total = (unsigned long long *)take(8);
  w.bytes = o;
  return w;
}

// ---------------------------------------------------------------------------------
// observed points of a depth map

struct DepthSample {
  const float *depth;
  const uint8_t *mask;
  uint8_t bits;
  int W, H, step, sx;
  float fx, fy, cx, cy;
};

__device__ __forceinline__ bool sample_point(const DepthSample &D, int64_t s, float &x, float &y, float &z) {
  const int yy = (int)(s / D.sx), xx = (int)(s - (int64_t)yy * D.sx);
  const int px = xx * D.step, py = yy * D.step;
  const int64_t p = (int64_t)py * D.W + px;
  const float d = D.depth[p];
  if (!(d > 0.f)) return false;
  if (D.mask && (D.mask[p] & D.bits) == 0) return false;
  x = __fmul_rn(__fdiv_rn(__fsub_rn((float)px, D.cx), D.fx), d);
  y = __fmul_rn(__fdiv_rn(__fsub_rn((float)py, D.cy), D.fy), d);
  z = d;
  return true;
}

__global__ void __launch_bounds__(kGBlock) k_dp_count(DepthSample D, int64_t S, uint32_t *__restrict__ bsum) {
  pdl_enter();
  __shared__ uint32_t red[kGBlock / 32];
  const int64_t s = blockIdx.x * (int64_t)kGBlock + threadIdx.x;
  float x, y, z;
  const bool keep = s < S && sample_point(D, s, x, y, z);
  const uint32_t b = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kGBlock / 32; ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kGBlock) k_dp_scatter(DepthSample D, int64_t S, const int32_t *__restrict__ off,
                                                        int64_t nb, float *__restrict__ xyz, int64_t cap,
                                                        int64_t *__restrict__ d_n, int32_t *__restrict__ d_status) {
  pdl_enter();
  __shared__ uint32_t wsum[kGBlock / 32];
  const int64_t s = blockIdx.x * (int64_t)kGBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float x = 0.f, y = 0.f, z = 0.f;
  const bool keep = s < S && sample_point(D, s, x, y, z);
  const uint32_t b = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) wsum[warp] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kGBlock / 32; ++w) {
      const uint32_t t = wsum[w];
      wsum[w] = run;
      run += t;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t total = off[nb];
    *d_n = total < cap ? total : cap;
    if (total > cap && d_status) atomicOr(d_status, FGS_DEV_MAP_FULL);
  }
  if (!keep) return;
  const int64_t pos = (int64_t)off[blockIdx.x] + wsum[warp] + __popc(b & ((1u << lane) - 1u));
  if (pos < cap) {
    xyz[3 * pos] = x;
    xyz[3 * pos + 1] = y;
    xyz[3 * pos + 2] = z;
  }
}

// ---------------------------------------------------------------------------------
// rigid transform of points and covariances

struct PoseF {
  float R[9], t[3];
};

__device__ __forceinline__ PoseF pose_f(const double *__restrict__ P) {
  PoseF T;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) T.R[3 * r + c] = (float)P[4 * r + c];
    T.t[r] = (float)P[4 * r + 3];
  }
  return T;
}

__device__ __forceinline__ void apply_pose(const PoseF &T, float x, float y, float z, float &ox, float &oy,
                                           float &oz) {
  ox = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T.R[0], x), __fmul_rn(T.R[1], y)), __fmul_rn(T.R[2], z)), T.t[0]);
  oy = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T.R[3], x), __fmul_rn(T.R[4], y)), __fmul_rn(T.R[5], z)), T.t[1]);
  oz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T.R[6], x), __fmul_rn(T.R[7], y)), __fmul_rn(T.R[8], z)), T.t[2]);
}

// R C R^T for symmetric C given as (xx, xy, xz, yy, yz, zz)
__device__ __forceinline__ void rotate_cov(const float *R, const float *c, float *o) {
  const float C[9] = {c[0], c[1], c[2], c[1], c[3], c[4], c[2], c[4], c[5]};
  float RC[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) RC[3 * i + j] = R[3 * i] * C[j] + R[3 * i + 1] * C[3 + j] + R[3 * i + 2] * C[6 + j];
  float M[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      M[3 * i + j] = RC[3 * i] * R[3 * j] + RC[3 * i + 1] * R[3 * j + 1] + RC[3 * i + 2] * R[3 * j + 2];
  o[0] = M[0];
  o[1] = 0.5f * (M[1] + M[3]);
  o[2] = 0.5f * (M[2] + M[6]);
  o[3] = M[4];
  o[4] = 0.5f * (M[5] + M[7]);
  o[5] = M[8];
}

// one thread per point: reads its own slots before writing them, so in place is safe
__global__ void k_transform(const float *xyz_in, const float *cov_in, const int64_t *__restrict__ d_n, int64_t n_max,
                            const double *__restrict__ pose, float *xyz_out, float *cov_out) {
  pdl_enter();
  const int64_t n = min(*d_n, n_max);
  const PoseF T = pose_f(pose);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float ox, oy, oz;
    apply_pose(T, xyz_in[3 * i], xyz_in[3 * i + 1], xyz_in[3 * i + 2], ox, oy, oz);
    if (cov_in && cov_out) {
      float c[6], o[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) c[k] = cov_in[6 * i + k];
      rotate_cov(T.R, c, o);
#pragma unroll
      for (int k = 0; k < 6; ++k) cov_out[6 * i + k] = o[k];
    }
    xyz_out[3 * i] = ox;
    xyz_out[3 * i + 1] = oy;
    xyz_out[3 * i + 2] = oz;
  }
}

// ---------------------------------------------------------------------------------
// grid index (counting sort) and voxel downsampling

__global__ void k_grid_count(const float *__restrict__ xyz, const int64_t *__restrict__ d_n, int64_t n_max, GridDev G,
                             uint32_t *__restrict__ count, int32_t *__restrict__ cell_of_pt) {
  pdl_enter();
  const int64_t n = min(*d_n, n_max);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    int c = -1;
    if (cell_of(G, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], cx, cy, cz)) {
      c = cell_index(G, cx, cy, cz);
      atomicAdd(count + c, 1u);
    }
    cell_of_pt[i] = c;
  }
}

__global__ void k_grid_fill(const int64_t *__restrict__ d_n, int64_t n_max, const int32_t *__restrict__ cell_of_pt,
                            const int32_t *__restrict__ cell_start, uint32_t *__restrict__ fill,
                            int32_t *__restrict__ order) {
  pdl_enter();
  const int64_t n = min(*d_n, n_max);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell_of_pt[i];
    if (c >= 0) order[cell_start[c] + (int)atomicAdd(fill + c, 1u)] = (int32_t)i;
  }
}

__global__ void k_voxel_first(const float *__restrict__ xyz, const int64_t *__restrict__ d_n, int64_t n_max,
                              GridDev G, uint32_t *__restrict__ first, int32_t *__restrict__ cell_of_pt) {
  pdl_enter();
  const int64_t n = min(*d_n, n_max);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    int c = -1;
    if (cell_of(G, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], cx, cy, cz)) {
      c = cell_index(G, cx, cy, cz);
      atomicMin(first + c, (uint32_t)i);
    }
    cell_of_pt[i] = c;
  }
}

__device__ __forceinline__ bool voxel_keep(const int32_t *cell_of_pt, const uint32_t *first, int64_t i, int64_t n) {
  if (i >= n) return false;
  const int c = cell_of_pt[i];
  return c >= 0 && first[c] == (uint32_t)i;
}

__global__ void __launch_bounds__(kGBlock) k_voxel_count(const int64_t *__restrict__ d_n, int64_t n_max,
                                                         const int32_t *__restrict__ cell_of_pt,
                                                         const uint32_t *__restrict__ first,
                                                         uint32_t *__restrict__ bsum) {
  pdl_enter();
  __shared__ uint32_t red[kGBlock / 32];
  const int64_t n = min(*d_n, n_max);
  const int64_t i = blockIdx.x * (int64_t)kGBlock + threadIdx.x;
  const uint32_t b = __ballot_sync(0xffffffffu, voxel_keep(cell_of_pt, first, i, n));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kGBlock / 32; ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kGBlock) k_voxel_scatter(const float *__restrict__ xyz,
                                                           const int64_t *__restrict__ d_n, int64_t n_max,
                                                           const int32_t *__restrict__ cell_of_pt,
                                                           const uint32_t *__restrict__ first,
                                                           const int32_t *__restrict__ off, float *__restrict__ out,
                                                           int64_t cap, const int64_t *__restrict__ d_n_out) {
  pdl_enter();
  __shared__ uint32_t wsum[kGBlock / 32];
  __shared__ int64_t s_base;
  const int64_t n = min(*d_n, n_max);
  const int64_t i = blockIdx.x * (int64_t)kGBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool keep = voxel_keep(cell_of_pt, first, i, n);
  const uint32_t b = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) wsum[warp] = __popc(b);
  if (threadIdx.x == 0) s_base = *d_n_out;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kGBlock / 32; ++w) {
      const uint32_t t = wsum[w];
      wsum[w] = run;
      run += t;
    }
  }
  __syncthreads();
  if (!keep) return;
  const int64_t pos = s_base + off[blockIdx.x] + wsum[warp] + __popc(b & ((1u << lane) - 1u));
  if (pos < cap) {
    out[3 * pos] = xyz[3 * i];
    out[3 * pos + 1] = xyz[3 * i + 1];
    out[3 * pos + 2] = xyz[3 * i + 2];
  }
}

__global__ void k_voxel_finish(const int32_t *__restrict__ off, int64_t nb, int64_t cap, int64_t *__restrict__ d_n_out,
                               int32_t *__restrict__ d_status) {
  pdl_enter();
  const int64_t total = *d_n_out + off[nb];
  *d_n_out = total < cap ? total : cap;
  if (total > cap && d_status) atomicOr(d_status, FGS_DEV_MAP_FULL);
}

// ---------------------------------------------------------------------------------
// covariances

// Eigen-decomposition of a symmetric 3x3 (a00 a01 a02 a11 a12 a22) by cyclic
// Jacobi rotations: eigenvalues on the diagonal, eigenvectors in V's columns.
__device__ void jacobi3(const float a[6], float V[9], float ev[3]) {
  float A[3][3] = {{a[0], a[1], a[2]}, {a[1], a[3], a[4]}, {a[2], a[4], a[5]}};
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.f : 0.f;
  for (int sweep = 0; sweep < 10; ++sweep) {
    const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
    if (off == 0.f) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      if (A[p][q] == 0.f) continue;
      const float theta = 0.5f * (A[q][q] - A[p][p]) / A[p][q];
      const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      const float c = 1.f / sqrtf(t * t + 1.f), s = t * c;
      for (int k = 0; k < 3; ++k) {  // A <- A J
        const float akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {  // A <- J^T A
        const float apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {  // V <- V J
        const float vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - s * vkq;
        V[3 * k + q] = s * vkp + c * vkq;
      }
    }
  }
  ev[0] = A[0][0];
  ev[1] = A[1][1];
  ev[2] = A[2][2];
}

__global__ void __launch_bounds__(128) k_covariances(const float *__restrict__ xyz, const int64_t *__restrict__ d_n,
                                                     int64_t n_max, GridDev G, const int32_t *__restrict__ cell_start,
                                                     const int32_t *__restrict__ order, int k, float eps,
                                                     float *__restrict__ cov) {
  pdl_enter();
  const int64_t n = min(*d_n, n_max);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2];
  const float r2 = __fmul_rn(G.cell, G.cell);
  float bd[kMaxK];
  int bi[kMaxK];
  int m = 0;  // neighbours found, sorted by (d2, index)
  int cx, cy, cz;
  if (cell_of(G, px, py, pz, cx, cy, cz)) {
    for (int z = max(cz - 1, 0); z <= min(cz + 1, G.dz - 1); ++z)
      for (int y = max(cy - 1, 0); y <= min(cy + 1, G.dy - 1); ++y)
        for (int x = max(cx - 1, 0); x <= min(cx + 1, G.dx - 1); ++x) {
          const int c = cell_index(G, x, y, z);
          for (int e = cell_start[c]; e < cell_start[c + 1]; ++e) {
            const int j = order[e];
            const float d2 = dist2(px, py, pz, xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]);
            if (d2 > r2) continue;
            if (m == k && !before(d2, j, bd[k - 1], bi[k - 1])) continue;
            int pos = m < k ? m : k - 1;  // insertion from the back (drops the last when full)
            while (pos > 0 && before(d2, j, bd[pos - 1], bi[pos - 1])) {
              bd[pos] = bd[pos - 1];
              bi[pos] = bi[pos - 1];
              --pos;
            }
            bd[pos] = d2;
            bi[pos] = j;
            if (m < k) ++m;
          }
        }
  }
  float out[6] = {1.f, 0.f, 0.f, 1.f, 0.f, 1.f};
  if (m >= 3) {
    float mx = 0.f, my = 0.f, mz = 0.f;
    for (int a = 0; a < m; ++a) {
      const int j = bi[a];
      mx += xyz[3 * j];
      my += xyz[3 * j + 1];
      mz += xyz[3 * j + 2];
    }
    const float inv = 1.f / (float)m;
    mx *= inv;
    my *= inv;
    mz *= inv;
    float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < m; ++a) {
      const int j = bi[a];
      const float dx = xyz[3 * j] - mx, dy = xyz[3 * j + 1] - my, dz = xyz[3 * j + 2] - mz;
      c[0] += dx * dx;
      c[1] += dx * dy;
      c[2] += dx * dz;
      c[3] += dy * dy;
      c[4] += dy * dz;
      c[5] += dz * dz;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) c[q] *= inv;
    float V[9], ev[3];
    jacobi3(c, V, ev);
    int s = 0;  // smallest eigenvalue
    if (ev[1] < ev[s]) s = 1;
    if (ev[2] < ev[s]) s = 2;
    const float nx = V[s], ny = V[3 + s], nz = V[6 + s];
    const float w = 1.f - eps;  // eps n n^T + (I - n n^T) = I - (1 - eps) n n^T
    out[0] = 1.f - w * nx * nx;
    out[1] = -w * nx * ny;
    out[2] = -w * nx * nz;
    out[3] = 1.f - w * ny * ny;
    out[4] = -w * ny * nz;
    out[5] = 1.f - w * nz * nz;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) cov[6 * i + q] = out[q];
}

// ---------------------------------------------------------------------------------
// Gauss-Newton on eq14

struct GicpCtl {
  int32_t done;        // set once |xi| fell below the stop threshold or the system degenerated
  int32_t iterations;  // steps run
};

// adjugate / determinant of a symmetric 3x3 (xx xy xz yy yz zz)
__device__ __forceinline__ void inverse_sym3(const float *c, float *m) {
  const float a = c[0], b = c[1], d = c[2], e = c[3], f = c[4], g = c[5];
  const float A = e * g - f * f, B = -(b * g - f * d), C = b * f - e * d;
  const float det = a * A + b * B + d * C;
  const float r = 1.f / det;
  m[0] = A * r;
  m[1] = B * r;
  m[2] = C * r;
  m[3] = (a * g - d * d) * r;
  m[4] = -(a * f - b * d) * r;
  m[5] = (a * e - b * b) * r;
}

__global__ void __launch_bounds__(kGBlock) k_gicp_step(const float *__restrict__ src, const float *__restrict__ src_cov,
                                                       const int64_t *__restrict__ d_n_src, int64_t n_max,
                                                       const float *__restrict__ tgt, const float *__restrict__ tgt_cov,
                                                       GridDev G, const int32_t *__restrict__ cell_start,
                                                       const int32_t *__restrict__ order,
                                                       const double *__restrict__ pose, float max_dist,
                                                       float overlap_dist, const GicpCtl *__restrict__ ctl,
                                                       double *__restrict__ partials) {
  pdl_enter();
  __shared__ float s_red[kGBlock / 32][kSums];
  if (ctl->done) return;
  const int64_t n = min(*d_n_src, n_max);
  const int64_t i = blockIdx.x * (int64_t)kGBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float v[kSums];
#pragma unroll
  for (int q = 0; q < kSums; ++q) v[q] = 0.f;
  if (i < n) {
    const PoseF T = pose_f(pose);
    float px, py, pz;
    apply_pose(T, src[3 * i], src[3 * i + 1], src[3 * i + 2], px, py, pz);
    const float md2 = __fmul_rn(max_dist, max_dist), od2 = __fmul_rn(overlap_dist, overlap_dist);
    float best = INFINITY;
    int bj = -1;
    int cx, cy, cz;
    if (cell_of(G, px, py, pz, cx, cy, cz)) {
      for (int z = max(cz - 1, 0); z <= min(cz + 1, G.dz - 1); ++z)
        for (int y = max(cy - 1, 0); y <= min(cy + 1, G.dy - 1); ++y)
          for (int x = max(cx - 1, 0); x <= min(cx + 1, G.dx - 1); ++x) {
            const int c = cell_index(G, x, y, z);
            for (int e = cell_start[c]; e < cell_start[c + 1]; ++e) {
              const int j = order[e];
              const float d2 = dist2(px, py, pz, tgt[3 * j], tgt[3 * j + 1], tgt[3 * j + 2]);
              if (before(d2, j, best, bj)) {
                best = d2;
                bj = j;
              }
            }
          }
    }
    if (bj >= 0 && best <= od2) v[29] = 1.f;
    if (bj >= 0 && best <= md2) {
      const float d[3] = {tgt[3 * bj] - px, tgt[3 * bj + 1] - py, tgt[3 * bj + 2] - pz};
      float cp[6], cr[6], cs[6], M[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) cp[q] = src_cov[6 * i + q];
      rotate_cov(T.R, cp, cr);
#pragma unroll
      for (int q = 0; q < 6; ++q) cs[q] = tgt_cov[6 * bj + q] + cr[q];
      inverse_sym3(cs, M);
      const float Mf[9] = {M[0], M[1], M[2], M[1], M[3], M[4], M[2], M[4], M[5]};
      // J = [[p]_x, -I]: d(xi) = d + [p]_x w - v for T <- (Rodrigues(w), v) T
      const float J[3][6] = {{0.f, -pz, py, -1.f, 0.f, 0.f}, {pz, 0.f, -px, 0.f, -1.f, 0.f},
                             {-py, px, 0.f, 0.f, 0.f, -1.f}};
      float MJ[3][6], Md[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Md[a] = Mf[3 * a] * d[0] + Mf[3 * a + 1] * d[1] + Mf[3 * a + 2] * d[2];
#pragma unroll
        for (int c = 0; c < 6; ++c)
          MJ[a][c] = Mf[3 * a] * J[0][c] + Mf[3 * a + 1] * J[1][c] + Mf[3 * a + 2] * J[2][c];
      }
      int q = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) v[q++] = J[0][r] * MJ[0][c] + J[1][r] * MJ[1][c] + J[2][r] * MJ[2][c];
#pragma unroll
      for (int r = 0; r < 6; ++r) v[21 + r] = J[0][r] * Md[0] + J[1][r] * Md[1] + J[2][r] * Md[2];
      v[27] = d[0] * Md[0] + d[1] * Md[1] + d[2] * Md[2];
      v[28] = 1.f;
    }
  }
#pragma unroll
  for (int q = 0; q < kSums; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < kSums; ++q) s_red[warp][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < kSums) {
    double s = 0.0;
    for (int w = 0; w < kGBlock / 32; ++w) s += (double)s_red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kSums + threadIdx.x] = s;
  }
}

// 6x6 solve by Cholesky (H = L L^T); false when H is not positive definite
__device__ bool cholesky_solve6(const double (&H)[6][6], const double *b, double *x) {
  double L[6][6] = {};
  for (int j = 0; j < 6; ++j) {
    double s = H[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) return false;
    L[j][j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = H[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < 6; ++k) t -= L[k][i] * x[k];
    x[i] = t / L[i][i];
  }
  return true;
}

__global__ void __launch_bounds__(64) k_gicp_solve(const double *__restrict__ partials, int nb,
                                                   const int64_t *__restrict__ d_n_src, int64_t n_max,
                                                   double *__restrict__ pose, GicpCtl *__restrict__ ctl,
                                                   double *__restrict__ stats) {
  pdl_enter();
  __shared__ double s[kSums];
  if (ctl->done) return;
  if (threadIdx.x < kSums) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partials[(int64_t)b * kSums + threadIdx.x];
    s[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int64_t n = min(*d_n_src, n_max);
  stats[0] = s[27];
  stats[1] = s[28];
  stats[2] = n > 0 ? s[29] / (double)n : 0.0;
  ctl->iterations += 1;
  stats[3] = (double)ctl->iterations;
  double H[6][6];
  int q = 0;
  for (int r = 0; r < 6; ++r)
    for (int c = r; c < 6; ++c) {
      H[r][c] = H[c][r] = s[q];
      ++q;
    }
  double rhs[6], xi[6];
  for (int r = 0; r < 6; ++r) rhs[r] = -s[21 + r];
  if (s[28] < 6.0 || !cholesky_solve6(H, rhs, xi)) {
    ctl->done = 1;  // too few correspondences or a degenerate system: keep the pose
    return;
  }
  // T <- (Rodrigues(w), v) T
  const double wx = xi[0], wy = xi[1], wz = xi[2];
  const double th = sqrt(wx * wx + wy * wy + wz * wz);
  double Rw[9];
  if (th < 1e-12) {
    const double I[9] = {1, -wz, wy, wz, 1, -wx, -wy, wx, 1};
    for (int k = 0; k < 9; ++k) Rw[k] = I[k];
  } else {
    const double kx = wx / th, ky = wy / th, kz = wz / th, c = cos(th), sn = sin(th), v1 = 1.0 - c;
    Rw[0] = c + kx * kx * v1;
    Rw[1] = kx * ky * v1 - kz * sn;
    Rw[2] = kx * kz * v1 + ky * sn;
    Rw[3] = ky * kx * v1 + kz * sn;
    Rw[4] = c + ky * ky * v1;
    Rw[5] = ky * kz * v1 - kx * sn;
    Rw[6] = kz * kx * v1 - ky * sn;
    Rw[7] = kz * ky * v1 + kx * sn;
    Rw[8] = c + kz * kz * v1;
  }
  double P[12];
  for (int k = 0; k < 12; ++k) P[k] = pose[k];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      pose[4 * r + c] = Rw[3 * r] * P[c] + Rw[3 * r + 1] * P[4 + c] + Rw[3 * r + 2] * P[8 + c];
    pose[4 * r + 3] = Rw[3 * r] * P[3] + Rw[3 * r + 1] * P[7] + Rw[3 * r + 2] * P[11] + xi[3 + r];
  }
  double nrm = 0.0;
  for (int r = 0; r < 6; ++r) nrm += xi[r] * xi[r];
  if (sqrt(nrm) < 1e-6) ctl->done = 1;
}

__global__ void k_gicp_init(GicpCtl *ctl, double *stats) {
  pdl_enter();
  ctl->done = 0;
  ctl->iterations = 0;
  for (int k = 0; k < 4; ++k) stats[k] = 0.0;
}

// voxel downsampling scratch: per-cell lowest index, per-point cell, compaction
struct VoxelWs {
  uint32_t *first;
  int32_t *cell_of_pt;
  CompactWs c;
  size_t bytes;
};

static VoxelWs voxel_carve(void *base, const fgs_grid &g, int64_t n_max) {
  VoxelWs w;
  char *p = static_cast<char *>(base);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char *q = p ? p + o : nullptr;
    o += align_up(std::max<size_t>(bytes, 1));
    return q;
  };
  w.first = (uint32_t *)take((size_t)grid_cells(g) * 4);
  w.cell_of_pt = (int32_t *)take((size_t)std::max<int64_t>(n_max, 1) * 4);
  const int64_t nb = (std::max<int64_t>(n_max, 1) + kGBlock - 1) / kGBlock;
  w.c = compact_carve(p ? p + o : nullptr, nb);
  o += w.c.bytes;
  w.bytes = o;
  return w;
}

// grid build scratch: per-cell counts and fill cursors, per-point cell, scan sums
struct GridWs {
  uint32_t *count, *fill;
  int32_t *cell_of_pt;
  unsigned long long *sums, *total;
  size_t bytes;
};

static GridWs grid_carve(void *base, const fgs_grid &g, int64_t n_max) {
  GridWs w;
  char *p = static_cast<char *>(base);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char *q = p ? p + o : nullptr;
    o += align_up(std::max<size_t>(bytes, 1));
    return q;
  };
  const int64_t cells = grid_cells(g);
  w.count = (uint32_t *)take((size_t)cells * 4);
  w.fill = (uint32_t *)take((size_t)cells * 4);
  w.cell_of_pt = (int32_t *)take((size_t)std::max<int64_t>(n_max, 1) * 4);
  w.sums = (unsigned long long *)take((size_t)((cells + kScanChunk - 1) / kScanChunk + 1) * 8);
  w.total = (unsigned long long *)take(8);
  w.bytes = o;
  return w;
}

// gicp scratch: per-block partial sums and the control word
static size_t gicp_carve(int64_t n_src_max, double **partials, GicpCtl **ctl, void *base) {
  const int64_t nb = std::max<int64_t>(1, (n_src_max + kGBlock - 1) / kGBlock);
  char *p = static_cast<char *>(base);
  const size_t a = align_up((size_t)nb * kSums * 8);
  if (p) {
    *partials = reinterpret_cast<double *>(p);
    *ctl = reinterpret_cast<GicpCtl *>(p + a);
  }
  return a + align_up(sizeof(GicpCtl));
}

static int64_t dp_blocks(int32_t W, int32_t H, int32_t step) {
  const int64_t S = (int64_t)((W + step - 1) / step) * ((H + step - 1) / step);
  return (S + kGBlock - 1) / kGBlock;
}

}  // namespace fgs

using namespace fgs;

// ---------------------------------------------------------------------------------
// entry points

extern "C" size_t fgs_depth_points_workspace_size(int32_t width, int32_t height, int32_t step) {
  if (width <= 0 || height <= 0 || step < 1) return 0;
  return compact_carve(nullptr, dp_blocks(width, height, step)).bytes;
}

extern "C" fgs_status fgs_depth_points(const float *depth, const uint8_t *mask, uint8_t mask_bits,
                                       const fgs_camera *cam, int32_t step, float *xyz, int64_t capacity,
                                       int64_t *d_n, void *ws, size_t ws_bytes, int32_t *d_status, void *stream) {
  FGS_CHECK_ARG(depth && cam && xyz && d_n, "fgs_depth_points: NULL argument");
  FGS_CHECK_ARG(step >= 1 && capacity >= 1, "fgs_depth_points: step and capacity must be >= 1");
  FGS_CHECK_ARG(cam->width > 0 && cam->height > 0 && cam->fx > 0 && cam->fy > 0, "fgs_depth_points: camera");
  DepthSample D{depth, mask, mask_bits, cam->width, cam->height, step, (cam->width + step - 1) / step,
                cam->fx, cam->fy, cam->cx, cam->cy};
  const int64_t S = (int64_t)D.sx * ((cam->height + step - 1) / step);
  const int64_t nb = dp_blocks(cam->width, cam->height, step);
  CompactWs w = compact_carve(ws, nb);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= w.bytes, "fgs_depth_points: workspace %zu < %zu bytes", ws_bytes,
                w.bytes);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fgs_depth_points: workspace not 256-byte aligned");
  cudaStream_t st = as_stream(stream);
  pdl_launch(k_dp_count, (unsigned)nb, kGBlock, 0, st, D, S, w.cnt);
  count_launch();
  fgs_status s = exclusive_scan(w.cnt, nb, w.sums, w.total, w.off, st);
  if (s != FGS_OK) return s;
  pdl_launch(k_dp_scatter, (unsigned)nb, kGBlock, 0, st, D, S, w.off, nb, xyz, capacity, d_n, d_status);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_depth_points");
  return FGS_OK;
}

extern "C" fgs_status fgs_transform_points(const float *xyz_in, const float *cov_in, const int64_t *d_n,
                                           int64_t n_max, const double *d_pose, float *xyz_out, float *cov_out,
                                           void *stream) {
  FGS_CHECK_ARG(xyz_in && xyz_out && d_n && d_pose, "fgs_transform_points: NULL argument");
  FGS_CHECK_ARG((cov_in == nullptr) == (cov_out == nullptr), "fgs_transform_points: both covariances or neither");
  if (n_max <= 0) return FGS_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((n_max + 255) / 256, 8 * num_sms());
  pdl_launch(k_transform, blocks, 256, 0, as_stream(stream), xyz_in, cov_in, d_n, n_max, d_pose, xyz_out, cov_out);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_transform_points");
  return FGS_OK;
}

extern "C" size_t fgs_voxel_workspace_size(const fgs_grid *grid, int64_t n_max) {
  if (!grid_ok(grid) || n_max < 0) return 0;
  return voxel_carve(nullptr, *grid, n_max).bytes;
}

extern "C" fgs_status fgs_voxel_downsample(const float *xyz, const int64_t *d_n, int64_t n_max, const fgs_grid *grid,
                                           void *ws, size_t ws_bytes, float *out_xyz, int64_t out_capacity,
                                           int64_t *d_n_out, int32_t *d_status, void *stream) {
  FGS_CHECK_ARG(xyz && d_n && out_xyz && d_n_out, "fgs_voxel_downsample: NULL argument");
  FGS_CHECK_ARG(grid_ok(grid), "fgs_voxel_downsample: bad grid");
  FGS_CHECK_ARG(n_max >= 0 && n_max < 0x7FFFFFFFll && out_capacity >= 1, "fgs_voxel_downsample: sizes");
  VoxelWs w = voxel_carve(ws, *grid, n_max);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= w.bytes, "fgs_voxel_downsample: workspace %zu < %zu bytes", ws_bytes,
                w.bytes);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0,
                "fgs_voxel_downsample: workspace not 256-byte aligned");
  if (n_max == 0) return FGS_OK;
  cudaStream_t st = as_stream(stream);
  const GridDev G = grid_dev(*grid);
  FGS_CUDA(cudaMemsetAsync(w.first, 0xFF, (size_t)grid_cells(*grid) * 4, st), "voxel first");
  const int64_t nb = (n_max + kGBlock - 1) / kGBlock;
  const unsigned gblocks = (unsigned)std::min<int64_t>(nb, 8 * num_sms());
  pdl_launch(k_voxel_first, gblocks, kGBlock, 0, st, xyz, d_n, n_max, G, w.first, w.cell_of_pt);
  pdl_launch(k_voxel_count, (unsigned)nb, kGBlock, 0, st, d_n, n_max, w.cell_of_pt, w.first, w.c.cnt);
  count_launch(2);
  fgs_status s = exclusive_scan(w.c.cnt, nb, w.c.sums, w.c.total, w.c.off, st);
  if (s != FGS_OK) return s;
  pdl_launch(k_voxel_scatter, (unsigned)nb, kGBlock, 0, st, xyz, d_n, n_max, w.cell_of_pt, w.first, w.c.off, out_xyz,
             out_capacity, d_n_out);
  pdl_launch(k_voxel_finish, 1, 1, 0, st, w.c.off, nb, out_capacity, d_n_out, d_status);
  count_launch(2);
  FGS_CHECK_LAUNCH("fgs_voxel_downsample");
  return FGS_OK;
}

extern "C" size_t fgs_grid_workspace_size(const fgs_grid *grid, int64_t n_max) {
  if (!grid_ok(grid) || n_max < 0) return 0;
  return grid_carve(nullptr, *grid, n_max).bytes;
}

extern "C" fgs_status fgs_grid_build(const float *xyz, const int64_t *d_n, int64_t n_max, const fgs_grid *grid,
                                     int32_t *cell_start, int32_t *order, void *ws, size_t ws_bytes, void *stream) {
  FGS_CHECK_ARG(xyz && d_n && cell_start && order, "fgs_grid_build: NULL argument");
  FGS_CHECK_ARG(grid_ok(grid), "fgs_grid_build: bad grid");
  FGS_CHECK_ARG(n_max >= 0 && n_max < 0x7FFFFFFFll, "fgs_grid_build: n_max");
  GridWs w = grid_carve(ws, *grid, n_max);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= w.bytes, "fgs_grid_build: workspace %zu < %zu bytes", ws_bytes,
                w.bytes);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fgs_grid_build: workspace not 256-byte aligned");
  cudaStream_t st = as_stream(stream);
  const int64_t cells = grid_cells(*grid);
  const GridDev G = grid_dev(*grid);
  FGS_CUDA(cudaMemsetAsync(w.count, 0, (size_t)cells * 4, st), "grid count");
  FGS_CUDA(cudaMemsetAsync(w.fill, 0, (size_t)cells * 4, st), "grid fill");
  const unsigned gblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_max + 255) / 256, 8 * num_sms()));
  pdl_launch(k_grid_count, gblocks, 256, 0, st, xyz, d_n, n_max, G, w.count, w.cell_of_pt);
  count_launch();
  fgs_status s = exclusive_scan(w.count, cells, w.sums, w.total, cell_start, st);
  if (s != FGS_OK) return s;
  pdl_launch(k_grid_fill, gblocks, 256, 0, st, d_n, n_max, w.cell_of_pt, cell_start, w.fill, order);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_grid_build");
  return FGS_OK;
}

extern "C" fgs_status fgs_point_covariances(const float *xyz, const int64_t *d_n, int64_t n_max, const fgs_grid *grid,
                                            const int32_t *cell_start, const int32_t *order, int32_t k, float eps,
                                            float *cov, void *stream) {
  FGS_CHECK_ARG(xyz && d_n && cell_start && order && cov, "fgs_point_covariances: NULL argument");
  FGS_CHECK_ARG(grid_ok(grid), "fgs_point_covariances: bad grid");
  FGS_CHECK_ARG(k >= 3 && k <= kMaxK, "fgs_point_covariances: k must be 3..%d", kMaxK);
  if (n_max <= 0) return FGS_OK;
  pdl_launch(k_covariances, (unsigned)((n_max + 127) / 128), 128, 0, as_stream(stream), xyz, d_n, n_max,
             grid_dev(*grid), cell_start, order, k, eps, cov);
  count_launch();
  FGS_CHECK_LAUNCH("fgs_point_covariances");
  return FGS_OK;
}

extern "C" size_t fgs_gicp_workspace_size(int64_t n_src_max) {
  if (n_src_max < 0) return 0;
  return gicp_carve(n_src_max, nullptr, nullptr, nullptr);
}

extern "C" fgs_status fgs_gicp(const float *src_xyz, const float *src_cov, const int64_t *d_n_src, int64_t n_src_max,
                               const float *tgt_xyz, const float *tgt_cov, const fgs_grid *grid,
                               const int32_t *cell_start, const int32_t *order, const fgs_gicp_params *p,
                               double *d_pose, double *d_stats, void *ws, size_t ws_bytes, void *stream) {
  FGS_CHECK_ARG(src_xyz && src_cov && d_n_src && tgt_xyz && tgt_cov && cell_start && order && p && d_pose &&
                    d_stats,
                "fgs_gicp: NULL argument");
  FGS_CHECK_ARG(grid_ok(grid), "fgs_gicp: bad grid");
  FGS_CHECK_ARG(p->iterations >= 1 && p->iterations <= 1000 && p->max_dist > 0.f && p->max_dist <= grid->cell &&
                    p->overlap_dist > 0.f && p->overlap_dist <= grid->cell,
                "fgs_gicp: 1 <= iterations <= 1000 and 0 < max_dist, overlap_dist <= the grid's cell");
  FGS_CHECK_ARG(n_src_max >= 1 && n_src_max < 0x7FFFFFFFll, "fgs_gicp: n_src_max");
  double *partials = nullptr;
  GicpCtl *ctl = nullptr;
  const size_t need = gicp_carve(n_src_max, &partials, &ctl, ws);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= need, "fgs_gicp: workspace %zu < %zu bytes", ws_bytes, need);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fgs_gicp: workspace not 256-byte aligned");
  cudaStream_t st = as_stream(stream);
  const int nb = (int)((n_src_max + kGBlock - 1) / kGBlock);
  const GridDev G = grid_dev(*grid);
  pdl_launch(k_gicp_init, 1, 1, 0, st, ctl, d_stats);
  count_launch();
  for (int it = 0; it < p->iterations; ++it) {
    pdl_launch(k_gicp_step, nb, kGBlock, 0, st, src_xyz, src_cov, d_n_src, n_src_max, tgt_xyz, tgt_cov, G, cell_start,
               order, d_pose, p->max_dist, p->overlap_dist, ctl, partials);
    pdl_launch(k_gicp_solve, 1, 64, 0, st, partials, nb, d_n_src, n_src_max, d_pose, ctl, d_stats);
    count_launch(2);
  }
  FGS_CHECK_LAUNCH("fgs_gicp");
  return FGS_OK;
}
