// prune.cu -- Gaussian pruning (Sec. III-A, "Gaussian Pruning"): the Gaussians
// that grew too large in some dimension or whose opacity fell below a threshold
// are removed, together with their Adam moments.  With K survivors, the
// survivors below index K stay in place and each removed slot below K, lowest
// first, receives a survivor from index K on, highest first: only as many
// Gaussians move as there are slots to fill (the paper fixes no storage order).
//
//   k_prune_count   per block of 1024 Gaussians: survivors
//   k_prune_scan    one CTA: exclusive scan of the block counts, the new count K
//   k_prune_index   survivors before each Gaussian give its rank among the removed
//                   slots below K (hole list) or among the survivors from K on
//                   (mover list, counted from the top)
//   k_prune_move    mover h -> hole h for every plane of the map and its moments
//
// A mover sits at or above K and its hole below K, so the moves never overlap
// and need no scratch copy.
#include "common.cuh"

namespace fgs {

constexpr int kPruneBlock = 1024;

struct PruneScratch {
  uint32_t *bsum;   // ceil(cap / 1024) + 1
  int64_t *ctl;     // [0] new count K, [1] slots to fill, [2] live count before
  uint32_t *hole;   // cap: removed slots below K, lowest first
  uint32_t *mover;  // cap: survivors from K on, highest first
  size_t bytes;
};

static PruneScratch prune_carve(void *base, int64_t cap) {
  PruneScratch w;
  char *p = static_cast<char *>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *q = p ? p + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1));
    return q;
  };
  cap = std::max<int64_t>(cap, 1);
  w.bsum = (uint32_t *)take((size_t)((cap + kPruneBlock - 1) / kPruneBlock + 1) * 4);
  w.ctl = (int64_t *)take(24);
  w.hole = (uint32_t *)take((size_t)cap * 4);
  w.mover = (uint32_t *)take((size_t)cap * 4);
  w.bytes = off;
  return w;
}

__device__ __forceinline__ bool survives(const float *__restrict__ ls, const float *__restrict__ logit, int64_t cap,
                                         int64_t i, float min_logit, float max_log_scale) {
  const float m = fmaxf(fmaxf(ls[i], ls[cap + i]), ls[2 * cap + i]);
  return !(logit[i] < min_logit) && !(m > max_log_scale);
}

__global__ void __launch_bounds__(kPruneBlock) k_prune_count(const float *__restrict__ ls,
                                                             const float *__restrict__ logit, int64_t cap,
                                                             float min_logit, float max_log_scale,
                                                             uint32_t *__restrict__ bsum, int64_t *__restrict__ ctl) {
  pdl_enter();
  __shared__ uint32_t red[kPruneBlock / 32];
  const int64_t live = ctl[2];
  const int64_t i = blockIdx.x * (int64_t)kPruneBlock + threadIdx.x;
  const bool in = i < live;
  const bool keep = in && survives(ls, logit, cap, i, min_logit, max_log_scale);
  const uint32_t b = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

// ctl[1] (slots to fill) is counted by k_prune_index; ctl[2] keeps the live count
// the whole call works on.
__global__ void k_prune_init(const int64_t *d_n, int64_t n, int64_t *ctl) {
  pdl_enter();
  ctl[0] = 0;
  ctl[1] = 0;
  ctl[2] = live_count(d_n, n);
}

__global__ void k_prune_finish(const int64_t *__restrict__ ctl, int64_t *__restrict__ d_n) {
  pdl_enter();
  *d_n = ctl[0];
}

__global__ void __launch_bounds__(1024) k_prune_scan(uint32_t *__restrict__ bsum, int nb, int64_t *__restrict__ ctl,
                                                     int64_t *__restrict__ d_num_kept) {
  pdl_enter();
  __shared__ unsigned long long part[1024];
  const int per = (nb + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += bsum[i];
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
    const uint32_t v = bsum[i];
    bsum[i] = (uint32_t)run;
    run += v;
  }
  if (threadIdx.x == 1023) {
    const int64_t kept = (int64_t)part[1023];
    ctl[0] = kept;
    *d_num_kept = kept;
  }
}

__global__ void __launch_bounds__(kPruneBlock) k_prune_index(const float *__restrict__ ls,
                                                             const float *__restrict__ logit, int64_t cap,
                                                             float min_logit, float max_log_scale,
                                                             const uint32_t *__restrict__ bsum,
                                                             int64_t *__restrict__ ctl, uint32_t *__restrict__ hole,
                                                             uint32_t *__restrict__ mover) {
  pdl_enter();
  __shared__ uint32_t wsum[kPruneBlock / 32];
  const int64_t live = ctl[2];
  const int64_t K = ctl[0];
  const int64_t i = blockIdx.x * (int64_t)kPruneBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool in = i < live;
  const bool keep = in && survives(ls, logit, cap, i, min_logit, max_log_scale);
  const uint32_t b = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) wsum[warp] = __popc(b);
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = wsum[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    wsum[lane] = wi - w;
  }
  __syncthreads();
  const bool is_hole = in && !keep && i < K;
  const uint32_t hb = __ballot_sync(0xffffffffu, is_hole);
  if (hb && lane == __ffs(hb) - 1)
    atomicAdd(reinterpret_cast<unsigned long long *>(ctl + 1), (unsigned long long)__popc(hb));
  if (!in) return;
  const int64_t S = (int64_t)bsum[blockIdx.x] + wsum[warp] + __popc(b & ((1u << lane) - 1u));  // survivors below i
  if (is_hole) hole[i - S] = (uint32_t)i;
  if (keep && i >= K) mover[K - 1 - S] = (uint32_t)i;
}

struct PlaneSet {
  float *p[42];  // up to the 14 planes of the map and of each Adam moment
};

// Mover h goes to hole h in every plane; blockIdx.y selects the plane.
__global__ void k_prune_move(PlaneSet P, const uint32_t *__restrict__ hole, const uint32_t *__restrict__ mover,
                             const int64_t *__restrict__ ctl) {
  pdl_enter();
  const int64_t H = ctl[1];
  float *__restrict__ plane = P.p[blockIdx.y];
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < H; h += (int64_t)gridDim.x * blockDim.x)
    plane[hole[h]] = plane[mover[h]];
}

static PlaneSet planes_of(fgs_gaussians *g) {
  PlaneSet P;
  const int64_t c = g->capacity;
  for (int k = 0; k < 3; ++k) P.p[k] = g->means + k * c;
  for (int k = 0; k < 3; ++k) P.p[3 + k] = g->log_scales + k * c;
  for (int k = 0; k < 4; ++k) P.p[6 + k] = g->quats + k * c;
  P.p[10] = g->opacity_logits;
  for (int k = 0; k < 3; ++k) P.p[11 + k] = g->rgb + k * c;
  return P;
}

}  // namespace fgs

using namespace fgs;

extern "C" size_t fgs_prune_workspace_size(int64_t capacity) {
  if (capacity < 0) return 0;
  return prune_carve(nullptr, capacity).bytes;
}

extern "C" fgs_status fgs_prune(fgs_gaussians *g, fgs_gaussians *m, fgs_gaussians *v, const fgs_prune_params *p,
                                void *ws, size_t ws_bytes, int64_t *d_num_kept, void *stream) {
  if (!gaussians_ok(g, "g")) return FGS_ERR_INVALID_ARGUMENT;
  FGS_CHECK_ARG(p && d_num_kept, "fgs_prune: NULL argument");
  FGS_CHECK_ARG((m == nullptr) == (v == nullptr), "fgs_prune: give both Adam moments or neither");
  if (m) {
    if (!gaussians_ok(m, "m") || !gaussians_ok(v, "v")) return FGS_ERR_INVALID_ARGUMENT;
    FGS_CHECK_ARG(m->capacity == g->capacity && v->capacity == g->capacity,
                  "fgs_prune: moments must have the map's capacity");
  }
  const int64_t cap = g->capacity;
  PruneScratch w = prune_carve(ws, cap);
  FGS_CHECK_ARG(ws != nullptr && ws_bytes >= w.bytes, "fgs_prune: workspace %zu < %zu bytes", ws_bytes, w.bytes);
  FGS_CHECK_ARG((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fgs_prune: workspace not 256-byte aligned");
  cudaStream_t st = as_stream(stream);
  const int64_t n = g->n;
  if (n == 0 && g->d_n == nullptr) {
    FGS_CUDA(cudaMemsetAsync(d_num_kept, 0, 8, st), "memset kept");
    return FGS_OK;
  }
  const int64_t nb = std::max<int64_t>(1, (n + kPruneBlock - 1) / kPruneBlock);
  FGS_CHECK_ARG(nb <= 1024 * 1024, "fgs_prune: too many Gaussians");
  pdl_launch(k_prune_init, 1, 1, 0, st, g->d_n, n, w.ctl);
  pdl_launch(k_prune_count, (unsigned)nb, kPruneBlock, 0, st, g->log_scales, g->opacity_logits, cap, p->min_logit,
             p->max_log_scale, w.bsum, w.ctl);
  pdl_launch(k_prune_scan, 1, 1024, 0, st, w.bsum, (int)nb, w.ctl, d_num_kept);
  pdl_launch(k_prune_index, (unsigned)nb, kPruneBlock, 0, st, g->log_scales, g->opacity_logits, cap, p->min_logit,
             p->max_log_scale, w.bsum, w.ctl, w.hole, w.mover);
  count_launch(4);
  // the moves of all 42 planes in one launch: blockIdx.y = buffer * 14 + plane
  PlaneSet P;
  int planes = 0;
  fgs_gaussians *bufs[3] = {g, m, v};
  for (int b = 0; b < 3; ++b) {
    if (!bufs[b]) continue;
    const PlaneSet Q = planes_of(bufs[b]);
    for (int k = 0; k < 14; ++k) P.p[planes++] = Q.p[k];
  }
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8));
  pdl_launch(k_prune_move, dim3(gx, planes), 256, 0, st, P, w.hole, w.mover, w.ctl);
  count_launch();
  if (g->d_n) {
    pdl_launch(k_prune_finish, 1, 1, 0, st, w.ctl, g->d_n);
    count_launch();
  }
  FGS_CHECK_LAUNCH("fgs_prune");
  return FGS_OK;
}
