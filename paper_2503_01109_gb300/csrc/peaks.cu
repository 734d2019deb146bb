// peaks.cu -- microbenchmarks of the on-chip rates the blend kernels are bound by:
// FP32 fused multiply-add, the MUFU ex2 approximation and shared-memory loads.
// The benchmark times one launch with CUDA events and divides the operation
// count the call reports by it, so the roofline of the render kernels rests on
// rates measured on the part at its running clock rather than on unit counts.
//
// Each kernel keeps 16 independent dependency chains per thread so that the
// pipe, not the latency of one chain, limits the rate; every chain's result is
// folded into `sink` so that nothing is dead code.
#include "common.cuh"

namespace fgs {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 16;
constexpr int kPeakSmemFloat4 = 2048;  // 32 KiB of shared memory per block

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(int64_t iters, float a, float b, float *sink) {
  float x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // never true for the probe's inputs; keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(int64_t iters, float *sink) {
  float x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = 1.0f + (float)c * 0.01f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = ex2_approx(-x[c]);  // x -> 2^-x stays in (0.5, 1)
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == 12345.678f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_lds(int64_t iters, float *sink) {
  __shared__ float4 buf[kPeakSmemFloat4];
  for (int e = threadIdx.x; e < kPeakSmemFloat4; e += kPeakThreads)
    buf[e] = make_float4((float)e, 1.f, 2.f, 3.f);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int idx = threadIdx.x;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) {
      // consecutive lanes read consecutive 16-byte words: four conflict-free wavefronts per warp load
      const float4 v = buf[(idx + c * kPeakThreads) & (kPeakSmemFloat4 - 1)];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    idx = (idx + 32) & (kPeakSmemFloat4 - 1);
  }
  const float s = acc.x + acc.y + acc.z + acc.w;
  if (s == 12345.678f) sink[blockIdx.x] = s;
}

}  // namespace fgs

using namespace fgs;

extern "C" int32_t fgs_num_sms(void) { return num_sms(); }

extern "C" fgs_status fgs_peak_probe(int32_t kind, int32_t blocks_per_sm, int64_t iters, float *sink,
                                     int64_t *ops, void *stream) {
  FGS_CHECK_ARG(kind >= FGS_PEAK_FFMA && kind <= FGS_PEAK_LDS, "fgs_peak_probe: unknown kind %d", kind);
  FGS_CHECK_ARG(blocks_per_sm >= 1 && blocks_per_sm <= 32 && iters >= 1 && iters <= (int64_t(1) << 32) && sink &&
                    ops,
                "fgs_peak_probe: bad argument");
  const int blocks = num_sms() * blocks_per_sm;
  const int64_t per_thread = iters * kPeakChains;
  const int64_t threads = (int64_t)blocks * kPeakThreads;
  cudaStream_t st = as_stream(stream);
  if (kind == FGS_PEAK_FFMA) {
    k_peak_ffma<<<blocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-4f, sink);
    *ops = 2 * per_thread * threads;  // two floating-point operations per FMA
  } else if (kind == FGS_PEAK_EX2) {
    k_peak_ex2<<<blocks, kPeakThreads, 0, st>>>(iters, sink);
    *ops = per_thread * threads;
  } else {
    k_peak_lds<<<blocks, kPeakThreads, 0, st>>>(iters, sink);
    *ops = 16 * per_thread * threads;  // bytes loaded from shared memory
  }
  count_launch();
  FGS_CHECK_LAUNCH("fgs_peak_probe");
  return FGS_OK;
}
