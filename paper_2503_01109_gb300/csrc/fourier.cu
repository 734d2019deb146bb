// fourier.cu -- Fourier seeding of Sec. III-A (eq2-eq11).  Entry points report
// FGS_ERR_UNSUPPORTED until the kernels land.
#include "common.cuh"

using namespace fgs;

extern "C" size_t fgs_fourier_seed_workspace_size(int32_t width, int32_t height) {
  (void)width;
  (void)height;
  return 0;
}

extern "C" fgs_status fgs_fourier_seed(const float *, const float *, const float *, const float *, const float *,
                                       const fgs_camera *, const fgs_seed_params *, const fgs_mlp *, uint8_t *,
                                       float *, fgs_gaussians *, int32_t *, int32_t *, void *, size_t, int32_t *,
                                       void *) {
  set_error("fgs_fourier_seed: not built yet");
  return FGS_ERR_UNSUPPORTED;
}
