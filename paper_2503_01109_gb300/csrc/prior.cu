// prior.cu -- learned seeding prior (features + MLP).  Entry points report
// FGS_ERR_UNSUPPORTED until the kernels land.
#include "common.cuh"

using namespace fgs;

extern "C" int64_t fgs_prior_num_params(void) { return 0; }
extern "C" size_t fgs_prior_train_workspace_size(int64_t) { return 0; }
extern "C" fgs_status fgs_prior_features(const float *, const float *, int32_t, int32_t, const int32_t *, int64_t,
                                         uint16_t *, void *) {
  set_error("fgs_prior_features: not built yet");
  return FGS_ERR_UNSUPPORTED;
}
extern "C" fgs_status fgs_prior_infer(const fgs_mlp *, const uint16_t *, int64_t, float *, void *) {
  set_error("fgs_prior_infer: not built yet");
  return FGS_ERR_UNSUPPORTED;
}
extern "C" fgs_status fgs_prior_train(fgs_mlp *, fgs_mlp_master *, const uint16_t *, const float *, int64_t,
                                      const fgs_train_params *, float *, void *, size_t, void *) {
  set_error("fgs_prior_train: not built yet");
  return FGS_ERR_UNSUPPORTED;
}
