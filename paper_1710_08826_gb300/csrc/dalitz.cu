// dalitz.cu -- three-body amplitude models (placeholder until the amplitude kernels land).
#include "common.cuh"
#include "model.cuh"

namespace goo {
int build_dalitz_model(goo_ctx*, const goo_node*, int, int, int, const double*, const double*, goo_model*) {
  return set_error(GOO_ERR_UNSUPPORTED, "amplitude models are not built yet");
}
int dalitz_set_norm(goo_model*, const goo_norm_spec*) { return set_error(GOO_ERR_UNSUPPORTED, "amplitude models"); }
void dalitz_free(goo_model*) {}
int dalitz_normalise(goo_model*, const double*, int, double*) { return set_error(GOO_ERR_UNSUPPORTED, "amplitude models"); }
int dalitz_nll(goo_model*, const goo_dataset*, int64_t, int64_t, const double*, int, bool, double*, int) {
  return set_error(GOO_ERR_UNSUPPORTED, "amplitude models");
}
int dalitz_eval_logf(goo_model*, const goo_dataset*, const double*, int, double*) {
  return set_error(GOO_ERR_UNSUPPORTED, "amplitude models");
}
}  // namespace goo
