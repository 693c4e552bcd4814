// Hand adjoint of the RK2 step: placeholder until the adjoint stage kernels land.
#include "dh_internal.h"

namespace dh {
void adjoint_free(dh_ctx*) {}
}  // namespace dh

extern "C" dh_status dh_adjoint_advance(dh_ctx* c, int, int, const void*, void*, int) {
  if (c) c->err = "adjoint not available in this build";
  return DH_ERR_ARG;
}
extern "C" dh_status dh_get_potential(dh_ctx* c, double*, int, int*, double*) {
  if (c) c->err = "gravity not available in this build";
  return DH_ERR_STATE;
}
