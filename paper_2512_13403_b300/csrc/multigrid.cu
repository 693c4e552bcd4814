// Multigrid self-gravity (Sec. 5.2): placeholder until the V-cycle kernels land.
#include "dh_internal.h"

namespace dh {
std::string mg_validate(const dh_config&) { return "gravity is not available in this build"; }
cudaError_t mg_allocate(dh_ctx*) { return cudaSuccess; }
void mg_setup_host(dh_ctx*) {}
cudaError_t mg_reset(dh_ctx*) { return cudaSuccess; }
void mg_free(dh_ctx*) {}
template <typename real> cudaError_t gravity_sources(dh_ctx*, void*) { return cudaErrorNotSupported; }
template cudaError_t gravity_sources<float>(dh_ctx*, void*);
template cudaError_t gravity_sources<double>(dh_ctx*, void*);
}  // namespace dh
