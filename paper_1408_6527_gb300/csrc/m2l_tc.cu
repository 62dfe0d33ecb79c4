// Multipole-to-local translation on the tensor cores (placeholder until the
// tcgen05 kernel lands; MIXED mode uses the SIMT kernel meanwhile).
#include "internal.cuh"

namespace polfmm {

bool m2l_tensor_enabled(polfmm_ctx*) { return false; }
void m2l_tensor_launch(polfmm_ctx*) {}
int m2l_tensor_prepare(polfmm_ctx*) { return POLFMM_OK; }
void m2l_tensor_release(polfmm_ctx*) {}

}  // namespace polfmm
