// BF16 tensor-core operator (tcgen05 + TMA) for CMCS_BF16_REFINE.
#include <stdio.h>

#include "cmcs_internal.cuh"

namespace cmcs {

int tc_create(Ctx* c) {
  snprintf(c->err, sizeof(c->err), "the BF16 tensor-core operator is not built yet");
  return 1;
}

void tc_destroy(Ctx* c) { c->tc = nullptr; }

cudaError_t tc_operator(Ctx*, const float*, float*) { return cudaErrorNotSupported; }

}  // namespace cmcs
