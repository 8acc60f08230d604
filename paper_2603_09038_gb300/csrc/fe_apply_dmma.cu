// FP64 tensor-core (mma.sync.m8n8k4.f64) variant of the fused apply: placeholder until built.
#include "fe_internal.h"

namespace fe {

int launch_apply_dmma(int, const ApplyArgs&, cudaStream_t) {
  return set_error(FE_ERR_UNSUPPORTED, "the DMMA variant is not built yet");
}

}  // namespace fe
