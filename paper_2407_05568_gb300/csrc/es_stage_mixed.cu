// es_stage_mixed.cu -- mixed-precision form of the fused stage kernel (placeholder until built).
#include "es_internal.h"

namespace es {
cudaError_t stage_prepare_mixed(int) { return cudaErrorNotSupported; }
cudaError_t launch_stage_mixed(const StageParams&, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace es
