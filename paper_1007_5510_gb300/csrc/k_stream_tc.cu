// Tensor-core streamed passes (tcgen05, sm_103a).  Placeholder until the
// kernel lands: reports "unsupported" so the CUDA-core pass runs.
#include "common.cuh"
#include "kernels.h"

namespace rpca {
bool launch_pass_tc(const PassArgs&, cudaStream_t, uint32_t*) { return false; }
}  // namespace rpca
