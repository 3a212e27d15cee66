// tcgen05 / TMA form of the distance pass (BF16 and split-BF16 Gram products).
#include "kkm_internal.cuh"

namespace kkm {

bool tc_available() { return false; }

cudaError_t tc_prepare(Dev&) { return cudaErrorNotSupported; }

cudaError_t launch_dist_tc(const Dev&, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace kkm
