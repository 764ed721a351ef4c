// a2, tensor-core variant (tcgen05): not built yet; the CUDA-core kernel
// serves every request until it is.
#include "common.cuh"

namespace iht {

int launch_grad_tc(iht_dataset *, const float *, float *, const int32_t *) { return IHT_EINVAL; }

}  // namespace iht
