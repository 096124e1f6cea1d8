// Parameter adjoint (placeholder until the adjoint kernels land).
#include "md_device.cuh"

namespace mdk {

int launch_param_grad(Engine&, const double*, const double*, double*, cudaStream_t) { return MD_ERR_UNSUPPORTED; }

}  // namespace mdk
