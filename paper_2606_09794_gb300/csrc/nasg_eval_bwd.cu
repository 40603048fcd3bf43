// Instantiation of the bwd NASGabor evaluation kernels (see nasg_kernels.cuh).
#include "nasg_kernels.cuh"

namespace nasg {
template nasg_status launch_eval<kBwd>(const nasg_desc*, EvalArgs, cudaStream_t);
}  // namespace nasg
