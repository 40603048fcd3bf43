// Instantiation of the fwd NASGabor evaluation kernels (see nasg_kernels.cuh).
#include "nasg_kernels.cuh"

namespace nasg {
template nasg_status launch_eval<kFwd>(const nasg_desc*, EvalArgs, cudaStream_t);
}  // namespace nasg
