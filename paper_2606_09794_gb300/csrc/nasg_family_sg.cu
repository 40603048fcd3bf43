// Forward, backward and fused kernels of the SG (no anisotropy, no carrier) lobe family
// (QUAT frames), instantiated in their own translation unit.
#include "nasg_kernels.cuh"

namespace nasg {

template nasg_status launch_family<kFwd, kFamSg>(const EvalArgs&, bool, bool, cudaStream_t);
template nasg_status launch_family<kBwd, kFamSg>(const EvalArgs&, bool, bool, cudaStream_t);
template nasg_status launch_family<kFwdBwd, kFamSg>(const EvalArgs&, bool, bool, cudaStream_t);

}  // namespace nasg
