// Forward, backward and fused kernels of the NASG (no carrier) lobe family
// (QUAT frames), instantiated in their own translation unit.
#include "nasg_kernels.cuh"

namespace nasg {

template nasg_status launch_family<kFwd, kFamNasg>(const EvalArgs&, bool, bool, cudaStream_t);
template nasg_status launch_family<kBwd, kFamNasg>(const EvalArgs&, bool, bool, cudaStream_t);
template nasg_status launch_family<kFwdBwd, kFamNasg>(const EvalArgs&, bool, bool, cudaStream_t);

}  // namespace nasg
