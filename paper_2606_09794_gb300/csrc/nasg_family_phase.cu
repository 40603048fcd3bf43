// Forward, backward and fused kernels of the phase-shifted-carrier lobe family
// (QUAT frames), instantiated in their own translation unit.
#include "nasg_kernels.cuh"

namespace nasg {

template nasg_status launch_family<kFwd, kFamPhase>(const EvalArgs&, bool, bool, cudaStream_t);
template nasg_status launch_family<kBwd, kFamPhase>(const EvalArgs&, bool, bool, cudaStream_t);
template nasg_status launch_family<kFwdBwd, kFamPhase>(const EvalArgs&, bool, bool, cudaStream_t);

}  // namespace nasg
