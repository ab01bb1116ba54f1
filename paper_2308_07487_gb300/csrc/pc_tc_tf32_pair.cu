// Instantiation of the fused tensor-core kernel for the TF32 form, CTA pairs (see
// pc_tc_kernel.cuh).
#include "pc_tc_kernel.cuh"

namespace asd {
template int tc_launch_pair<ASD_TF32>(const TcLaunchArgs &, size_t, int, int, int, cudaStream_t);
}  // namespace asd
