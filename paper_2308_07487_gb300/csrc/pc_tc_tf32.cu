// Instantiation of the fused tensor-core kernel for the TF32 form, one CTA per tile
// (see pc_tc_kernel.cuh; the CTA-pair kernels are in pc_tc_tf32_pair.cu).
#include "pc_tc_kernel.cuh"

namespace asd {
extern template int tc_launch_pair<ASD_TF32>(const TcLaunchArgs &, size_t, int, int, int,
                                             cudaStream_t);
template int tc_launch_form<ASD_TF32>(const TcLaunchArgs &, size_t, int, int, int, int,
                                      cudaStream_t);
}  // namespace asd
