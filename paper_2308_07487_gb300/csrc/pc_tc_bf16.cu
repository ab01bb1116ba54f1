// Instantiation of the fused tensor-core kernel for the BF16 form, one CTA per tile
// (see pc_tc_kernel.cuh; the CTA-pair kernels are in pc_tc_bf16_pair.cu).
#include "pc_tc_kernel.cuh"

namespace asd {
extern template int tc_launch_pair<ASD_BF16>(const TcLaunchArgs &, size_t, int, int, int,
                                             cudaStream_t);
template int tc_launch_form<ASD_BF16>(const TcLaunchArgs &, size_t, int, int, int, int,
                                      cudaStream_t);
}  // namespace asd
