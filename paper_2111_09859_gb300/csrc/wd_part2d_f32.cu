// wd_part2d_f32.cu -- FP32 instantiations of the warp partition passes (wd_part2d.cuh).
#include "wd_part2d.cuh"

namespace wd {

template cudaError_t p2_launch<float, float>(const F2Args<float, float>&, const PartTab<float>&, int, int,
                                             cudaStream_t);
template bool p2_supported<float, float>(const F2Args<float, float>&, const PartTab<float>&, int, int);

template cudaError_t p2_div2<float, float>(const F2Args<float, float>&, const PartTab<float>&, const PartTab<float>&,
                                         cudaStream_t);

}  // namespace wd
