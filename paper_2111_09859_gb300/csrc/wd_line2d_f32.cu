// wd_line2d_f32.cu -- FP32 instantiations of the line-resident 2-D passes (wd_line2d.cuh).
#include "wd_line2d.cuh"

namespace wd {

template cudaError_t l2_launch<float, float>(const L2Args<float, float>&, const PartTab<float>&, int, int, cudaStream_t);
template bool l2_supported<float, float>(const Dims&, const PartTab<float>&, const PartTab<float>&, int);

}  // namespace wd
