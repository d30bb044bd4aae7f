// wd_line2d_f64.cu -- FP64 instantiations of the line-resident 2-D passes (wd_line2d.cuh).
#include "wd_line2d.cuh"

namespace wd {

template cudaError_t l2_launch<double, double>(const L2Args<double, double>&, const PartTab<double>&, int, int, cudaStream_t);
template bool l2_supported<double, double>(const Dims&, const PartTab<double>&, const PartTab<double>&, int);

}  // namespace wd
