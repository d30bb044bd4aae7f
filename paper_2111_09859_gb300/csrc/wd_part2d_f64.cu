// wd_part2d_f64.cu -- FP64 instantiations of the warp partition passes (wd_part2d.cuh).
#include "wd_part2d.cuh"

namespace wd {

template cudaError_t p2_launch<double, double>(const F2Args<double, double>&, const PartTab<double>&, int,
                                               int, cudaStream_t);
template bool p2_supported<double, double>(const F2Args<double, double>&, const PartTab<double>&, int, int);

template cudaError_t p2_div2<double, double>(const F2Args<double, double>&, const PartTab<double>&, const PartTab<double>&,
                                         cudaStream_t);

}  // namespace wd
