// kernels_ct_b.cu -- FP32 compile-time-length chain kernels, lengths 64, 72, 80, 96.
#include "kernels_ct.cuh"

namespace vloc {
template struct LaunchCT<float, 64>;
template struct LaunchCT<float, 72>;
template struct LaunchCT<float, 80>;
template struct LaunchCT<float, 96>;
}  // namespace vloc
