// kernels_ct_c.cu -- FP32 compile-time-length chain kernels, lengths 100, 120, 128, 144.
#include "kernels_ct.cuh"

namespace vloc {
template struct LaunchCT<float, 100>;
template struct LaunchCT<float, 120>;
template struct LaunchCT<float, 128>;
template struct LaunchCT<float, 144>;
}  // namespace vloc
