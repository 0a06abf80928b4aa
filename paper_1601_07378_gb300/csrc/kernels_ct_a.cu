// kernels_ct_a.cu -- FP32 compile-time-length chain kernels, lengths 24, 32, 48, 60.
#include "kernels_ct.cuh"

namespace vloc {
template struct LaunchCT<float, 24>;
template struct LaunchCT<float, 32>;
template struct LaunchCT<float, 48>;
template struct LaunchCT<float, 60>;
}  // namespace vloc
