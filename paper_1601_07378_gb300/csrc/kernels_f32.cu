// kernels_f32.cu -- float instantiation of the V_loc kernels.
#include "kernels_impl.cuh"

namespace vloc {
template struct Launch<float>;
}  // namespace vloc
