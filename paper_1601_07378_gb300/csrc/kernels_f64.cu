// kernels_f64.cu -- double instantiation of the V_loc kernels.
#include "kernels_impl.cuh"

namespace vloc {
template struct Launch<double>;
}  // namespace vloc
