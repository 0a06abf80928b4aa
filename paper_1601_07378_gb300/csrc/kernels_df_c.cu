// kernels_df_c.cu -- Double-float chain kernels, lengths 100, 120, 128, 144.
#include "kernels_df.cuh"

namespace vloc {
template struct LaunchDF<100>;
template struct LaunchDF<120>;
template struct LaunchDF<128>;
template struct LaunchDF<144>;
}  // namespace vloc
