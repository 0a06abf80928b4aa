// kernels_df_c.cu -- FP64-data chain kernels (double-float and native), lengths 100, 120, 128, 144.
#include "kernels_df.cuh"

namespace vloc {
template struct LaunchF64<0, 100>;
template struct LaunchF64<1, 100>;
template struct LaunchF64<0, 120>;
template struct LaunchF64<1, 120>;
template struct LaunchF64<0, 128>;
template struct LaunchF64<1, 128>;
template struct LaunchF64<0, 144>;
template struct LaunchF64<1, 144>;
}  // namespace vloc
