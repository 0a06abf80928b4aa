// kernels_df_a.cu -- FP64-data chain kernels (double-float and native), lengths 24, 32, 48, 60.
#include "kernels_df.cuh"

namespace vloc {
template struct LaunchF64<0, 24>;
template struct LaunchF64<1, 24>;
template struct LaunchF64<0, 32>;
template struct LaunchF64<1, 32>;
template struct LaunchF64<0, 48>;
template struct LaunchF64<1, 48>;
template struct LaunchF64<0, 60>;
template struct LaunchF64<1, 60>;
}  // namespace vloc
