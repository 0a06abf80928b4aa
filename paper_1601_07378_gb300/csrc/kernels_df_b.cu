// kernels_df_b.cu -- FP64-data chain kernels (double-float and native), lengths 64, 72, 80, 96.
#include "kernels_df.cuh"

namespace vloc {
template struct LaunchF64<0, 64>;
template struct LaunchF64<1, 64>;
template struct LaunchF64<0, 72>;
template struct LaunchF64<1, 72>;
template struct LaunchF64<0, 80>;
template struct LaunchF64<1, 80>;
template struct LaunchF64<0, 96>;
template struct LaunchF64<1, 96>;
}  // namespace vloc
