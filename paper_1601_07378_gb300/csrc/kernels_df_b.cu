// kernels_df_b.cu -- Double-float chain kernels, lengths 64, 72, 80, 96.
#include "kernels_df.cuh"

namespace vloc {
template struct LaunchDF<64>;
template struct LaunchDF<72>;
template struct LaunchDF<80>;
template struct LaunchDF<96>;
}  // namespace vloc
