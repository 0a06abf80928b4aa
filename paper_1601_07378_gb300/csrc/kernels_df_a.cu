// kernels_df_a.cu -- Double-float chain kernels, lengths 24, 32, 48, 60.
#include "kernels_df.cuh"

namespace vloc {
template struct LaunchDF<24>;
template struct LaunchDF<32>;
template struct LaunchDF<48>;
template struct LaunchDF<60>;
}  // namespace vloc
