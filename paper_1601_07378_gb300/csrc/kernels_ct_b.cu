// kernels_ct_b.cu -- FP32 compile-time-length chain kernels, lengths 64, 72, 80, 96.
#include "k3_tma.cuh"

namespace vloc {
template struct LaunchCT<float, 64>;
template struct LaunchCT<float, 72>;
template struct LaunchCT<float, 80>;
template struct LaunchCT<float, 96>;
template int launch_k3_tma<64>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<72>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<80>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<96>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
}  // namespace vloc
