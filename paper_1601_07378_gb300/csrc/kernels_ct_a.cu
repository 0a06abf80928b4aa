// kernels_ct_a.cu -- FP32 compile-time-length chain kernels, lengths 24, 32, 48, 60.
#include "k3_tma.cuh"

namespace vloc {
template struct LaunchCT<float, 24>;
template struct LaunchCT<float, 32>;
template struct LaunchCT<float, 48>;
template struct LaunchCT<float, 60>;
template int launch_k3_tma<24>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<32>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<48>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<60>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
}  // namespace vloc
