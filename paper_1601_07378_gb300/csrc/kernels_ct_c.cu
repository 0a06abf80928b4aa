// kernels_ct_c.cu -- FP32 compile-time-length chain kernels, lengths 100, 120, 128, 144.
#include "k3_tma.cuh"

namespace vloc {
template struct LaunchCT<float, 100>;
template struct LaunchCT<float, 120>;
template struct LaunchCT<float, 128>;
template struct LaunchCT<float, 144>;
template int launch_k3_tma<100>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<120>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<128>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
template int launch_k3_tma<144>(const DevTables&, const void*, const void*, long long, void*, const K3Tma&,
                                   cudaStream_t);
}  // namespace vloc
