// kernels_ct.cuh -- the chain kernels with compile-time axis lengths.
//
// Same five steps as kernels_impl.cuh (K1 scatter + inverse z-pass, K2
// y-passes, K3 x-pass with V(r), K4 forward z-pass + gather), specialised
// for one axis length N per instantiation so the Stockham stages of
// fft_ct.cuh fold their index arithmetic, use one shared buffer per tile,
// and K3 chains the inverse x-FFT's last stage, the multiply by V and the
// forward x-FFT's first stage in registers (no shared-memory round trip
// between the two transforms).  Instantiated for the common grid lengths in
// kernels_ct_*.cu; other lengths use the runtime-radix kernels.
#pragma once

#include "fft_ct.cuh"
#include "kernels_impl.cuh"

namespace vloc {

template <int N> __host__ __device__ constexpr size_t ct_smem(size_t elem) {
    return (size_t)N * kLd * elem + (size_t)N * elem + (size_t)N * sizeof(int) + 16;
}

// rows of a tile with a compile-time row length
template <int NN, typename V>
__device__ __forceinline__ void rows_out_ct(const V* buf, V* __restrict__ cb, const int* sticks, int lines) {
    const int total = lines * NN;
    for (int i = threadIdx.x; i < total; i += kThreads) {
        const int l = i / NN, z = i - l * NN;
        cb[(long long)sticks[l] * NN + z] = buf[z * kLd + l];
    }
}
template <int NN, typename V>
__device__ __forceinline__ void rows_in_ct(V* buf, const V* __restrict__ cb, const int* sticks, int lines) {
    const int total = lines * NN;
    for (int base = threadIdx.x; base < total; base += kBatch * kThreads) {
        V val[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = base + u * kThreads;
            if (i < total) {
                const int l = i / NN, z = i - l * NN;
                val[u] = cb[(long long)sticks[l] * NN + z];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = base + u * kThreads;
            if (i < total) {
                const int l = i / NN, z = i - l * NN;
                buf[z * kLd + l] = val[u];
            }
        }
    }
}

// ------------------------------------------------------------------ K1
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k1_ct(DevTables t, const V2<T>* __restrict__ tw3,
                                                 const V2<T>* __restrict__ coeffs, V2<T>* __restrict__ cyl) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    V* stw = buf + N * kLd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    load_tw<T>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    for (int i = threadIdx.x; i < N * kLd; i += kThreads) buf[i] = czero<V>();
    __syncthreads();
    scatter_entries(t.tile_pw, t.tile_pw_ptr[tile], t.tile_pw_ptr[tile + 1], coeffs + b * t.npw, buf);
    __syncthreads();
    fft_ct<N, +1, kWarps, false, true, true>(stw, Smem<V>{buf}, Smem<V>{buf}, buf, lane, warp, lane < lines);
    __syncthreads();
    rows_out_ct<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
}

// ------------------------------------------------------------------ K2
template <typename T, int S, int N>
__global__ void __launch_bounds__(kThreads) k2_ct(DevTables t, const V2<T>* __restrict__ tw2, V2<T>* cyl,
                                                 V2<T>* slab) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = t.n3;
    V* buf = reinterpret_cast<V*>(smem_raw);
    V* stw = buf + N * kLd;
    int* rowmap = reinterpret_cast<int*>(stw + N);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int plane = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<T>(stw, tw2, N);
    for (int e = threadIdx.x; e < N; e += kThreads) rowmap[e] = -1;
    __syncthreads();
    for (int s = t.plane_ptr[plane] + threadIdx.x; s < t.plane_ptr[plane + 1]; s += kThreads) rowmap[t.stick_row[s]] = s;
    __syncthreads();
    CylRows<T> cr{cyl + b * (long long)t.S * n3, rowmap, n3, z0};
    SlabRows<T> sr{slab + ((b * t.NP + plane) * (long long)N) * n3 + z0, n3};
    if constexpr (S > 0) fft_ct<N, +1, kWarps, false, false, false>(stw, cr, sr, buf, lane, warp, lane < lines);
    else fft_ct<N, -1, kWarps, false, false, false>(stw, sr, cr, buf, lane, warp, lane < lines);
}

// ------------------------------------------------------------------ K3
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k3_ct(DevTables t, const V2<T>* __restrict__ tw1, const T* __restrict__ Vr,
                                                 V2<T>* slab) {
    using V = V2<T>;
    using SC = Sched<N>;
    constexpr int nst = SC::nst;
    static_assert(nst >= 2, "compile-time x-pass needs at least two stages");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    V* buf = reinterpret_cast<V*>(smem_raw);
    V* stw = buf + N * kLd;
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    const bool act = lane < lines;
    load_tw<T>(stw, tw1, N);
    for (int e = threadIdx.x; e < N; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const long long pstride = (long long)n2 * n3;
    XRows<T> xr{slab + b * t.NP * pstride + (long long)y * n3 + z0, xrow, pstride};
    const T* vrow = Vr + (long long)y * n3 + z0;
    Smem<V> sb{buf};

    // inverse x-FFT, stages 0 .. nst-2 (global rows -> buffer)
    NatStage<N, +1, kWarps, 0>::template run<false>(stw, xr, sb, lane, warp, act);
    __syncthreads();
    if constexpr (nst >= 3) {
        NatStage<N, +1, kWarps, 1>::template run<true>(stw, sb, sb, lane, warp, act);
        __syncthreads();
    }
    if constexpr (nst >= 4) {
        NatStage<N, +1, kWarps, 2>::template run<true>(stw, sb, sb, lane, warp, act);
        __syncthreads();
    }
    // last inverse stage -> psi(x) * V(x, y, z) -> first forward stage of the
    // reversed schedule, in registers: both work on elements i + r N/R.
    using L = NatStage<N, +1, kWarps, nst - 1>;
    using F = RevStage<N, -1, kWarps, 0>;
    constexpr int R = SC::R(nst - 1);
    static_assert(F::NI == L::NI && SC::RR(0) == R, "chained stages must share units");
    V h[L::U][R];
    if (act) {
        L::compute(h, stw, sb, lane, warp);
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = warp + u * kWarps;
            if (L::NI % kWarps == 0 || i < L::NI) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T w = vrow[(long long)(i + r * L::NI) * pstride + lane];
                    h[u][r] = cmk<V>(h[u][r].x * w, h[u][r].y * w);
                }
                Dft<R, -1>::run(h[u]);
            }
        }
    }
    __syncthreads();
    if (act) F::store(h, sb, lane, warp);
    __syncthreads();
    // forward x-FFT, remaining stages (buffer -> occupied global rows)
    if constexpr (nst >= 3) {
        RevStage<N, -1, kWarps, 1>::template run<true>(stw, sb, sb, lane, warp, act);
        __syncthreads();
    }
    if constexpr (nst >= 4) {
        RevStage<N, -1, kWarps, 2>::template run<true>(stw, sb, sb, lane, warp, act);
        __syncthreads();
    }
    RevStage<N, -1, kWarps, nst - 1>::template run<false>(stw, sb, xr, lane, warp, act);
}

// ------------------------------------------------------------------ K4
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k4_ct(DevTables t, const V2<T>* __restrict__ tw3,
                                                 const V2<T>* __restrict__ cyl, V2<T>* __restrict__ out, T scale) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    V* stw = buf + N * kLd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    load_tw<T>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    rows_in_ct<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
    __syncthreads();
    fft_ct<N, -1, kWarps, false, true, true>(stw, Smem<V>{buf}, Smem<V>{buf}, buf, lane, warp, lane < lines);
    __syncthreads();
    gather_entries(t.tile_pw, t.tile_pw_ptr[tile], t.tile_pw_ptr[tile + 1], buf, out + b * t.npw, scale);
}

// ------------------------------------------------------------ launchers
template <typename T, int N> struct LaunchCTImpl {
    static constexpr size_t sm = ct_smem<N>(sizeof(V2<T>));
    template <class K> static cudaError_t ensure(K kernel) {
        if (sm <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
};

template <typename T, int N>
int LaunchCT<T, N>::k1(const DevTables& t, const void* tw3, const void* coeffs, long long nb, void* cyl,
                       cudaStream_t st) {
    static const cudaError_t once = LaunchCTImpl<T, N>::ensure(k1_ct<T, N>);
    if (once) return (int)once;
    k1_ct<T, N><<<dim3(t.T, (unsigned)nb), kThreads, LaunchCTImpl<T, N>::sm, st>>>(
        t, (const V2<T>*)tw3, (const V2<T>*)coeffs, (V2<T>*)cyl);
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k2(int sign, const DevTables& t, const void* tw2, long long nb, void* cyl, void* slab,
                       cudaStream_t st) {
    const dim3 grid(t.NP, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    if (sign > 0) {
        static const cudaError_t once = LaunchCTImpl<T, N>::ensure(k2_ct<T, +1, N>);
        if (once) return (int)once;
        k2_ct<T, +1, N><<<grid, kThreads, LaunchCTImpl<T, N>::sm, st>>>(t, (const V2<T>*)tw2, (V2<T>*)cyl, (V2<T>*)slab);
    } else {
        static const cudaError_t once = LaunchCTImpl<T, N>::ensure(k2_ct<T, -1, N>);
        if (once) return (int)once;
        k2_ct<T, -1, N><<<grid, kThreads, LaunchCTImpl<T, N>::sm, st>>>(t, (const V2<T>*)tw2, (V2<T>*)cyl, (V2<T>*)slab);
    }
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k3(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab, cudaStream_t st) {
    static const cudaError_t once = LaunchCTImpl<T, N>::ensure(k3_ct<T, N>);
    if (once) return (int)once;
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    k3_ct<T, N><<<grid, kThreads, LaunchCTImpl<T, N>::sm, st>>>(t, (const V2<T>*)tw1, (const T*)V, (V2<T>*)slab);
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k4(const DevTables& t, const void* tw3, const void* cyl, long long nb, void* out,
                       cudaStream_t st) {
    static const cudaError_t once = LaunchCTImpl<T, N>::ensure(k4_ct<T, N>);
    if (once) return (int)once;
    const T scale = (T)(1.0 / ((double)t.n1 * t.n2 * t.n3));
    k4_ct<T, N><<<dim3(t.T, (unsigned)nb), kThreads, LaunchCTImpl<T, N>::sm, st>>>(
        t, (const V2<T>*)tw3, (const V2<T>*)cyl, (V2<T>*)out, scale);
    return (int)cudaGetLastError();
}

}  // namespace vloc
