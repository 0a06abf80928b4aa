// kernels_impl.cuh -- the hot path of the V_loc action on GB300 (sm_103a).
//
// One apply of a chunk of bands is five launches (Sec. 2's G->r FFT,
// multiply by V_loc(r), r->G FFT, done as the compact 3-D FFT of Sec. 4.3 /
// Fig. 5 with the pass order z, y, x and its mirror):
//   K1 scatter_zpass : sphere -> cylinder.  One CTA per stick part (Sec. 3.2
//                      greedy partition); scatter the part's plane waves into
//                      shared memory, inverse z-FFT of each stick.
//   K2 ypass<+1>     : cylinder -> slab.  One CTA per (plane, 32-z tile);
//                      inverse y-FFT whose input rows are the plane's sticks.
//   K3 xpass_v       : slab -> slab, in place.  One CTA per (y, 32-z tile);
//                      inverse x-FFT over the occupied planes, multiply by
//                      V(r), forward x-FFT keeping only the occupied planes.
//   K2 ypass<-1>     : slab -> cylinder, output pruned to the sticks.
//   K4 zpass_gather  : cylinder -> sphere, forward z-FFT, times 1/N, gather.
// The "transposes" of the paper's distributed FFT are the cylinder and slab
// round trips through L2/HBM; workspace chunks are sized to stay in L2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"
#include "internal.h"

namespace vloc {

template <typename T> using V2 = c2<T>;

// ------------------------------------------------------------- twiddles
// exp(+2 pi i j / n) made in FP64 (sincospi) and rounded to the plan's type.
template <typename T> __global__ void k_twiddles(V2<T>* tw, int n) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    tw[j] = cmk<V2<T>>((T)c, (T)s);
}

template <typename T> __device__ __forceinline__ void load_tw(V2<T>* stw, const V2<T>* tw, int n) {
    for (int j = threadIdx.x; j < n; j += kThreads) stw[j] = tw[j];
}

// ------------------------------------------------------------- tile I/O
// Flat, batched loops over a tile's plane-wave entries and stick rows: each
// thread issues its independent loads before the dependent stores, so a CTA
// keeps many requests in flight instead of walking one stick at a time.
constexpr int kBatch = 4;

template <typename V>
__device__ __forceinline__ void scatter_entries(const int2* __restrict__ ent, int e0, int e1, const V* __restrict__ c,
                                                V* buf) {
    for (int base = e0 + (int)threadIdx.x; base < e1; base += kBatch * kThreads) {
        int2 en[kBatch];
        V val[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int e = base + u * kThreads;
            en[u] = e < e1 ? ent[e] : make_int2(0, -1);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) val[u] = en[u].y >= 0 ? c[en[u].x] : czero<V>();
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (en[u].y >= 0) buf[(en[u].y & 0xffff) * kLd + (en[u].y >> 16)] = val[u];
    }
}

template <typename V, typename T>
__device__ __forceinline__ void gather_entries(const int2* __restrict__ ent, int e0, int e1, const V* buf,
                                               V* o, T scale, const T* __restrict__ diag, const V* cin) {
    for (int e = e0 + (int)threadIdx.x; e < e1; e += kThreads) {
        const int2 en = ent[e];
        V v = cscale(buf[(en.y & 0xffff) * kLd + (en.y >> 16)], scale);
        if (diag) {  // H = diag + A: add the diagonal term (read before the write: out may alias c)
            const T d = diag[en.x];
            const V ci = cin[en.x];
            v = cmk<V>(v.x + d * ci.x, v.y + d * ci.y);
        }
        o[en.x] = v;
    }
}

// rows of a tile: line l <-> stick sticks[l], element z of that stick's row
template <typename V>
__device__ __forceinline__ void rows_out(const V* buf, V* __restrict__ cb, const int* sticks, int lines, int n) {
    const int total = lines * n;
    for (int i = threadIdx.x; i < total; i += kThreads) {
        const int l = i / n, z = i - l * n;
        cb[(long long)sticks[l] * n + z] = buf[z * kLd + l];
    }
}
template <typename V>
__device__ __forceinline__ void rows_in(V* buf, const V* __restrict__ cb, const int* sticks, int lines, int n) {
    const int total = lines * n;
    for (int base = threadIdx.x; base < total; base += kBatch * kThreads) {
        V val[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = base + u * kThreads;
            if (i < total) {
                const int l = i / n, z = i - l * n;
                val[u] = cb[(long long)sticks[l] * n + z];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = base + u * kThreads;
            if (i < total) {
                const int l = i / n, z = i - l * n;
                buf[z * kLd + l] = val[u];
            }
        }
    }
}

// ------------------------------------------------------------------ K1
template <typename T>
__global__ void __launch_bounds__(kThreads) k1_scatter_zpass(DevTables t, AxisPlan az, const V2<T>* __restrict__ tw3,
                                                            const V2<T>* __restrict__ coeffs, V2<T>* __restrict__ cyl) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = t.n3;
    V* P = reinterpret_cast<V*>(smem_raw);
    V* Q = P + n3 * kLd;
    V* stw = Q + n3 * kLd;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    load_tw<T>(stw, tw3, n3);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    for (int i = threadIdx.x; i < n3 * kLd; i += kThreads) Q[i] = czero<V>();
    __syncthreads();
    scatter_entries(t.tile_pw, t.tile_pw_ptr[tile], t.tile_pw_ptr[tile + 1], coeffs + b * t.npw, Q);
    __syncthreads();
    V* D = final_buf(az.nst, P, Q);
    fft_lines<+1>(az, stw, Smem<V>{Q}, Smem<V>{D}, P, Q, lines);
    __syncthreads();
    rows_out(D, cyl + b * (long long)t.S * n3, t.tile_sticks + s0, lines, n3);
}

// ------------------------------------------------------------------ K2
template <typename T> struct CylRows {  // input rows of a y-line tile: the plane's sticks
    V2<T>* cb;
    const int* rowmap;
    int n3, z0;
    __device__ __forceinline__ V2<T> operator()(int e, int l) const {
        const int s = rowmap[e];
        return s >= 0 ? cb[(long long)s * n3 + z0 + l] : czero<V2<T>>();
    }
    __device__ __forceinline__ void operator()(int e, int l, V2<T> v) const {
        const int s = rowmap[e];
        if (s >= 0) cb[(long long)s * n3 + z0 + l] = v;
    }
};
template <typename T> struct SlabRows {  // all y rows of one plane's slab tile
    V2<T>* p;  // points at slab[b][plane][0][z0]
    int n3;
    __device__ __forceinline__ V2<T> operator()(int e, int l) const { return p[(long long)e * n3 + l]; }
    __device__ __forceinline__ void operator()(int e, int l, V2<T> v) const { p[(long long)e * n3 + l] = v; }
};

template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k2_ypass(DevTables t, AxisPlan ay, const V2<T>* __restrict__ tw2,
                                                    V2<T>* cyl, V2<T>* slab) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    V* P = reinterpret_cast<V*>(smem_raw);
    V* Q = P + n2 * kLd;
    V* stw = Q + n2 * kLd;
    int* rowmap = reinterpret_cast<int*>(stw + n2);
    const int plane = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<T>(stw, tw2, n2);
    for (int e = threadIdx.x; e < n2; e += kThreads) rowmap[e] = -1;
    __syncthreads();
    for (int s = t.plane_ptr[plane] + threadIdx.x; s < t.plane_ptr[plane + 1]; s += kThreads) rowmap[t.stick_row[s]] = s;
    __syncthreads();
    CylRows<T> cr{cyl + b * (long long)t.S * n3, rowmap, n3, z0};
    SlabRows<T> sr{slab + ((b * t.NP + plane) * (long long)n2) * n3 + z0, n3};
    if (S > 0) fft_lines<+1>(ay, stw, cr, sr, P, Q, lines);
    else fft_lines<-1>(ay, stw, sr, cr, P, Q, lines);
}

// ------------------------------------------------------------------ K3
template <typename T> struct XRows {  // x-line tile at fixed y: rows = occupied planes
    V2<T>* sb;  // slab[b][0][y][z0]
    const int* xrow;
    long long pstride;  // n2 * n3
    __device__ __forceinline__ V2<T> operator()(int e, int l) const {
        const int p = xrow[e];
        return p >= 0 ? sb[p * pstride + l] : czero<V2<T>>();
    }
    __device__ __forceinline__ void operator()(int e, int l, V2<T> v) const {
        const int p = xrow[e];
        if (p >= 0) sb[p * pstride + l] = v;
    }
};
template <typename T> struct TimesV {  // psi(x) * V(x, y, z) into shared memory
    V2<T>* d;
    const T* vrow;  // V[0][y][z0]
    long long xstride;  // n2 * n3
    __device__ __forceinline__ void operator()(int e, int l, V2<T> v) const {
        const T w = vrow[e * xstride + l];
        d[e * kLd + l] = cmk<V2<T>>(v.x * w, v.y * w);
    }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k3_xpass_v(DevTables t, AxisPlan ax, const V2<T>* __restrict__ tw1,
                                                      const T* __restrict__ Vr, V2<T>* slab) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = t.n1, n2 = t.n2, n3 = t.n3;
    V* P = reinterpret_cast<V*>(smem_raw);
    V* Q = P + n1 * kLd;
    V* stw = Q + n1 * kLd;
    int* xrow = reinterpret_cast<int*>(stw + n1);
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<T>(stw, tw1, n1);
    for (int e = threadIdx.x; e < n1; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const long long pstride = (long long)n2 * n3;
    XRows<T> xr{slab + b * t.NP * pstride + (long long)y * n3 + z0, xrow, pstride};
    V* D = final_buf(ax.nst, P, Q);
    fft_lines<+1>(ax, stw, xr, TimesV<T>{D, Vr + (long long)y * n3 + z0, pstride}, P, Q, lines);
    __syncthreads();
    V* P2 = (D == P) ? Q : P;
    fft_lines<-1>(ax, stw, Smem<V>{D}, xr, P2, D, lines);
}

// ------------------------------------------------------------------ K4
template <typename T>
__global__ void __launch_bounds__(kThreads) k4_zpass_gather(DevTables t, AxisPlan az, const V2<T>* __restrict__ tw3,
                                                           const V2<T>* __restrict__ cyl, V2<T>* out, T scale,
                                                           const T* __restrict__ diag, const V2<T>* cin) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = t.n3;
    V* P = reinterpret_cast<V*>(smem_raw);
    V* Q = P + n3 * kLd;
    V* stw = Q + n3 * kLd;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    load_tw<T>(stw, tw3, n3);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    rows_in(Q, cyl + b * (long long)t.S * n3, t.tile_sticks + s0, lines, n3);
    __syncthreads();
    V* D = final_buf(az.nst, P, Q);
    fft_lines<-1>(az, stw, Smem<V>{Q}, Smem<V>{D}, P, Q, lines);
    __syncthreads();
    gather_entries(t.tile_pw, t.tile_pw_ptr[tile], t.tile_pw_ptr[tile + 1], D, out + b * t.npw, scale, diag,
                   diag ? cin + b * t.npw : cin);
}

// ----------------------------------------------------------- K3b (dL/dV)
// For each (y, z tile): psi = inverse x-FFT of the c-slab tile, g = inverse
// x-FFT of the grad-slab tile, acc(x, y, z) += sum_b Re(conj(g) psi) / N,
// bands in order (deterministic), FP64 accumulation.
template <typename T> struct AccumProduct {
    const V2<T>* psi;  // shared [n1][kLd]
    double* acc;       // shared [n1][kLd]
    __device__ __forceinline__ void operator()(int e, int l, V2<T> g) const {
        const V2<T> p = psi[e * kLd + l];
        acc[e * kLd + l] += (double)g.x * (double)p.x + (double)g.y * (double)p.y;
    }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k3b_grad_v(DevTables t, AxisPlan ax, const V2<T>* __restrict__ tw1,
                                                      const V2<T>* slab_c, const V2<T>* slab_g, int nb, int bpg,
                                                      double* __restrict__ partial, double invN) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = t.n1, n2 = t.n2, n3 = t.n3;
    V* stw = reinterpret_cast<V*>(smem_raw);
    V* P = stw + n1;
    V* Q = P + n1 * kLd;
    V* R3 = Q + n1 * kLd;
    double* acc = reinterpret_cast<double*>(R3 + n1 * kLd);
    int* xrow = reinterpret_cast<int*>(acc + n1 * kLd);
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const int grp = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<T>(stw, tw1, n1);
    for (int e = threadIdx.x; e < n1; e += kThreads) xrow[e] = t.xrow_plane[e];
    for (int i = threadIdx.x; i < n1 * kLd; i += kThreads) acc[i] = 0.0;
    __syncthreads();
    const long long pstride = (long long)n2 * n3;
    // psi lands in D1 (a buffer of {P, Q}); g's transform ping-pongs in the
    // two buffers that are not D1.
    V* D1 = final_buf(ax.nst, P, Q);
    V* G1 = (D1 == P) ? Q : P;
    const int b1 = min(nb, (grp + 1) * bpg);
    for (int b = grp * bpg; b < b1; ++b) {
        XRows<T> xc{const_cast<V*>(slab_c) + (long long)b * t.NP * pstride + (long long)y * n3 + z0, xrow, pstride};
        XRows<T> xg{const_cast<V*>(slab_g) + (long long)b * t.NP * pstride + (long long)y * n3 + z0, xrow, pstride};
        fft_lines<+1>(ax, stw, xc, Smem<V>{D1}, P, Q, lines);
        __syncthreads();
        fft_lines<+1>(ax, stw, xg, AccumProduct<T>{D1, acc}, G1, R3, lines);
        __syncthreads();
    }
    // this band group's partial sum (overwritten; summed over groups later
    // in a fixed order, so the result is deterministic)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* part = partial + (long long)grp * n1 * pstride;
    if (lane < lines) {
        for (int e = warp; e < n1; e += kWarps) part[((long long)e * n2 + y) * n3 + z0 + lane] = acc[e * kLd + lane] * invN;
    }
}

template <typename T> __global__ void k_finish_grad_v(const double* __restrict__ acc, T* __restrict__ g, long long N) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < N) g[i] = (T)acc[i];
}

// ------------------------------------------- half transforms and density
// The two halves of the chain on their own (x-pass to / from a full grid),
// and the charge density rho(r) = sum_n f_n |psi_n(r)|^2 (Sec. 3.1).
template <typename T> struct GridRows {  // x line at fixed (y, z0 + l) of a full grid
    V2<T>* g;           // grid[b][0][y][z0]
    long long pstride;  // n2 * n3
    __device__ __forceinline__ V2<T> operator()(int e, int l) const { return g[e * pstride + l]; }
    __device__ __forceinline__ void operator()(int e, int l, V2<T> v) const { g[e * pstride + l] = v; }
};

// S = +1: inverse x-pass of a slab tile (input pruned to the occupied
// planes) into the full grid [b][n1][n2][n3]; S = -1: forward x-pass of a
// full grid, kept on the occupied planes of the slab (output pruned).
template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k3_grid(DevTables t, AxisPlan ax, const V2<T>* __restrict__ tw1,
                                                   V2<T>* slab, V2<T>* grid) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = t.n1, n2 = t.n2, n3 = t.n3;
    V* P = reinterpret_cast<V*>(smem_raw);
    V* Q = P + n1 * kLd;
    V* stw = Q + n1 * kLd;
    int* xrow = reinterpret_cast<int*>(stw + n1);
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<T>(stw, tw1, n1);
    for (int e = threadIdx.x; e < n1; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const long long pstride = (long long)n2 * n3;
    XRows<T> xr{slab + b * t.NP * pstride + (long long)y * n3 + z0, xrow, pstride};
    GridRows<T> gr{grid + b * (long long)n1 * pstride + (long long)y * n3 + z0, pstride};
    if constexpr (S > 0) fft_lines<+1>(ax, stw, xr, gr, P, Q, lines);
    else fft_lines<-1>(ax, stw, gr, xr, P, Q, lines);
}

// Weights of band b in the density: (f_b, f_b) for a complex band; for a
// Gamma-point pair b = (2b, 2b + 1) packed as psi_2b + i psi_2b+1 (both
// real), (f_2b, f_2b+1) on the real and imaginary parts, 0 past the last
// real band.  f = 1 when occ is null.
template <typename T>
__device__ __forceinline__ void density_weights(const T* occ, long long b, int pair, long long nreal, double& wx,
                                                double& wy) {
    if (!pair) {
        wx = wy = occ ? (double)occ[b] : 1.0;
        return;
    }
    wx = occ ? (double)occ[2 * b] : 1.0;
    wy = 2 * b + 1 < nreal ? (occ ? (double)occ[2 * b + 1] : 1.0) : 0.0;
}
template <typename T> struct AccumNorm {  // acc += wx re^2 + wy im^2
    double* acc;                          // shared [n1][kLd]
    double wx, wy;
    __device__ __forceinline__ void operator()(int e, int l, V2<T> v) const {
        acc[e * kLd + l] += wx * ((double)v.x * (double)v.x) + wy * ((double)v.y * (double)v.y);
    }
};

// One (y, z tile, band group): psi = inverse x-pass of each band's slab tile,
// acc += weighted |psi|^2 in FP64, then the group's partial sum is written
// (groups are added later in a fixed order).
template <typename T>
__global__ void __launch_bounds__(kThreads) k3d_density(DevTables t, AxisPlan ax, const V2<T>* __restrict__ tw1,
                                                       const V2<T>* slab, int nb, int bpg, const T* __restrict__ occ,
                                                       long long b_base, int pair, long long nreal,
                                                       double* __restrict__ partial) {
    using V = V2<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = t.n1, n2 = t.n2, n3 = t.n3;
    V* P = reinterpret_cast<V*>(smem_raw);
    V* Q = P + n1 * kLd;
    V* stw = Q + n1 * kLd;
    double* acc = reinterpret_cast<double*>(stw + n1);
    int* xrow = reinterpret_cast<int*>(acc + n1 * kLd);
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const int grp = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<T>(stw, tw1, n1);
    for (int e = threadIdx.x; e < n1; e += kThreads) xrow[e] = t.xrow_plane[e];
    for (int i = threadIdx.x; i < n1 * kLd; i += kThreads) acc[i] = 0.0;
    __syncthreads();
    const long long pstride = (long long)n2 * n3;
    const int b1 = min(nb, (grp + 1) * bpg);
    for (int b = grp * bpg; b < b1; ++b) {
        double wx, wy;
        density_weights(occ, b_base + b, pair, nreal, wx, wy);
        XRows<T> xc{const_cast<V*>(slab) + (long long)b * t.NP * pstride + (long long)y * n3 + z0, xrow, pstride};
        fft_lines<+1>(ax, stw, xc, AccumNorm<T>{acc, wx, wy}, P, Q, lines);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* part = partial + (long long)grp * n1 * pstride;
    if (lane < lines) {
        for (int e = warp; e < n1; e += kWarps) part[((long long)e * n2 + y) * n3 + z0 + lane] = acc[e * kLd + lane];
    }
}

// ====================================================== typed launchers
// Members of Launch<T> (declared in internal.h), instantiated once per
// precision in kernels_f32.cu / kernels_f64.cu.
inline AxisPlan axis_of(const LaunchAxes& ax, int a) {
    AxisPlan p;
    p.n = ax.n[a];
    p.nst = ax.nst[a];
    for (int i = 0; i < kMaxStages; ++i) p.radix[i] = ax.radix[a][i];
    return p;
}

template <typename T> size_t Launch<T>::smem(int n) {
    return 2 * (size_t)n * kLd * sizeof(V2<T>) + (size_t)n * sizeof(V2<T>) + (size_t)n * sizeof(int) + 16;
}
template <typename T> size_t Launch<T>::smem_grad(int n) {
    return 3 * (size_t)n * kLd * sizeof(V2<T>) + (size_t)n * kLd * sizeof(double) + (size_t)n * sizeof(V2<T>) +
           (size_t)n * sizeof(int) + 16;
}
template <typename T> size_t Launch<T>::smem_dens(int n) {
    return 2 * (size_t)n * kLd * sizeof(V2<T>) + (size_t)n * sizeof(V2<T>) + (size_t)n * kLd * sizeof(double) +
           (size_t)n * sizeof(int) + 16;
}
template <typename T> int Launch<T>::set_limits(int nmax, int optin) {
    const int b = (int)smem(nmax);
    const int bg = (int)smem_grad(nmax);
    const int bd = (int)smem_dens(nmax);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k1_scatter_zpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k2_ypass<T, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k2_ypass<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k3_xpass_v<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k4_zpass_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if (bg <= optin && (e = cudaFuncSetAttribute(k3b_grad_v<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bg))) return e;
    if ((e = cudaFuncSetAttribute(k3_grid<T, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k3_grid<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if (bd <= optin && (e = cudaFuncSetAttribute(k3d_density<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bd))) return e;
    return 0;
}
template <typename T> int Launch<T>::twiddles(void* tw, int n, cudaStream_t st) {
    k_twiddles<T><<<(n + 127) / 128, 128, 0, st>>>((V2<T>*)tw, n);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k1(const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* coeffs, long long nb, void* cyl,
                  cudaStream_t st) {
    k1_scatter_zpass<T><<<dim3(t.T, (unsigned)nb), kThreads, smem(t.n3), st>>>(t, axis_of(ax, 2), (const V2<T>*)tw3,
                                                                               (const V2<T>*)coeffs, (V2<T>*)cyl);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k2(int sign, const DevTables& t, const LaunchAxes& ax, const void* tw2, long long nb, void* cyl,
                  void* slab, cudaStream_t st) {
    const dim3 grid(t.NP, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    if (sign > 0)
        k2_ypass<T, +1><<<grid, kThreads, smem(t.n2), st>>>(t, axis_of(ax, 1), (const V2<T>*)tw2, (V2<T>*)cyl, (V2<T>*)slab);
    else
        k2_ypass<T, -1><<<grid, kThreads, smem(t.n2), st>>>(t, axis_of(ax, 1), (const V2<T>*)tw2, (V2<T>*)cyl, (V2<T>*)slab);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k3(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* V, long long nb, void* slab,
                  cudaStream_t st) {
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    k3_xpass_v<T><<<grid, kThreads, smem(t.n1), st>>>(t, axis_of(ax, 0), (const V2<T>*)tw1, (const T*)V, (V2<T>*)slab);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k4(const DevTables& t, const LaunchAxes& ax, const void* tw3, const void* cyl, long long nb, void* out,
                  const void* diag, const void* cin, cudaStream_t st) {
    const T scale = (T)(1.0 / ((double)t.n1 * t.n2 * t.n3));
    k4_zpass_gather<T><<<dim3(t.T, (unsigned)nb), kThreads, smem(t.n3), st>>>(
        t, axis_of(ax, 2), (const V2<T>*)tw3, (const V2<T>*)cyl, (V2<T>*)out, scale, (const T*)diag, (const V2<T>*)cin);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k3b(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* sc, const void* sg,
                   long long nb, int ngroups, double* partial, cudaStream_t st) {
    const int bpg = (int)((nb + ngroups - 1) / ngroups);
    const int ng = (int)((nb + bpg - 1) / bpg);
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, ng);
    const double invN = 1.0 / ((double)t.n1 * t.n2 * t.n3);
    k3b_grad_v<T><<<grid, kThreads, smem_grad(t.n1), st>>>(t, axis_of(ax, 0), (const V2<T>*)tw1, (const V2<T>*)sc,
                                                           (const V2<T>*)sg, (int)nb, bpg, partial, invN);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k3g(int sign, const DevTables& t, const LaunchAxes& ax, const void* tw1, long long nb, void* slab,
                   void* grid, cudaStream_t st) {
    const dim3 grid3(t.n2, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    if (sign > 0)
        k3_grid<T, +1><<<grid3, kThreads, smem(t.n1), st>>>(t, axis_of(ax, 0), (const V2<T>*)tw1, (V2<T>*)slab,
                                                             (V2<T>*)grid);
    else
        k3_grid<T, -1><<<grid3, kThreads, smem(t.n1), st>>>(t, axis_of(ax, 0), (const V2<T>*)tw1, (V2<T>*)slab,
                                                             (V2<T>*)grid);
    return (int)cudaGetLastError();
}
template <typename T>
int Launch<T>::k3d(const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab, long long nb, int bpg,
                   const void* occ, long long b_base, int pair, long long nreal, double* partial, cudaStream_t st) {
    const int ng = (int)((nb + bpg - 1) / bpg);
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, ng);
    k3d_density<T><<<grid, kThreads, smem_dens(t.n1), st>>>(t, axis_of(ax, 0), (const V2<T>*)tw1, (const V2<T>*)slab,
                                                            (int)nb, bpg, (const T*)occ, b_base, pair, nreal, partial);
    return (int)cudaGetLastError();
}
template <typename T> int Launch<T>::finish_grad(const double* acc, void* g, long long N, cudaStream_t st) {
    k_finish_grad_v<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(acc, (T*)g, N);
    return (int)cudaGetLastError();
}

}  // namespace vloc
