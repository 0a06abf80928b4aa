// kernels_df.cuh -- compile-time-length chain kernels for FP64 data, one
// 16-byte value per lane slot (16-line tiles), in two arithmetics:
//  * PolNative: FP64 complex values (double2), FP64 instructions;
//  * PolDF: double-float (the double-float plan option), below.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so an FP64 chain is
// bound by its FP64 instructions.  Here the coefficients and the result stay
// FP64 in memory, while every transform runs on complex values whose parts
// are hi + lo pairs of FP32 (DFc, fft_core.cuh; the real and imaginary
// parts' operations paired in FP32 instructions): about 48 significant bits,
// the accuracy of an FP64 FFT to within a few units of 2^-48.  Each lane
// carries one line per slot, so a tile is 16 lines (z-pass: half of a
// 32-stick plan tile per CTA; y/x-passes: 16 consecutive z).  The cylinder
// and slab hold DFc (16 bytes, the size of an FP64 complex), V is converted
// to hi + lo once per call, and only the scatter and the gather convert
// between FP64 and double-float.  Same Stockham stages and compile-time
// schedules as the FP32 lane-pair kernels (fft_ct.cuh).
#pragma once

#include "fft_ct.cuh"
#include "kernels_impl.cuh"

namespace vloc {

constexpr int kLinesDF = 16;

// lane roles as in the FP32 lane-pair kernels: slot = line, two unit halves
__device__ __forceinline__ int slot_of_df() { return threadIdx.x & 15; }
__device__ __forceinline__ int sub_of_df() { return (threadIdx.x >> 4) & 1; }
__device__ __forceinline__ int warp_of_df() { return threadIdx.x >> 5; }

// Arithmetic policies: value type V, twiddle type TW, the V(r) element type
// VR, and the conversions at the scatter / gather / multiply by V.
struct PolDF {
    using V = DFc;
    using TW = TwDF;
    using VR = float2;  // V(r) as (hi, lo)
    __device__ __forceinline__ static DFc from(double2 v) { return df_from(v); }
    __device__ __forceinline__ static double2 out(DFc v, double scale) {
        const float2 sc = df_split(scale);
        return df_to(df2_mul(v, make_float2(sc.x, sc.x), make_float2(sc.y, sc.y)));
    }
    __device__ __forceinline__ static DFc mul_v(DFc h, float2 w) {
        return df2_mul(h, make_float2(w.x, w.x), make_float2(w.y, w.y));
    }
};
struct PolNative {
    using V = double2;
    using TW = double2;
    using VR = double;
    __device__ __forceinline__ static double2 from(double2 v) { return v; }
    __device__ __forceinline__ static double2 out(double2 v, double scale) { return cscale(v, scale); }
    __device__ __forceinline__ static double2 mul_v(double2 h, double w) { return cscale(h, w); }
};
template <int P> using PolOf = std::conditional_t<P == 0, PolDF, PolNative>;

// value as written to global memory (double-float values renormalised)
__device__ __forceinline__ DFc w_store(DFc v) { return df2_norm(v); }
__device__ __forceinline__ double2 w_store(double2 v) { return v; }

template <class Pol, int N> __host__ __device__ constexpr size_t w_smem() {
    return (size_t)N * kLdP * sizeof(float2) + (size_t)N * sizeof(typename Pol::TW) + (size_t)N * sizeof(int) + 16;
}


// element (row e, line l) of a tile buffer
template <class V> __device__ __forceinline__ V& w_at(float2* buf, int e, int l) {
    return *reinterpret_cast<V*>(buf + e * kLdP + 2 * l);
}

template <class TW> __device__ __forceinline__ void load_tww(TW* stw, const TW* __restrict__ tw, int n) {
    for (int j = threadIdx.x; j < n; j += kThreads) stw[j] = tw[j];
}

// Global row accessors (one DFc per slot)
template <class V> struct CylRowsD {  // rows = the plane's sticks (via rowmap), -1 = absent row
    V* cb;
    const int* rowmap;
    int n3, z0;
    __device__ __forceinline__ V operator()(int e, int slot) const {
        const int s = rowmap[e];
        return s >= 0 ? cb[s * n3 + z0 + slot] : czero<V>();
    }
    __device__ __forceinline__ void operator()(int e, int slot, V v) const {
        const int s = rowmap[e];
        if (s >= 0) cb[s * n3 + z0 + slot] = w_store(v);
    }
};
template <class V> struct SlabRowsD {  // every y row of one plane's tile
    V* p;           // slab[b][plane][0][z0]
    int n3;
    __device__ __forceinline__ V operator()(int e, int slot) const { return p[e * n3 + slot]; }
    __device__ __forceinline__ void operator()(int e, int slot, V v) const { p[e * n3 + slot] = w_store(v); }
};
template <class V> struct XRowsD {  // x rows at fixed y: the occupied planes
    V* sb;       // slab[b][0][y][z0]
    const int* xrow;
    int pstride;
    __device__ __forceinline__ V operator()(int e, int slot) const {
        const int p = xrow[e];
        return p >= 0 ? sb[p * pstride + slot] : czero<V>();
    }
    __device__ __forceinline__ void operator()(int e, int slot, V v) const {
        const int p = xrow[e];
        if (p >= 0) sb[p * pstride + slot] = w_store(v);
    }
};

// ------------------------------------------------------------------ K1
// CTA (tile, band, half): lines [16 half, 16 half + 16) of the plan tile.
template <class Pol, int N>
__device__ __forceinline__ void k1w_body(const DevTables& t, const typename Pol::TW* __restrict__ tw3,
                                         const double2* __restrict__ coeffs, typename Pol::V* __restrict__ cyl) {
    using V = typename Pol::V;
    using TW = typename Pol::TW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    TW* stw = reinterpret_cast<TW*>(buf + N * kLdP);
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int l0 = kLinesDF * (int)blockIdx.z;
    const int s0 = t.tile_ptr[tile] + l0;
    const int lines = min(kLinesDF, t.tile_ptr[tile + 1] - s0);
    if (lines <= 0) return;  // uniform over the CTA
    load_tww(stw, tw3, N);
    for (int i = threadIdx.x; i < N * kLdP / 2; i += kThreads)
        reinterpret_cast<float4*>(buf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const double2* c = coeffs + b * t.npw;
    for (int e = t.tile_pw_ptr[tile] + (int)threadIdx.x; e < t.tile_pw_ptr[tile + 1]; e += kThreads) {
        const int2 en = t.tile_pw[e];
        const int l = (en.y >> 16) - l0;
        if (l >= 0 && l < kLinesDF) w_at<V>(buf, en.y & 0xffff, l) = Pol::from(c[en.x]);
    }
    __syncthreads();
    fft_ct<N, +1, kWarps, false, true, true, V, TW>(stw, SmemT<V>{buf}, SmemT<V>{buf}, buf, slot_of_df(),
                                                       sub_of_df(), warp_of_df(), slot_of_df() < lines);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int l = threadIdx.x >> 5; l < lines; l += kWarps) {
        V* row = cyl + (b * t.S + t.tile_sticks[s0 + l]) * (long long)N;
        for (int z = lane; z < N; z += 32) row[z] = w_store(w_at<V>(buf, z, l));
    }
}

// Block floors for the double-float z- and y-passes at length 96 (the
// compiler's own choice leaves one or two resident CTAs per SM fewer):
// measured ms per 1024 bands at 96^3, own choice -> floor: K1 1.91 -> 1.76 (6
// CTAs, 80 registers) -> 1.66 (7, 72), inverse K2 3.74 -> 2.51 (6, 80) -> 2.46
// (7, 72), forward K2 3.09 -> 2.62 (7, 72; 8 measured 2.66), K4 1.95 -> 1.79
// (7, 72; 8 measured 1.82).  Floors make the compiler use registers up to the
// cap, so the other lengths keep its own choice.
template <class Pol, int N> constexpr bool df_floors() { return std::is_same<Pol, PolDF>::value && N == 96; }
#ifndef VLOC_MINB_K1DF
#define VLOC_MINB_K1DF 7
#endif
#ifndef VLOC_MINB_K2IDF
#define VLOC_MINB_K2IDF 7
#endif
#ifndef VLOC_MINB_K2FDF
#define VLOC_MINB_K2FDF 7
#endif
#ifndef VLOC_MINB_K4DF
#define VLOC_MINB_K4DF 7
#endif
// direct inverse z-pass (k1dw_body) where the dense z-band table exists
#ifndef VLOC_DF_DIRECT_Z
#define VLOC_DF_DIRECT_Z 1
#endif
template <class Pol, int N>
__global__ void __launch_bounds__(kThreads) k1_w(DevTables t, const typename Pol::TW* __restrict__ tw3,
                                                const double2* __restrict__ coeffs, typename Pol::V* __restrict__ cyl) {
    k1w_body<Pol, N>(t, tw3, coeffs, cyl);
}
template <class Pol, int N, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k1_wb(DevTables t, const typename Pol::TW* __restrict__ tw3,
                                                       const double2* __restrict__ coeffs,
                                                       typename Pol::V* __restrict__ cyl) {
    k1w_body<Pol, N>(t, tw3, coeffs, cyl);
}

// ------------------------------------------------- K1, direct form
// For plans whose plane waves all lie in the quarter band |l| <= n3/4 (the
// dense z-band table exists): each thread loads its own first-stage inputs,
// rows x = i + r NA of its line, through the table, and the rows outside the
// band are neither loaded nor transformed.  No buffer clearing and no
// scatter pass; the second stage and the row stores are those of k1w_body.
// Measured per 1024 bands at 96^3: double-float 1.54 against 1.66-1.76 ms,
// native 6.14 against 6.71 ms.  The mirror for K4 (the last forward stage
// storing each result straight to its caller position) measured slower,
// 2.01 against 1.78 ms (double-float) and 7.03 against 6.95 (native): its
// 16-byte stores go to 16 different sticks per instruction, where the tile
// form's gather writes the caller's band in order.
template <class Pol, int N>
__device__ __forceinline__ void k1dw_body(const DevTables& t, const typename Pol::TW* __restrict__ tw3,
                                          const double2* __restrict__ coeffs, typename Pol::V* __restrict__ cyl) {
    using V = typename Pol::V;
    using TW = typename Pol::TW;
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, NA = QR::NA, W = kWarps;
    constexpr int UA = (NA + 2 * W - 1) / (2 * W);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    TW* stw = reinterpret_cast<TW*>(buf + N * kLdP);
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int l0 = kLinesDF * (int)blockIdx.z;
    const int s0 = t.tile_ptr[tile] + l0;
    const int lines = min(kLinesDF, t.tile_ptr[tile + 1] - s0);
    if (lines <= 0) return;  // uniform over the CTA
    const int slot = slot_of_df(), sub = sub_of_df(), warp = warp_of_df();
    const bool act = slot < lines;
    // this slot's line of the plan tile (32 lines) in the table's rows
    const int* zd = t.zdense + (size_t)tile * (QR::groups() * NA) * kLines + l0 + slot;
    const double2* c = coeffs + b * t.npw;
    SmemT<V> sb{buf};
    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
                int e[R0];
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) != 0) e[r] = zd[(QR::group(r) * NA + i) * kLines];
                });
                V h[R0];
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) == 0) h[r] = czero<V>();
                    else h[r] = e[r] >= 0 ? Pol::from(c[e[r]]) : czero<V>();
                });
                DftZ<R0, +1, QR::mask()>::run(h);
#pragma unroll
                for (int r = 0; r < R0; ++r) sb(i * R0 + r, slot, h[r]);
            }
        }
    }
    load_tww(stw, tw3, N);
    __syncthreads();
    NatStage<N, +1, W, 1, V, TW>::template run<true>(stw, sb, sb, slot, sub, warp, act);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int l = threadIdx.x >> 5; l < lines; l += kWarps) {
        V* row = cyl + (b * t.S + t.tile_sticks[s0 + l]) * (long long)N;
        for (int z = lane; z < N; z += 32) row[z] = w_store(w_at<V>(buf, z, l));
    }
}
template <class Pol, int N>
__global__ void __launch_bounds__(kThreads) k1d_w(DevTables t, const typename Pol::TW* __restrict__ tw3,
                                                 const double2* __restrict__ coeffs, typename Pol::V* __restrict__ cyl) {
    k1dw_body<Pol, N>(t, tw3, coeffs, cyl);
}
template <class Pol, int N, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k1d_wb(DevTables t, const typename Pol::TW* __restrict__ tw3,
                                                        const double2* __restrict__ coeffs,
                                                        typename Pol::V* __restrict__ cyl) {
    k1dw_body<Pol, N>(t, tw3, coeffs, cyl);
}

// ------------------------------------------------------------------ K2
template <class Pol, int S, int N>
__device__ __forceinline__ void k2w_body(const DevTables& t, const typename Pol::TW* __restrict__ tw2,
                                         typename Pol::V* cyl, typename Pol::V* slab) {
    using V = typename Pol::V;
    using TW = typename Pol::TW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    TW* stw = reinterpret_cast<TW*>(buf + N * kLdP);
    int* rowmap = reinterpret_cast<int*>(stw + N);
    const int plane = blockIdx.x;
    const int z0 = blockIdx.y * kLinesDF;
    const long long b = blockIdx.z;
    const int lines = min(kLinesDF, n3 - z0);
    load_tww(stw, tw2, N);
    for (int e = threadIdx.x; e < N; e += kThreads) rowmap[e] = -1;
    __syncthreads();
    for (int s = t.plane_ptr[plane] + threadIdx.x; s < t.plane_ptr[plane + 1]; s += kThreads) rowmap[t.stick_row[s]] = s;
    __syncthreads();
    CylRowsD<V> cr{cyl + b * (long long)t.S * n3, rowmap, n3, z0};
    SlabRowsD<V> sr{slab + ((b * t.NP + plane) * (long long)N) * n3 + z0, n3};
    const bool act = slot_of_df() < lines;
    if constexpr (S > 0)
        fft_ct<N, +1, kWarps, false, false, false, V, TW>(stw, cr, sr, buf, slot_of_df(), sub_of_df(), warp_of_df(),
                                                             act);
    else
        fft_ct<N, -1, kWarps, false, false, false, V, TW>(stw, sr, cr, buf, slot_of_df(), sub_of_df(), warp_of_df(),
                                                             act);
}
template <class Pol, int S, int N>
__global__ void __launch_bounds__(kThreads) k2_w(DevTables t, const typename Pol::TW* __restrict__ tw2,
                                                typename Pol::V* cyl, typename Pol::V* slab) {
    k2w_body<Pol, S, N>(t, tw2, cyl, slab);
}
template <class Pol, int S, int N, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k2_wb(DevTables t, const typename Pol::TW* __restrict__ tw2,
                                                       typename Pol::V* cyl, typename Pol::V* slab) {
    k2w_body<Pol, S, N>(t, tw2, cyl, slab);
}

// ------------------------------------------------------------------ K3
// x-pass, x V(r) (V as hi + lo pairs), x-return; the last inverse stage, the
// multiply and the first forward stage of the reversed schedule in registers.
template <class Pol, int N>
__global__ void __launch_bounds__(kThreads) k3_w(DevTables t, const typename Pol::TW* __restrict__ tw1,
                                                const typename Pol::VR* __restrict__ Vr, typename Pol::V* slab) {
    using V = typename Pol::V;
    using TW = typename Pol::TW;
    using SC = Sched<N>;
    constexpr int nst = SC::nst;
    static_assert(nst >= 2, "compile-time x-pass needs at least two stages");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    TW* stw = reinterpret_cast<TW*>(buf + N * kLdP);
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int slot = slot_of_df(), sub = sub_of_df(), warp = warp_of_df();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLinesDF;
    const long long b = blockIdx.z;
    const int lines = min(kLinesDF, n3 - z0);
    const bool act = slot < lines;
    load_tww(stw, tw1, N);
    for (int e = threadIdx.x; e < N; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const int pstride = n2 * n3;
    XRowsD<V> xr{slab + b * t.NP * (long long)pstride + y * n3 + z0, xrow, pstride};
    const typename Pol::VR* vrow = Vr + (long long)y * n3 + z0 + slot;
    SmemT<V> sb{buf};

    NatStage<N, +1, kWarps, 0, V, TW>::template run<false>(stw, xr, sb, slot, sub, warp, act);
    __syncthreads();
    if constexpr (nst >= 3) {
        NatStage<N, +1, kWarps, 1, V, TW>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    if constexpr (nst >= 4) {
        NatStage<N, +1, kWarps, 2, V, TW>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    using L = NatStage<N, +1, kWarps, nst - 1, V, TW>;
    using F = RevStage<N, -1, kWarps, 0, V, TW>;
    constexpr int R = SC::R(nst - 1);
    static_assert(F::NI == L::NI && SC::RR(0) == R, "chained stages must share units");
    V h[L::U][R];
    if (act) {
        L::compute(h, stw, sb, slot, sub, warp);
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = 2 * (warp + u * kWarps) + sub;
            if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    h[u][r] = Pol::mul_v(h[u][r], vrow[(i + r * L::NI) * pstride]);
                }
                Dft<R, -1>::run(h[u]);
            }
        }
    }
    __syncthreads();
    if (act) F::store(h, sb, slot, sub, warp);
    __syncthreads();
    if constexpr (nst >= 3) {
        RevStage<N, -1, kWarps, 1, V, TW>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    if constexpr (nst >= 4) {
        RevStage<N, -1, kWarps, 2, V, TW>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    RevStage<N, -1, kWarps, nst - 1, V, TW>::template run<false>(stw, sb, xr, slot, sub, warp, act);
}

// ------------------------------------------------- K3, quarter-sphere form
// The x-pass of k3_w for the quarter-sphere x-plane set (QRows, fft_ct.cuh):
// rows known outside the cuboid are neither loaded nor transformed in the
// first inverse stage, and never formed in the last forward stage; the two
// table-twiddled stages read per-unit twiddle rows (twA / twB).
template <class Pol, int N> __host__ __device__ constexpr size_t k3q_w_smem() {
    return (size_t)N * kLdP * sizeof(float2) + 2 * (size_t)N * sizeof(typename Pol::TW);
}
template <class Pol, int N>
__global__ void __launch_bounds__(kThreads) k3q_w(DevTables t, const typename Pol::TW* __restrict__ tw1,
                                                 const typename Pol::VR* __restrict__ Vr, typename Pol::V* slab) {
    using V = typename Pol::V;
    using TW = typename Pol::TW;
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-sphere x-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int W = kWarps;
    constexpr int R0 = SC::R(0), R1 = SC::R(1);
    constexpr int NA = N / R0, NB = N / R1;
    constexpr int UA = (NA + 2 * W - 1) / (2 * W), UB = (NB + 2 * W - 1) / (2 * W);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    TW* twA = reinterpret_cast<TW*>(buf + N * kLdP);
    TW* twB = twA + N;
    const int n2 = t.n2, n3 = t.n3;
    const int slot = slot_of_df(), sub = sub_of_df(), warp = warp_of_df();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLinesDF;
    const long long b = blockIdx.z;
    const int lines = min(kLinesDF, n3 - z0);
    const bool act = slot < lines;
    for (int e = threadIdx.x; e < N; e += kThreads) {
        twA[e] = tw1[(e / R1) * (e % R1)];
        twB[e] = tw1[(e / R0) * (e % R0)];
    }
    __syncthreads();
    const int pstride = n2 * n3;
    V* sl = slab + b * t.NP * (long long)pstride + y * n3 + z0 + slot;
    const typename Pol::VR* vrow = Vr + (long long)y * n3 + z0 + slot;
    SmemT<V> sb{buf};

    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
                V h[R0];
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) == 0) h[r] = czero<V>();
                    else h[r] = QR::template inside<r>(i) ? sl[(i + QR::off(r)) * pstride] : czero<V>();
                });
                DftZ<R0, +1, QR::mask()>::run(h);
#pragma unroll
                for (int r = 0; r < R0; ++r) sb(i * R0 + r, slot, h[r]);
            }
        }
    }
    __syncthreads();
    V h[UB][R1];
    if (act) {
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NB % (2 * W) == 0 || i < NB) {
#pragma unroll
                for (int r = 0; r < R1; ++r) h[u][r] = sb(i + r * NB, slot);
                const TW* tw = twA + i * R1;
#pragma unroll
                for (int r = 1; r < R1; ++r) h[u][r] = cmul(h[u][r], tw[r]);
                Dft<R1, +1>::run(h[u]);
#pragma unroll
                for (int r = 0; r < R1; ++r) h[u][r] = Pol::mul_v(h[u][r], vrow[(i + r * NB) * pstride]);
                Dft<R1, -1>::run(h[u]);
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NB % (2 * W) == 0 || i < NB) {
#pragma unroll
                for (int r = 0; r < R1; ++r) sb(i * R1 + r, slot, h[u][r]);
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
                V g[R0];
#pragma unroll
                for (int r = 0; r < R0; ++r) g[r] = sb(i + r * NA, slot);
                const TW* tw = twB + i * R0;
#pragma unroll
                for (int r = 1; r < R0; ++r) g[r] = cmulc(g[r], tw[r]);
                Dft<R0, -1>::run(g);
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) != 0) {
                        if (QR::template inside<r>(i)) sl[(i + QR::off(r)) * pstride] = w_store(g[r]);
                    }
                });
            }
        }
    }
}

// ------------------------------------------------------------------ K4
template <class Pol, int N>
__device__ __forceinline__ void k4w_body(const DevTables& t, const typename Pol::TW* __restrict__ tw3,
                                         const typename Pol::V* __restrict__ cyl, double2* out, double scale,
                                         const double* __restrict__ diag, const double2* cin) {
    using V = typename Pol::V;
    using TW = typename Pol::TW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    TW* stw = reinterpret_cast<TW*>(buf + N * kLdP);
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int l0 = kLinesDF * (int)blockIdx.z;
    const int s0 = t.tile_ptr[tile] + l0;
    const int lines = min(kLinesDF, t.tile_ptr[tile + 1] - s0);
    if (lines <= 0) return;  // uniform over the CTA
    load_tww(stw, tw3, N);
    const int lane = threadIdx.x & 31;
    for (int l = threadIdx.x >> 5; l < lines; l += kWarps) {
        const V* row = cyl + (b * t.S + t.tile_sticks[s0 + l]) * (long long)N;
        for (int z = lane; z < N; z += 32) w_at<V>(buf, z, l) = row[z];
    }
    __syncthreads();
    fft_ct<N, -1, kWarps, false, true, true, V, TW>(stw, SmemT<V>{buf}, SmemT<V>{buf}, buf, slot_of_df(),
                                                       sub_of_df(), warp_of_df(), slot_of_df() < lines);
    __syncthreads();
    double2* o = out + b * t.npw;
    const double2* ci = diag ? cin + b * t.npw : cin;
    for (int e = t.tile_pw_ptr[tile] + (int)threadIdx.x; e < t.tile_pw_ptr[tile + 1]; e += kThreads) {
        const int2 en = t.tile_pw[e];
        const int l = (en.y >> 16) - l0;
        if (l < 0 || l >= kLinesDF) continue;
        double2 r = Pol::out(w_at<V>(buf, en.y & 0xffff, l), scale);
        if (diag) {  // H = diag + A (c is read before out is written: they may alias)
            const double d = diag[en.x];
            const double2 cc = ci[en.x];
            r.x += d * cc.x;
            r.y += d * cc.y;
        }
        o[en.x] = r;
    }
}

template <class Pol, int N>
__global__ void __launch_bounds__(kThreads) k4_w(DevTables t, const typename Pol::TW* __restrict__ tw3,
                                                const typename Pol::V* __restrict__ cyl, double2* out, double scale,
                                                const double* __restrict__ diag, const double2* cin) {
    k4w_body<Pol, N>(t, tw3, cyl, out, scale, diag, cin);
}
template <class Pol, int N, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k4_wb(DevTables t, const typename Pol::TW* __restrict__ tw3,
                                                       const typename Pol::V* __restrict__ cyl, double2* out,
                                                       double scale, const double* __restrict__ diag,
                                                       const double2* cin) {
    k4w_body<Pol, N>(t, tw3, cyl, out, scale, diag, cin);
}

// ------------------------------------------------------------ launchers
template <class Pol, int N> struct WSmem {
    static constexpr size_t sm = w_smem<Pol, N>();
    template <class K> static cudaError_t ensure(K kernel) {
        if (sm <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
};

template <int P, int N>
int LaunchF64<P, N>::k1(const DevTables& t, const void* tw3, const void* coeffs, long long nb, void* cyl,
                        cudaStream_t st) {
    using Pol = PolOf<P>;
    if constexpr (Sched<N>::nst == 2) {
        if (VLOC_DF_DIRECT_Z && t.zd_rows == QRows<N>::groups() * QRows<N>::NA) {
            if constexpr (df_floors<Pol, N>()) {
                static const cudaError_t onced = WSmem<Pol, N>::ensure(k1d_wb<Pol, N, VLOC_MINB_K1DF>);
                if (onced) return (int)onced;
                k1d_wb<Pol, N, VLOC_MINB_K1DF><<<dim3(t.T, (unsigned)nb, 2), kThreads, WSmem<Pol, N>::sm, st>>>(
                    t, (const typename Pol::TW*)tw3, (const double2*)coeffs, (typename Pol::V*)cyl);
            } else {
                static const cudaError_t onced = WSmem<Pol, N>::ensure(k1d_w<Pol, N>);
                if (onced) return (int)onced;
                k1d_w<Pol, N><<<dim3(t.T, (unsigned)nb, 2), kThreads, WSmem<Pol, N>::sm, st>>>(
                    t, (const typename Pol::TW*)tw3, (const double2*)coeffs, (typename Pol::V*)cyl);
            }
            return (int)cudaGetLastError();
        }
    }
    if constexpr (df_floors<Pol, N>()) {
        static const cudaError_t onceb = WSmem<Pol, N>::ensure(k1_wb<Pol, N, VLOC_MINB_K1DF>);
        if (onceb) return (int)onceb;
        k1_wb<Pol, N, VLOC_MINB_K1DF><<<dim3(t.T, (unsigned)nb, 2), kThreads, WSmem<Pol, N>::sm, st>>>(
            t, (const typename Pol::TW*)tw3, (const double2*)coeffs, (typename Pol::V*)cyl);
    } else {
        static const cudaError_t once = WSmem<Pol, N>::ensure(k1_w<Pol, N>);
        if (once) return (int)once;
        k1_w<Pol, N><<<dim3(t.T, (unsigned)nb, 2), kThreads, WSmem<Pol, N>::sm, st>>>(
            t, (const typename Pol::TW*)tw3, (const double2*)coeffs, (typename Pol::V*)cyl);
    }
    return (int)cudaGetLastError();
}
template <int P, int N>
int LaunchF64<P, N>::k2(int sign, const DevTables& t, const void* tw2, long long nb, void* cyl, void* slab,
                        cudaStream_t st) {
    using Pol = PolOf<P>;
    using V = typename Pol::V;
    const dim3 grid(t.NP, (t.n3 + kLinesDF - 1) / kLinesDF, (unsigned)nb);
    if constexpr (df_floors<Pol, N>()) {
        if (sign > 0) {
            static const cudaError_t onceb = WSmem<Pol, N>::ensure(k2_wb<Pol, +1, N, VLOC_MINB_K2IDF>);
            if (onceb) return (int)onceb;
            k2_wb<Pol, +1, N, VLOC_MINB_K2IDF><<<grid, kThreads, WSmem<Pol, N>::sm, st>>>(t, (const typename Pol::TW*)tw2, (V*)cyl,
                                                                            (V*)slab);
        } else {
            static const cudaError_t onceb = WSmem<Pol, N>::ensure(k2_wb<Pol, -1, N, VLOC_MINB_K2FDF>);
            if (onceb) return (int)onceb;
            k2_wb<Pol, -1, N, VLOC_MINB_K2FDF><<<grid, kThreads, WSmem<Pol, N>::sm, st>>>(t, (const typename Pol::TW*)tw2, (V*)cyl,
                                                                            (V*)slab);
        }
    } else {
        if (sign > 0) {
            static const cudaError_t once = WSmem<Pol, N>::ensure(k2_w<Pol, +1, N>);
            if (once) return (int)once;
            k2_w<Pol, +1, N><<<grid, kThreads, WSmem<Pol, N>::sm, st>>>(t, (const typename Pol::TW*)tw2, (V*)cyl,
                                                                        (V*)slab);
        } else {
            static const cudaError_t once = WSmem<Pol, N>::ensure(k2_w<Pol, -1, N>);
            if (once) return (int)once;
            k2_w<Pol, -1, N><<<grid, kThreads, WSmem<Pol, N>::sm, st>>>(t, (const typename Pol::TW*)tw2, (V*)cyl,
                                                                        (V*)slab);
        }
    }
    return (int)cudaGetLastError();
}
template <int P, int N>
int LaunchF64<P, N>::k3(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab,
                        cudaStream_t st) {
    using Pol = PolOf<P>;
    const dim3 grid(t.n2, (t.n3 + kLinesDF - 1) / kLinesDF, (unsigned)nb);
    if constexpr (Sched<N>::nst == 2) {
        if (t.xq) {
            constexpr size_t sm = k3q_w_smem<Pol, N>();
            static const cudaError_t onceq =
                sm <= 48 * 1024 ? cudaSuccess
                                : cudaFuncSetAttribute(k3q_w<Pol, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (onceq) return (int)onceq;
            k3q_w<Pol, N><<<grid, kThreads, sm, st>>>(t, (const typename Pol::TW*)tw1, (const typename Pol::VR*)V,
                                                      (typename Pol::V*)slab);
            return (int)cudaGetLastError();
        }
    }
    static const cudaError_t once = WSmem<Pol, N>::ensure(k3_w<Pol, N>);
    if (once) return (int)once;
    k3_w<Pol, N><<<grid, kThreads, WSmem<Pol, N>::sm, st>>>(t, (const typename Pol::TW*)tw1,
                                                           (const typename Pol::VR*)V, (typename Pol::V*)slab);
    return (int)cudaGetLastError();
}
template <int P, int N>
int LaunchF64<P, N>::k4(const DevTables& t, const void* tw3, const void* cyl, long long nb, void* out,
                        const void* diag, const void* cin, cudaStream_t st) {
    using Pol = PolOf<P>;
    const double scale = 1.0 / ((double)t.n1 * t.n2 * t.n3);
    if constexpr (df_floors<Pol, N>()) {
        static const cudaError_t onceb = WSmem<Pol, N>::ensure(k4_wb<Pol, N, VLOC_MINB_K4DF>);
        if (onceb) return (int)onceb;
        k4_wb<Pol, N, VLOC_MINB_K4DF><<<dim3(t.T, (unsigned)nb, 2), kThreads, WSmem<Pol, N>::sm, st>>>(
            t, (const typename Pol::TW*)tw3, (const typename Pol::V*)cyl, (double2*)out, scale, (const double*)diag,
            (const double2*)cin);
    } else {
        static const cudaError_t once = WSmem<Pol, N>::ensure(k4_w<Pol, N>);
        if (once) return (int)once;
        k4_w<Pol, N><<<dim3(t.T, (unsigned)nb, 2), kThreads, WSmem<Pol, N>::sm, st>>>(
            t, (const typename Pol::TW*)tw3, (const typename Pol::V*)cyl, (double2*)out, scale, (const double*)diag,
            (const double2*)cin);
    }
    return (int)cudaGetLastError();
}

}  // namespace vloc
