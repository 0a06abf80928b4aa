// kernels_zs.cuh -- the z-passes (K1 inverse z-FFT of each stick, K4 forward
// z-FFT of each stick) as warp-register transforms: one warp per pair of
// sticks, no shared memory and no block barrier.
//
// For n3 = 32 C (C = 1..4) a length-n3 line splits into C residue classes of
// 32 elements (Cooley-Tukey, Sec. 2's 1-D FFT sets along z):
//   inverse, classes of the input:  psi(n + 32 q) = sum_j W_C^{qj} W_n3^{nj} A_j[n],
//     A_j[n] = sum_m x(C m + j) W_32^{nm};
//   forward, classes of the output: X(C m + j) = sum_n W_32^{-mn} W_n3^{-jn} v_j[n],
//     v_j[n] = sum_q W_C^{-jq} y(n + 32 q).
// Lane i of the warp holds element i of each 32-point sequence; the 32-point
// DFTs run across the lanes as five radix-2 decimation-in-frequency exchange
// stages (warp shuffles), after which lane i holds output bitrev5(i).  The
// C-point DFTs and the twiddles W_n3^{nj} stay in each lane's registers.
//
// Caller positions come from the plan's class table zsh[S][n3]: entry
// [s][32 j + m] is the caller index of the plane wave of stick s at
// z = C m + j (l = z or z - n3), or -1.  So a warp's index loads are 128
// contiguous bytes, its coefficient loads (K1) and result stores (K4) go
// straight between the caller's band and registers, and its cylinder
// accesses are whole 256-byte blocks of one stick row.  Each lane carries
// the same element of two sticks (P2f), so the paired FP32 instructions serve
// both.  Plain plans only (Gamma-point pairs use the tile kernels).
#pragma once

#include "fft_ct.cuh"

#ifndef VLOC_ZS_WARPS
#define VLOC_ZS_WARPS 8
#endif
#ifndef VLOC_ZS_MINB
#define VLOC_ZS_MINB 4
#endif
#ifndef VLOC_ZS_PAIRS
#define VLOC_ZS_PAIRS 2  // stick pairs per warp (its twiddles are loaded once)
#endif

namespace vloc {

constexpr int kZsWarps = VLOC_ZS_WARPS;
constexpr int kZsThreads = 32 * kZsWarps;

template <int N> constexpr bool zs_length() { return N % 32 == 0 && N / 32 >= 1 && N / 32 <= 4; }

// This lane's exchange-stage constants for a 32-point DFT of sign S:
// stage k (half-span h = 16 >> k) combines lanes i and i ^ h; the lane with
// bit h clear keeps v + p, the other (p - v) W_{2h}^{S (i mod h)}.
// sg[k] = +1 / -1 for the two roles, w[k] the twiddle (1 for the first role;
// the last stage, h = 1, needs none).  tw is exp(+2 pi i k / N), k < N.
template <int N, int S>
__device__ __forceinline__ void zs_stage_consts(const float2* __restrict__ tw, int lane, float2 (&w)[4], float (&sg)[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int h = 16 >> k;
        const bool hi = (lane & h) != 0;
        sg[k] = hi ? -1.f : 1.f;
        if (k < 4) {
            float2 v = make_float2(1.f, 0.f);
            if (hi) {
                v = tw[(lane & (h - 1)) * (N / (2 * h))];
                if (S < 0) v.y = -v.y;
            }
            w[k] = v;
        }
    }
}

__device__ __forceinline__ P2f zs_shfl_xor(P2f v, int h) {
    P2f r;
    r.a.x = __shfl_xor_sync(0xffffffffu, v.a.x, h);
    r.a.y = __shfl_xor_sync(0xffffffffu, v.a.y, h);
    r.b.x = __shfl_xor_sync(0xffffffffu, v.b.x, h);
    r.b.y = __shfl_xor_sync(0xffffffffu, v.b.y, h);
    return r;
}

// 32-point DFT across the warp's lanes (lane i holds element i on entry and
// output bitrev5(i) on exit), for C independent sequences at once so their
// exchanges overlap.  Every lane of the warp must take part.
template <int C>
__device__ __forceinline__ void zs_dft32(P2f (&v)[C], const float2 (&w)[4], const float (&sg)[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int h = 16 >> k;
        P2f p[C];
#pragma unroll
        for (int j = 0; j < C; ++j) p[j] = zs_shfl_xor(v[j], h);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const P2f d = cfma(p[j], sg[k], v[j]);  // p + v or p - v
            if (k < 4) v[j] = cmul(d, w[k < 4 ? k : 0]);
            else v[j] = d;
        }
    }
}

__device__ __forceinline__ int zs_bitrev5(int i) { return (int)(__brev((unsigned)i) >> 27); }

// K1: inverse z-FFT of every stick, caller's band -> cylinder rows.
template <int N>
__global__ void __launch_bounds__(kZsThreads, VLOC_ZS_MINB) k1s_ct(DevTables t, const float2* __restrict__ tw3,
                                                                const float2* __restrict__ coeffs,
                                                                float2* __restrict__ cyl) {
    constexpr int C = N / 32;
    const int lane = threadIdx.x & 31;
    const int n = zs_bitrev5(lane);  // the output index this lane holds after the exchanges
    float2 w[4];
    float sg[5];
    zs_stage_consts<N, +1>(tw3, lane, w, sg);
    float2 wc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) wc[j] = j ? tw3[(n * j) % N] : make_float2(1.f, 0.f);
    const long long b = blockIdx.y;
    const float2* c = coeffs + b * t.npw;
    float2* cb = cyl + b * (long long)t.S * N;
    const int npair = (t.S + 1) / 2;
    for (int sp = blockIdx.x * kZsWarps + (int)(threadIdx.x >> 5); sp < npair; sp += gridDim.x * kZsWarps) {
        const int sa = 2 * sp;
        const bool two = sa + 1 < t.S;  // warp-uniform
        const int* za = t.zsh + (size_t)sa * N + lane;
        int ia[C], ib[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            ia[j] = za[32 * j];
            ib[j] = two ? za[N + 32 * j] : -1;
        }
        P2f x[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            x[j].a = ia[j] >= 0 ? c[ia[j]] : make_float2(0.f, 0.f);
            x[j].b = ib[j] >= 0 ? c[ib[j]] : make_float2(0.f, 0.f);
        }
        zs_dft32<C>(x, w, sg);
#pragma unroll
        for (int j = 1; j < C; ++j) x[j] = cmul(x[j], wc[j]);
        Dft<C, +1>::run(x);
        float2* ra = cb + (size_t)sa * N + n;
#pragma unroll
        for (int q = 0; q < C; ++q) {
            ra[32 * q] = x[q].a;
            if (two) ra[N + 32 * q] = x[q].b;
        }
    }
}

// K4: forward z-FFT of every stick, cylinder rows -> caller's band, times
// `scale`, plus diag times the input band for an H apply (each lane reads
// cin at a position before it writes out there, so the two may alias).
template <int N>
__global__ void __launch_bounds__(kZsThreads, VLOC_ZS_MINB) k4s_ct(DevTables t, const float2* __restrict__ tw3,
                                                                const float2* __restrict__ cyl, float2* out,
                                                                float scale, const float* __restrict__ diag,
                                                                const float2* cin) {
    constexpr int C = N / 32;
    const int lane = threadIdx.x & 31;
    const int m = zs_bitrev5(lane);  // the output class index this lane holds after the exchanges
    float2 w[4];
    float sg[5];
    zs_stage_consts<N, -1>(tw3, lane, w, sg);
    float2 wc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        wc[j] = j ? tw3[(lane * j) % N] : make_float2(1.f, 0.f);
        wc[j].y = -wc[j].y;
    }
    const long long b = blockIdx.y;
    const float2* cb = cyl + b * (long long)t.S * N;
    float2* o = out + b * t.npw;
    const float2* ci = cin + b * t.npw;
    const int npair = (t.S + 1) / 2;
    for (int sp = blockIdx.x * kZsWarps + (int)(threadIdx.x >> 5); sp < npair; sp += gridDim.x * kZsWarps) {
        const int sa = 2 * sp;
        const bool two = sa + 1 < t.S;  // warp-uniform
        const float2* ra = cb + (size_t)sa * N + lane;
        P2f y[C];
#pragma unroll
        for (int q = 0; q < C; ++q) {
            y[q].a = ra[32 * q];
            y[q].b = two ? ra[N + 32 * q] : make_float2(0.f, 0.f);
        }
        const int* za = t.zsh + (size_t)sa * N + m;
        int ia[C], ib[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            ia[j] = za[32 * j];
            ib[j] = two ? za[N + 32 * j] : -1;
        }
        Dft<C, -1>::run(y);
#pragma unroll
        for (int j = 1; j < C; ++j) y[j] = cmul(y[j], wc[j]);
        zs_dft32<C>(y, w, sg);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (diag) {
                if (ia[j] >= 0) {
                    const float d = diag[ia[j]];
                    const float2 cv = ci[ia[j]], v = cscale(y[j].a, scale);
                    o[ia[j]] = make_float2(v.x + d * cv.x, v.y + d * cv.y);
                }
                if (ib[j] >= 0) {
                    const float d = diag[ib[j]];
                    const float2 cv = ci[ib[j]], v = cscale(y[j].b, scale);
                    o[ib[j]] = make_float2(v.x + d * cv.x, v.y + d * cv.y);
                }
            } else {
                if (ia[j] >= 0) o[ia[j]] = cscale(y[j].a, scale);
                if (ib[j] >= 0) o[ib[j]] = cscale(y[j].b, scale);
            }
        }
    }
}

// Blocks per band: every warp takes VLOC_ZS_PAIRS stick pairs.
inline unsigned zs_blocks(int S) {
    const int npair = (S + 1) / 2;
    const int per = kZsWarps * VLOC_ZS_PAIRS;
    return (unsigned)((npair + per - 1) / per);
}

}  // namespace vloc
