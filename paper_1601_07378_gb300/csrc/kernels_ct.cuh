// kernels_ct.cuh -- the chain kernels with compile-time axis lengths (FP32).
//
// Same five steps as kernels_impl.cuh (K1 scatter + inverse z-pass, K2
// y-passes, K3 x-pass with V(r), K4 forward z-pass + gather), specialised
// for one axis length N per instantiation so the Stockham stages of
// fft_ct.cuh fold their index arithmetic.  Each lane carries two adjacent
// lines (one 16-byte vector), a tile uses one shared buffer, and K3 chains
// the inverse x-FFT's last stage, the multiply by V and the forward x-FFT's
// first stage in registers (no shared-memory round trip between the two
// transforms).  Instantiated for the common grid lengths (even, so a line
// pair is always 16-byte aligned) in kernels_ct_*.cu; other lengths use the
// runtime-radix kernels.
#pragma once

#include "fft_ct.cuh"
#include "kernels_impl.cuh"
#include "kernels_zs.cuh"
#include "bulk_ptx.cuh"

// Minimum resident CTAs per SM asked of the compiler (caps a kernel's
// registers at 65536 / (128 x MINB)).  Measured on GB300 at 96^3: the z- and
// y-pass kernels gain from more resident CTAs (K1, K2, K4: 6), the
// x-pass loses (its register-held chain wants the registers).  Applied up to
// length 96; longer lines keep the compiler's choice (the caps would spill).
#ifndef VLOC_MINB_K1
#define VLOC_MINB_K1 6
#endif
#ifndef VLOC_MINB_K2
#define VLOC_MINB_K2 6
#endif
#ifndef VLOC_MINB_K3
#define VLOC_MINB_K3 1
#endif
#ifndef VLOC_K3_WARPS
#define VLOC_K3_WARPS 4
#endif
// Warps per x-pass CTA by length, measured on GB300 (cubic grids, 1024
// bands): the units of a stage spread over 2 W slots, so 100 = 10 x 10 wants
// 5 warps and 120 = 12 x 10, 144 = 12 x 12 want 6 (K3 2.97 / 4.47 / 7.94 ms
// against 3.53 / 5.28 / 10.23 with 4); 96 and 128 keep 4.
constexpr int k3_warps(int n) { return n == 100 ? 5 : (n == 120 || n == 144) ? 6 : VLOC_K3_WARPS; }
// x-pass resident-CTA floors above length 96, measured on GB300 (cubic
// grids, 1024 bands; K3 ms without a floor -> with it): 100 (6 CTAs of 5
// warps) 2.96 -> 2.59, 120 (5 of 6) 4.44 -> 4.00, 128 (5 of 4) 4.16 -> 4.06,
// 144 (4 of 6) 7.88 -> 6.89.  One CTA more per SM spilled and measured slower
// at every length (144: 7.54).
constexpr int minb_k3(int n) {
    return n <= 96 ? VLOC_MINB_K3 : n == 100 ? 6 : n == 120 ? 5 : n == 128 ? 5 : n == 144 ? 4 : 1;
}
#ifndef VLOC_MINB_K4
#define VLOC_MINB_K4 6
#endif

namespace vloc {

constexpr int minb(int n, int m) { return n <= 96 ? m : 1; }
// Resident-CTA floors of the z/y-pass kernels above length 96, measured on
// GB300 (cubic grids, R = n/4, 1024 bands; floors 1, 4 and 5 compared, ms):
// K1 at 100: 0.57 with 5 against 0.64; K2 inverse at 100 / 120 / 128 / 144:
// 1.30 (5) / 2.35 (4) / 1.83 (5) / 3.87 (4) against 1.40 / 2.49 / 2.03 / 4.95;
// K2 forward at 100: 1.23 (5) against 1.45; K4 at 120: 1.07 (5) against 1.15.
// Elsewhere a floor measured the same or slower (K4 at 128: 1.59 with 4).
constexpr int minb_k1(int n) { return n <= 96 ? VLOC_MINB_K1 : n == 100 ? 5 : 1; }
constexpr int minb_k2(int n, int s) {
    return n <= 96 ? VLOC_MINB_K2
           : s > 0 ? ((n == 100 || n == 128) ? 5 : (n == 120 || n == 144) ? 4 : 1)
                   : (n == 100 ? 5 : 1);
}
constexpr int minb_k4(int n) { return n <= 96 ? VLOC_MINB_K4 : n == 120 ? 5 : 1; }

template <int N> __host__ __device__ constexpr size_t ct_smem() {
    return (size_t)N * kLdP * sizeof(float2) + (size_t)N * sizeof(float2) + (size_t)N * sizeof(int) + 16;
}

__device__ __forceinline__ int slot_of() { return threadIdx.x & 15; }
__device__ __forceinline__ int sub_of() { return (threadIdx.x >> 4) & 1; }
__device__ __forceinline__ int warp_of() { return threadIdx.x >> 5; }

// ------------------------------------------------------------- tile I/O
// Gamma-point real mode (Sec. 4.3): two real bands 2p, 2p + 1 travel as one
// complex band a + i b over the full G / -G list.  The z-passes can form
// that band from the caller's half-list arrays as they read them, and
// separate the two results as they write them, when every G shares a tile
// with its -G (DevTables::gok).
struct GammaArgs {
    long long nh;        // half-list plane waves per real band
    long long nreal;     // real bands of the call (the last pair may be half)
    const float* diag;   // H apply: real [nh] diagonal added in the gather, or null
    const float2* cin;   // the caller's bands [nreal][nh] (for diag)
};
// One batch of B of a tile's half-list entries {h, position of G, position
// of -G, 0} of a Gamma pair (real bands a and b, b null when absent): the
// entries and both bands' coefficients into registers, then a + i b at G and
// conj(a) + i conj(b) at -G into the tile buffer (the real parts at G = 0,
// whose two positions coincide).
template <int B>
__device__ __forceinline__ void gamma_load(const int4* __restrict__ ent, int base, int e1, const float2* __restrict__ a,
                                           const float2* __restrict__ b, int4 (&en)[B], float2 (&va)[B],
                                           float2 (&vb)[B]) {
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int e = base + u * kThreads;
        en[u] = e < e1 ? ent[e] : make_int4(-1, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
        va[u] = en[u].x >= 0 ? a[en[u].x] : make_float2(0.f, 0.f);
        vb[u] = (en[u].x >= 0 && b) ? b[en[u].x] : make_float2(0.f, 0.f);
    }
}
template <int B>
__device__ __forceinline__ void gamma_store(float2* buf, const int4 (&en)[B], const float2 (&va)[B],
                                            const float2 (&vb)[B]) {
#pragma unroll
    for (int u = 0; u < B; ++u) {
        if (en[u].x < 0) continue;
        float2* pg = buf + (en[u].y & 0xffff) * kLdP + (en[u].y >> 16);
        if (en[u].y == en[u].z) {
            *pg = make_float2(va[u].x, vb[u].x);
        } else {
            *pg = make_float2(va[u].x - vb[u].y, va[u].y + vb[u].x);
            buf[(en[u].z & 0xffff) * kLdP + (en[u].z >> 16)] = make_float2(va[u].x + vb[u].y, vb[u].x - va[u].y);
        }
    }
}
// One batch of B of a tile's plane-wave entries starting at `base` (stride
// kThreads): the entries and their coefficients into registers, then into
// the tile buffer.
template <int B>
__device__ __forceinline__ void entries_load_p(const int2* __restrict__ ent, int base, int e1,
                                               const float2* __restrict__ c, int2 (&en)[B], float2 (&val)[B]) {
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int e = base + u * kThreads;
        en[u] = e < e1 ? ent[e] : make_int2(0, -1);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) val[u] = en[u].y >= 0 ? c[en[u].x] : make_float2(0.f, 0.f);
}
template <int B>
__device__ __forceinline__ void entries_store_p(float2* buf, const int2 (&en)[B], const float2 (&val)[B]) {
#pragma unroll
    for (int u = 0; u < B; ++u)
        if (en[u].y >= 0) buf[(en[u].y & 0xffff) * kLdP + (en[u].y >> 16)] = val[u];
}
// Clear the tile buffer (N rows) and scatter the tile's plane waves into it;
// the first batch's loads are issued before the clearing so their latency
// hides behind it.  Ends with a barrier.  Batches of VLOC_SCATTER_BATCH
// entries per thread (a 32-stick tile holds about 1000 plane waves at 96^3,
// 8 per thread).
#ifndef VLOC_SCATTER_BATCH
#define VLOC_SCATTER_BATCH 8
#endif
template <int N>
__device__ __forceinline__ void scatter_tile_p(const int2* __restrict__ ent, int e0, int e1,
                                               const float2* __restrict__ c, float2* buf) {
    constexpr int B = VLOC_SCATTER_BATCH;
    int2 en[B];
    float2 val[B];
    const int base0 = e0 + (int)threadIdx.x;
    entries_load_p<B>(ent, base0, e1, c, en, val);
    for (int i = threadIdx.x; i < N * kLdP / 2; i += kThreads)
        reinterpret_cast<float4*>(buf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    entries_store_p<B>(buf, en, val);
    for (int base = base0 + B * kThreads; base < e1; base += B * kThreads) {
        entries_load_p<B>(ent, base, e1, c, en, val);
        entries_store_p<B>(buf, en, val);
    }
    __syncthreads();
}
// The same for a Gamma pair p of the caller's real bands (GammaArgs).
template <int N>
__device__ __forceinline__ void scatter_tile_gamma(const DevTables& t, int tile, const float2* __restrict__ coeffs,
                                                   long long p, const GammaArgs& g, float2* buf) {
    constexpr int B = VLOC_SCATTER_BATCH;
    int4 en[B];
    float2 va[B], vb[B];
    const float2* a = coeffs + 2 * p * g.nh;
    const float2* b = 2 * p + 1 < g.nreal ? coeffs + (2 * p + 1) * g.nh : nullptr;
    const int e0 = t.gamma_h_ptr[tile], e1 = t.gamma_h_ptr[tile + 1];
    const int base0 = e0 + (int)threadIdx.x;
    gamma_load<B>(t.gamma_h, base0, e1, a, b, en, va, vb);
    for (int i = threadIdx.x; i < N * kLdP / 2; i += kThreads)
        reinterpret_cast<float4*>(buf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    gamma_store<B>(buf, en, va, vb);
    for (int base = base0 + B * kThreads; base < e1; base += B * kThreads) {
        gamma_load<B>(t.gamma_h, base, e1, a, b, en, va, vb);
        gamma_store<B>(buf, en, va, vb);
    }
    __syncthreads();
}
#ifndef VLOC_GATHER_BATCH
#define VLOC_GATHER_BATCH 8
#endif
__device__ __forceinline__ void gather_entries_p(const int2* __restrict__ ent, int e0, int e1, const float2* buf,
                                                 float2* o, float scale, const float* __restrict__ diag,
                                                 const float2* cin) {
    constexpr int GB = VLOC_GATHER_BATCH;
    for (int base = e0 + (int)threadIdx.x; base < e1; base += GB * kThreads) {
        int2 en[GB];
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const int e = base + u * kThreads;
            en[u] = e < e1 ? ent[e] : make_int2(0, -1);
        }
        if (diag) {  // H = diag + A (c is read before out is written: they may alias)
            float d[GB];
            float2 ci[GB];
#pragma unroll
            for (int u = 0; u < GB; ++u)
                if (en[u].y >= 0) { d[u] = diag[en[u].x]; ci[u] = cin[en[u].x]; }
#pragma unroll
            for (int u = 0; u < GB; ++u)
                if (en[u].y >= 0) {
                    const float2 v = cscale(buf[(en[u].y & 0xffff) * kLdP + (en[u].y >> 16)], scale);
                    o[en[u].x] = make_float2(v.x + d[u] * ci[u].x, v.y + d[u] * ci[u].y);
                }
        } else {
#pragma unroll
            for (int u = 0; u < GB; ++u)
                if (en[u].y >= 0) o[en[u].x] = cscale(buf[(en[u].y & 0xffff) * kLdP + (en[u].y >> 16)], scale);
        }
    }
}
// Gamma-point gather of pair p: for every half-list plane wave of the tile,
// U(G) and U(-G) (both in the tile buffer, times 1/N) give the two real
// bands' results, A a = (U(G) + conj U(-G)) / 2 and A b = (U(G) - conj
// U(-G)) / 2i, plus diag times the band for an H apply.
__device__ __forceinline__ void gather_gamma(const int4* __restrict__ ent, int e0, int e1, const float2* buf,
                                             float2* oa, float2* ob, float scale, const float* __restrict__ diag,
                                             const float2* ca, const float2* cb) {
    for (int e = e0 + (int)threadIdx.x; e < e1; e += kThreads) {
        const int4 en = ent[e];
        const float2 x = cscale(buf[(en.y & 0xffff) * kLdP + (en.y >> 16)], scale);   // U(G)
        const float2 y = cscale(buf[(en.z & 0xffff) * kLdP + (en.z >> 16)], scale);   // U(-G)
        float2 a = make_float2((x.x + y.x) * 0.5f, (x.y - y.y) * 0.5f);
        float2 b = make_float2((x.y + y.y) * 0.5f, (y.x - x.x) * 0.5f);
        if (diag) {  // c is read before out is written (they may alias)
            const float d = diag[en.x];
            const float2 va = ca[en.x];
            a.x += d * va.x; a.y += d * va.y;
            if (ob) {
                const float2 vb = cb[en.x];
                b.x += d * vb.x; b.y += d * vb.y;
            }
        }
        oa[en.x] = a;
        if (ob) ob[en.x] = b;
    }
}
template <bool GM>
__device__ __forceinline__ void gather_tile(const DevTables& t, int tile, const float2* buf, float2* out, long long b,
                                            float scale, const float* diag, const float2* cin, const GammaArgs& g) {
    if constexpr (!GM) {
        gather_entries_p(t.tile_pw, t.tile_pw_ptr[tile], t.tile_pw_ptr[tile + 1], buf, out + b * t.npw, scale, diag,
                         diag ? cin + b * t.npw : cin);
    } else {
        const bool two = 2 * b + 1 < g.nreal;
        gather_gamma(t.gamma_h, t.gamma_h_ptr[tile], t.gamma_h_ptr[tile + 1], buf, out + 2 * b * g.nh,
                     two ? out + (2 * b + 1) * g.nh : nullptr, scale, g.diag, g.cin + 2 * b * g.nh,
                     g.cin + (2 * b + 1) * g.nh);
    }
}
// Tile rows <-> cylinder, a line pair (2s, 2s + 1) per warp pass: lane j
// moves elements z = j, j + 32, ... of both lines as one 16-byte shared-memory
// access (rows are 272 bytes apart, so the 16-byte accesses of a warp hit
// distinct banks; one line per lane would be a 2-way conflict) and two
// coalesced global accesses, one per stick.
template <int NN>
__device__ __forceinline__ void rows_out_p(const float2* buf, float2* __restrict__ cb, const int* sticks, int lines) {
    constexpr int K = (NN + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int sp = threadIdx.x >> 5; 2 * sp < lines; sp += kWarps) {
        const bool two = 2 * sp + 1 < lines;
        float2* row0 = cb + (long long)sticks[2 * sp] * NN;
        float2* row1 = cb + (long long)sticks[two ? 2 * sp + 1 : 2 * sp] * NN;
        P2f v[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (NN % 32 == 0 || lane + 32 * k < NN)
                v[k] = *reinterpret_cast<const P2f*>(buf + (lane + 32 * k) * kLdP + 2 * sp);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (NN % 32 == 0 || lane + 32 * k < NN) {
                row0[lane + 32 * k] = v[k].a;
                if (two) row1[lane + 32 * k] = v[k].b;
            }
    }
}
template <int NN>
__device__ __forceinline__ void rows_in_p(float2* buf, const float2* __restrict__ cb, const int* sticks, int lines) {
    constexpr int K = (NN + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int sp = threadIdx.x >> 5; 2 * sp < lines; sp += kWarps) {
        const bool two = 2 * sp + 1 < lines;
        const float2* row0 = cb + (long long)sticks[2 * sp] * NN;
        const float2* row1 = cb + (long long)sticks[two ? 2 * sp + 1 : 2 * sp] * NN;
        P2f v[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (NN % 32 == 0 || lane + 32 * k < NN) {
                v[k].a = row0[lane + 32 * k];
                v[k].b = two ? row1[lane + 32 * k] : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (NN % 32 == 0 || lane + 32 * k < NN)
                *reinterpret_cast<P2f*>(buf + (lane + 32 * k) * kLdP + 2 * sp) = v[k];
    }
}

// Global row accessors for line pairs (z0 even, rows of even length).
struct CylRowsP {  // rows = the plane's sticks (via rowmap), -1 = absent row
    float2* cb;
    const int* rowmap;
    int n3, z0;
    __device__ __forceinline__ P2f operator()(int e, int slot) const {
        const int s = rowmap[e];
        return s >= 0 ? *reinterpret_cast<const P2f*>(cb + s * n3 + z0 + 2 * slot) : czero<P2f>();
    }
    __device__ __forceinline__ void operator()(int e, int slot, P2f v) const {
        const int s = rowmap[e];
        if (s >= 0) *reinterpret_cast<P2f*>(cb + s * n3 + z0 + 2 * slot) = v;
    }
};
struct SlabRowsP {  // every y row of one plane's tile
    float2* p;       // slab[b][plane][0][z0]
    int n3;
    __device__ __forceinline__ P2f operator()(int e, int slot) const {
        return *reinterpret_cast<const P2f*>(p + e * n3 + 2 * slot);
    }
    __device__ __forceinline__ void operator()(int e, int slot, P2f v) const {
        *reinterpret_cast<P2f*>(p + e * n3 + 2 * slot) = v;
    }
};
struct XRowsP {  // x rows at fixed y: the occupied planes
    float2* sb;      // slab[b][0][y][z0]
    const int* xrow;
    int pstride;  // n2 * n3 (in-band offsets stay 32-bit)
    __device__ __forceinline__ P2f operator()(int e, int slot) const {
        const int p = xrow[e];
        return p >= 0 ? *reinterpret_cast<const P2f*>(sb + p * pstride + 2 * slot) : czero<P2f>();
    }
    __device__ __forceinline__ void operator()(int e, int slot, P2f v) const {
        const int p = xrow[e];
        if (p >= 0) *reinterpret_cast<P2f*>(sb + p * pstride + 2 * slot) = v;
    }
};

// ------------------------------------------------------------------ K1
template <int N, bool GM = false>
__global__ void __launch_bounds__(kThreads, minb_k1(N)) k1_ct(DevTables t, const float2* __restrict__ tw3,
                                                 const float2* __restrict__ coeffs, float2* __restrict__ cyl,
                                                 GammaArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    load_tw<float>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    if constexpr (GM) scatter_tile_gamma<N>(t, tile, coeffs, b, g, buf);
    else scatter_tile_p<N>(t.tile_pw, t.tile_pw_ptr[tile], t.tile_pw_ptr[tile + 1], coeffs + b * t.npw, buf);
    fft_ct<N, +1, kWarps, false, true, true>(stw, SmemP{buf}, SmemP{buf}, buf, slot_of(), sub_of(), warp_of(),
                                             2 * slot_of() < lines);
    __syncthreads();
    rows_out_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
}

// ------------------------------------------------- K1, quarter-band form
// When every plane wave has |l| <= N/4 (a sphere of radius n3/4: the z rows
// of each stick lie in the band of Fig. 5), only the rows the first inverse
// stage reads are cleared, and that stage skips the rows known to be zero.
// The first batch of the tile's entries and coefficients is requested before
// the clearing, the twiddle table after the scatter.  GM: a Gamma-point pair per block,
// formed from the caller's two real bands as they are read.
template <int N, bool GM = false>
__global__ void __launch_bounds__(kThreads, minb_k1(N)) k1q_ct(DevTables t, const float2* __restrict__ tw3,
                                                  const float2* __restrict__ coeffs, float2* __restrict__ cyl,
                                                  GammaArgs g) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-band z-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, NA = QR::NA, W = kWarps;
    constexpr int UA = (NA + 2 * W - 1) / (2 * W);
    constexpr int B = VLOC_SCATTER_BATCH;
    constexpr int RW = kLdP / 2;  // float4 per row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    auto clear_read_rows = [&] {
        for (int i = threadIdx.x; i < N * RW; i += kThreads)
            if (xq_row_read<N>(i / RW)) reinterpret_cast<float4*>(buf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    if constexpr (GM) {
        int4 en[B];
        float2 va[B], vb[B];
        const float2* a = coeffs + 2 * b * g.nh;
        const float2* bb = 2 * b + 1 < g.nreal ? coeffs + (2 * b + 1) * g.nh : nullptr;
        const int e0 = t.gamma_h_ptr[tile], e1 = t.gamma_h_ptr[tile + 1];
        const int base0 = e0 + (int)threadIdx.x;
        gamma_load<B>(t.gamma_h, base0, e1, a, bb, en, va, vb);
        clear_read_rows();
        __syncthreads();
        gamma_store<B>(buf, en, va, vb);
        for (int base = base0 + B * kThreads; base < e1; base += B * kThreads) {
            gamma_load<B>(t.gamma_h, base, e1, a, bb, en, va, vb);
            gamma_store<B>(buf, en, va, vb);
        }
    } else {
        int2 en[B];
        float2 val[B];
        const float2* c = coeffs + b * t.npw;
        const int e0 = t.tile_pw_ptr[tile], e1 = t.tile_pw_ptr[tile + 1];
        const int base0 = e0 + (int)threadIdx.x;
        entries_load_p<B>(t.tile_pw, base0, e1, c, en, val);
        clear_read_rows();
        __syncthreads();
        entries_store_p<B>(buf, en, val);
        for (int base = base0 + B * kThreads; base < e1; base += B * kThreads) {
            entries_load_p<B>(t.tile_pw, base, e1, c, en, val);
            entries_store_p<B>(buf, en, val);
        }
    }
    load_tw<float>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    const bool act = 2 * slot < lines;
    __syncthreads();
    SmemP sb{buf};
    // first inverse stage in place (every unit's values in registers, then stored)
    P2f h[UA][R0];
    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) == 0) h[u][r] = czero<P2f>();
                    else h[u][r] = sb(i + r * NA, slot);
                });
                DftZ<R0, +1, QR::mask()>::run(h[u]);
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
#pragma unroll
                for (int r = 0; r < R0; ++r) sb(i * R0 + r, slot, h[u][r]);
            }
        }
    }
    __syncthreads();
    NatStage<N, +1, W, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
    __syncthreads();
    rows_out_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
}

// ------------------------------------------------- K1, direct form
// The quarter-band z-pass without the tile scatter: each thread loads its
// own first-stage inputs through the dense z-band table (row x = i + r NA,
// two lines per lane), so the tile buffer needs no clearing and the first
// stage no shared-memory round trip before it.  Plain (complex) plans only:
// for Gamma-point pairs the scatter over half-list entries, which reads each
// pair of real coefficients once for G and -G, measured faster (0.207
// against 0.298 ms per 1024 real bands at 96^3).
#ifndef VLOC_K1_DIRECT
#define VLOC_K1_DIRECT 1
#endif
// RUNS: the caller's list in stick order (DevTables::runs); each line's
// inputs are addressed from its run (first caller index, its l, count)
// instead of the dense table.
template <int N, bool RUNS>
__global__ void __launch_bounds__(kThreads, minb_k1(N)) k1d_ct(DevTables t, const float2* __restrict__ tw3,
                                                  const float2* __restrict__ coeffs, float2* __restrict__ cyl) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-band z-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, NA = QR::NA, W = kWarps;
    constexpr int UA = (NA + 2 * W - 1) / (2 * W);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int* zd = t.zdense + (size_t)tile * (QR::groups() * NA) * kLines + 2 * slot;
    const float2* c = coeffs + b * t.npw;
    auto coef = [&](int x) { return x == -1 ? make_float2(0.f, 0.f) : c[x]; };
    SmemP sb{buf};
#pragma unroll
    for (int u = 0; u < UA; ++u) {
        const int i = 2 * (warp + u * W) + sub;
        if (NA % (2 * W) == 0 || i < NA) {
            P2f h[R0];
            if constexpr (RUNS) {
                const int lines = t.tile_ptr[tile + 1] - t.tile_ptr[tile];
                const int4* rt = t.run_tab + (size_t)tile * kLines + 2 * slot;
                const int4 ra = 2 * slot < lines ? rt[0] : make_int4(0, 0, 0, 0);
                const int4 rb = 2 * slot + 1 < lines ? rt[1] : make_int4(0, 0, 0, 0);
                auto at = [&](const int4& rr, int x) {
                    const int p = (x <= N / 2 ? x : x - N) - rr.y;
                    return (p >= 0 && p < rr.z) ? c[rr.x + p] : make_float2(0.f, 0.f);
                };
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) == 0) h[r] = czero<P2f>();
                    else h[r] = P2f{at(ra, i + r * NA), at(rb, i + r * NA)};
                });
            } else {
                int2 e[R0];
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) != 0)
                        e[r] = *reinterpret_cast<const int2*>(zd + (QR::group(r) * NA + i) * kLines);
                });
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) == 0) h[r] = czero<P2f>();
                    else h[r] = P2f{coef(e[r].x), coef(e[r].y)};
                });
            }
            DftZ<R0, +1, QR::mask()>::run(h);
#pragma unroll
            for (int r = 0; r < R0; ++r) sb(i * R0 + r, slot, h[r]);
        }
    }
    load_tw<float>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    const bool act = 2 * slot < lines;
    __syncthreads();
    NatStage<N, +1, W, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
    __syncthreads();
    rows_out_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
}

// ------------------------------------------------- K1, bulk-staged form
// For caller lists in stick order (every stick's plane waves consecutive with
// l ascending and no gap, as the canonical order gives) each stick of the
// tile is one contiguous run of the band's coefficients.  Lane l of warp 0
// stages run l in shared memory: one 1-D bulk copy of its 16-byte-aligned
// interior, completing on the block's mbarrier, and plain loads of the at
// most two 8-byte end elements.  The threads then take their first-stage
// inputs (row x = i + r NA of each of their two lines) from the staged runs
// at position l(x) - lmin.  The staged runs share the tile buffer, so the
// first stage's results wait in registers for a barrier.  The wait is
// bounded: a copy that has not landed within about a second sets the error
// flag, and the block waits (bounded) for its copies and returns.
#ifndef VLOC_K1_BULK
#define VLOC_K1_BULK 1
#endif
template <int N> constexpr int k1b_run_stride() { return (N / 2 + 3) & ~1; }  // >= count + 1, even
template <int N> constexpr size_t k1b_smem() { return ct_smem<N>() + 16; }  // + mbarrier and flag
template <int N>
__global__ void __launch_bounds__(kThreads, minb_k1(N)) k1b_ct(DevTables t, const float2* __restrict__ tw3,
                                                  const float2* __restrict__ coeffs, float2* __restrict__ cyl) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-band z-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, NA = QR::NA, W = kWarps;
    constexpr int UA = (NA + 2 * W - 1) / (2 * W);
    constexpr int RS = k1b_run_stride<N>();
    static_assert(kLines * RS <= N * kLdP, "the staged runs fit in the tile buffer");
    static_assert(ct_smem<N>() % 8 == 0, "mbarrier alignment");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + ct_smem<N>());
    int* okf = reinterpret_cast<int*>(bar + 1);
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    const float2* c = coeffs + b * t.npw;
    const int4* rt = t.run_tab + (size_t)tile * kLines;
    if (threadIdx.x == 0) {
        mbar_init(bar, 32);
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {
        const int lane = threadIdx.x;
        unsigned bytes = 0;
        const float2* src = nullptr;
        float2* dst = nullptr;
        if (lane < lines) {
            const int4 r = rt[lane];
            const float2* run = c + r.x;
            const int a = (int)((reinterpret_cast<uintptr_t>(run) >> 3) & 1);  // element 0 off the 16-byte grid
            const int n2 = (r.z - a) & ~1;                                     // aligned interior, even length
            float2* st = buf + lane * RS;  // element p at slot p + a
            if (a) st[1] = run[0];
            if ((r.z - a) & 1) st[r.z - 1 + a] = run[r.z - 1];
            if (n2 > 0) {
                bytes = 8u * (unsigned)n2;
                src = run + a;
                dst = st + 2 * a;
            }
        }
        mbar_expect_tx(bar, bytes);  // every lane of warp 0 arrives once
        if (bytes) bulk_load_1d(dst, src, bytes, bar);
    }
    load_tw<float>(stw, tw3, N);
    if (threadIdx.x == 0) *okf = mbar_wait_bounded(bar, 0) ? 1 : 0;
    __syncthreads();
    if (!*okf) {  // the same for every thread of the block
        if (threadIdx.x == 0) {
            if (t.err) atomicExch(t.err, 1);
            mbar_wait_bounded(bar, 0);
        }
        return;
    }
    const int la = 2 * slot, lb = la + 1;
    const int4 ra = la < lines ? rt[la] : make_int4(0, 0, 0, 0);
    const int4 rb = lb < lines ? rt[lb] : make_int4(0, 0, 0, 0);
    const int aa = (int)((reinterpret_cast<uintptr_t>(c + ra.x) >> 3) & 1);
    const int ab = (int)((reinterpret_cast<uintptr_t>(c + rb.x) >> 3) & 1);
    auto staged = [&](const int4& r, int a, int line, int x) {
        const int p = (x <= N / 2 ? x : x - N) - r.y;
        return (p >= 0 && p < r.z) ? buf[line * RS + p + a] : make_float2(0.f, 0.f);
    };
    SmemP sb{buf};
    P2f h[UA][R0];
#pragma unroll
    for (int u = 0; u < UA; ++u) {
        const int i = 2 * (warp + u * W) + sub;
        if (NA % (2 * W) == 0 || i < NA) {
            sfor<R0>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                if constexpr (QR::kind(r) == 0) h[u][r] = czero<P2f>();
                else h[u][r] = P2f{staged(ra, aa, la, i + r * NA), staged(rb, ab, lb, i + r * NA)};
            });
            DftZ<R0, +1, QR::mask()>::run(h[u]);
        }
    }
    __syncthreads();  // every staged run has been read
#pragma unroll
    for (int u = 0; u < UA; ++u) {
        const int i = 2 * (warp + u * W) + sub;
        if (NA % (2 * W) == 0 || i < NA) {
#pragma unroll
            for (int r = 0; r < R0; ++r) sb(i * R0 + r, slot, h[u][r]);
        }
    }
    __syncthreads();
    const bool act = 2 * slot < lines;
    NatStage<N, +1, W, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
    __syncthreads();
    rows_out_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
}

// ------------------------------------------------------------------ K2
template <int S, int N>
__global__ void __launch_bounds__(kThreads, minb_k2(N, S)) k2_ct(DevTables t, const float2* __restrict__ tw2, float2* cyl,
                                                 float2* slab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    int* rowmap = reinterpret_cast<int*>(stw + N);
    const int plane = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<float>(stw, tw2, N);
    for (int e = threadIdx.x; e < N; e += kThreads) rowmap[e] = -1;
    __syncthreads();
    for (int s = t.plane_ptr[plane] + threadIdx.x; s < t.plane_ptr[plane + 1]; s += kThreads) rowmap[t.stick_row[s]] = s;
    __syncthreads();
    CylRowsP cr{cyl + b * (long long)t.S * n3, rowmap, n3, z0};
    SlabRowsP sr{slab + ((b * t.NP + plane) * (long long)N) * n3 + z0, n3};
    const bool act = 2 * slot_of() < lines;
    if constexpr (S > 0) fft_ct<N, +1, kWarps, false, false, false>(stw, cr, sr, buf, slot_of(), sub_of(), warp_of(), act);
    else fft_ct<N, -1, kWarps, false, false, false>(stw, sr, cr, buf, slot_of(), sub_of(), warp_of(), act);
}

// ------------------------------------------------------------------ K3
// W warps per CTA (the tile is always 32 lines; more warps split its units).
template <int N, int W>
__global__ void __launch_bounds__(32 * W, minb_k3(N)) k3_ct(DevTables t, const float2* __restrict__ tw1,
                                                 const float* __restrict__ Vr, float2* slab) {
    using SC = Sched<N>;
    constexpr int nst = SC::nst;
    static_assert(nst >= 2, "compile-time x-pass needs at least two stages");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    const bool act = 2 * slot < lines;
    for (int e = threadIdx.x; e < N; e += 32 * W) {
        stw[e] = tw1[e];
        xrow[e] = t.xrow_plane[e];
    }
    __syncthreads();
    const int pstride = n2 * n3;
    XRowsP xr{slab + b * t.NP * (long long)pstride + y * n3 + z0, xrow, pstride};
    const float* vrow = Vr + (long long)y * n3 + z0 + 2 * slot;
    SmemP sb{buf};

    // inverse x-FFT, stages 0 .. nst-2 (global rows -> buffer)
    NatStage<N, +1, W, 0>::template run<false>(stw, xr, sb, slot, sub, warp, act);
    __syncthreads();
    if constexpr (nst >= 3) {
        NatStage<N, +1, W, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    if constexpr (nst >= 4) {
        NatStage<N, +1, W, 2>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    // last inverse stage -> psi(x) * V(x, y, z) -> first forward stage of the
    // reversed schedule, in registers: both work on elements i + r N/R.
    using L = NatStage<N, +1, W, nst - 1>;
    using F = RevStage<N, -1, W, 0>;
    constexpr int R = SC::R(nst - 1);
    static_assert(F::NI == L::NI && SC::RR(0) == R, "chained stages must share units");
    P2f h[L::U][R];
    if (act) {
        L::compute(h, stw, sb, slot, sub, warp);
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (L::NI % (2 * W) == 0 || i < L::NI) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 w = *reinterpret_cast<const float2*>(vrow + (i + r * L::NI) * pstride);
                    h[u][r].a = cscale(h[u][r].a, w.x);
                    h[u][r].b = cscale(h[u][r].b, w.y);
                }
                Dft<R, -1>::run(h[u]);
            }
        }
    }
    __syncthreads();
    if (act) F::store(h, sb, slot, sub, warp);
    __syncthreads();
    // forward x-FFT, remaining stages (buffer -> occupied global rows)
    if constexpr (nst >= 3) {
        RevStage<N, -1, W, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    if constexpr (nst >= 4) {
        RevStage<N, -1, W, 2>::template run<true>(stw, sb, sb, slot, sub, warp, act);
        __syncthreads();
    }
    RevStage<N, -1, W, nst - 1>::template run<false>(stw, sb, xr, slot, sub, warp, act);
}

// ------------------------------------------------- K3, quarter-sphere form
// Twiddle tables of the two table-twiddled stages of a two-stage length
// N = R0 R1, one row per unit residue k: twA[k][r] = w^(k r), k < R0, r < R1
// (the inverse stage that ends the first transform) and twB[k][r] = w^(k r),
// k < R1, r < R0 (the forward stage that ends the second), w = exp(2 pi i /
// N), so a unit reads its R - 1 twiddles at consecutive addresses.
template <int N> __host__ __device__ constexpr size_t k3q_smem() {
    return (size_t)N * kLdP * sizeof(float2) + 2 * (size_t)N * sizeof(float2);
}

#ifndef VLOC_MINB_K3Q
#define VLOC_MINB_K3Q 6
#endif
// chain units left over after the full rounds run as single-line tasks
// spread over every thread (1), or as a partial round of line-pair units (0)
#ifndef VLOC_K3Q_SPLIT
#define VLOC_K3Q_SPLIT 1
#endif

#ifndef VLOC_MINB_K3Q_96
#define VLOC_MINB_K3Q_96 7  // 72 registers, no spills: 1.547 against 1.572 ms per 1024 bands with 6 (8: 1.69)
#endif
#ifndef VLOC_MINB_K3Q_100
#define VLOC_MINB_K3Q_100 6
#endif
#ifndef VLOC_MINB_K3Q_120
#define VLOC_MINB_K3Q_120 5
#endif
#ifndef VLOC_MINB_K3Q_128
#define VLOC_MINB_K3Q_128 5
#endif
#ifndef VLOC_MINB_K3Q_144
#define VLOC_MINB_K3Q_144 4
#endif
constexpr int minb_k3q(int n) {
    return n == 96 ? VLOC_MINB_K3Q_96 : n < 96 ? VLOC_MINB_K3Q : n == 100 ? VLOC_MINB_K3Q_100 : n == 120 ? VLOC_MINB_K3Q_120
           : n == 128 ? VLOC_MINB_K3Q_128 : n == 144 ? VLOC_MINB_K3Q_144 : 1;
}
// FLAT: tiles of 16 consecutive line pairs of the band (any even n3);
// otherwise block (y, 32-z tile, band) for n3 a multiple of 32 (the same
// tiles without the per-lane division that maps a flat index to (y, z pair)).
template <int N, int W, bool FLAT = true>
__global__ void __launch_bounds__(32 * W, minb_k3q(N)) k3q_ct(DevTables t, const float2* __restrict__ tw1,
                                                  const float* __restrict__ Vr, float2* slab) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-sphere x-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int R0 = SC::R(0), R1 = SC::R(1);
    constexpr int NA = N / R0;  // units of the first inverse and the last forward stage
    constexpr int NB = N / R1;  // units of the chained middle stage
    constexpr int UA = (NA + 2 * W - 1) / (2 * W);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* twA = buf + N * kLdP;
    float2* twB = twA + N;
    const int n2 = t.n2, n3 = t.n3;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    // tile = 16 consecutive line pairs (y, z pair) of the band in y-major
    // order, so a tile may span two y rows and none is ragged (n3 / 2 line
    // pairs per y row; 3 tiles a row at n3 = 96)
    const int hz = n3 >> 1, npairs = n2 * hz;
    const long long b = blockIdx.z;
    // flat line-pair index of slot s (its tile's first pair + s)
    const int fbase = FLAT ? (int)blockIdx.x * 16 : (int)blockIdx.x * hz + (int)blockIdx.y * 16;
    auto pair_of = [&](int s) { return min(fbase + s, npairs - 1); };
    const bool act = fbase + slot < npairs;
    int y, zq;
    if constexpr (FLAT) {
        const int f = pair_of(slot);
        y = f / hz;
        zq = 2 * (f - y * hz);
    } else {
        y = blockIdx.x;
        zq = (int)blockIdx.y * kLines + 2 * slot;
    }
    // twiddle rows (first read after the barrier that ends stage 0, which
    // needs none)
    for (int e = threadIdx.x; e < N; e += 32 * W) {
        twA[e] = tw1[(e / R1) * (e % R1)];
        twB[e] = tw1[(e / R0) * (e % R0)];
    }
    const int pstride = n2 * n3;
    float2* sl = slab + b * t.NP * (long long)pstride + y * n3 + zq;  // plane 0, this lane's pair
    const float* vrow = Vr + (long long)y * n3 + zq;
    SmemP sb{buf};

    // inverse x-FFT, first stage (radix R0, no twiddles): global rows -> buffer
    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
                P2f h[R0];
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) == 0) h[r] = czero<P2f>();
                    else h[r] = QR::template inside<r>(i) ? *reinterpret_cast<const P2f*>(sl + (i + QR::off(r)) * pstride)
                                                          : czero<P2f>();
                });
                DftZ<R0, +1, QR::mask()>::run(h);
#pragma unroll
                for (int r = 0; r < R0; ++r) sb(i * R0 + r, slot, h[r]);
            }
        }
    }
    __syncthreads();
    // last inverse stage -> psi(x) V(x, y, z) -> first forward stage, in
    // registers (unit i holds x = i + r NB in both).  FR full rounds give
    // every unit slot a line-pair unit; the LU units left over are split into
    // single lines (32 line tasks per unit) spread over all threads, so no
    // warp waits at the next barrier for a half-empty round.
    constexpr int FR = VLOC_K3Q_SPLIT ? NB / (2 * W) : (NB + 2 * W - 1) / (2 * W);
    constexpr int LU = VLOC_K3Q_SPLIT ? NB % (2 * W) : 0;
    constexpr int LT = (LU * 32 + 32 * W - 1) / (32 * W);  // line tasks per thread
    auto chain = [&](auto& hv, int i, const float* vr, auto vload) {
        const float2* tw = twA + i * R1;  // i < NB = R0
#pragma unroll
        for (int r = 1; r < R1; ++r) hv[r] = cmul(hv[r], tw[r]);
        Dft<R1, +1>::run(hv);
#pragma unroll
        for (int r = 0; r < R1; ++r) vload(hv[r], vr + (i + r * NB) * pstride);
        Dft<R1, -1>::run(hv);
    };
    P2f h[FR > 0 ? FR : 1][R1];
    float2 hl[LT > 0 ? LT : 1][R1];
    if (act) {
#pragma unroll
        for (int u = 0; u < FR; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NB % (2 * W) != 0 && i >= NB) continue;
#pragma unroll
            for (int r = 0; r < R1; ++r) h[u][r] = sb(i + r * NB, slot);
            chain(h[u], i, vrow, [](P2f& v, const float* q) {
                const float2 w = *reinterpret_cast<const float2*>(q);
                v.a = cscale(v.a, w.x);
                v.b = cscale(v.b, w.y);
            });
        }
    }
    if constexpr (LU > 0) {
#pragma unroll
        for (int k = 0; k < LT; ++k) {
            const int tk = threadIdx.x + k * 32 * W;  // line task: unit, slot, line
            const int i = FR * 2 * W + tk / 32, ls = (tk >> 1) & 15, ln = tk & 1;
            if (tk < LU * 32 && fbase + ls < npairs) {
                int yl, zl;
                if constexpr (FLAT) {
                    const int fl = pair_of(ls);
                    yl = fl / hz;
                    zl = 2 * (fl - yl * hz);
                } else {
                    yl = y;
                    zl = (int)blockIdx.y * kLines + 2 * ls;
                }
#pragma unroll
                for (int r = 0; r < R1; ++r) hl[k][r] = buf[(i + r * NB) * kLdP + 2 * ls + ln];
                chain(hl[k], i, Vr + (long long)yl * n3 + zl + ln, [](float2& v, const float* q) { v = cscale(v, *q); });
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int u = 0; u < FR; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NB % (2 * W) != 0 && i >= NB) continue;
#pragma unroll
            for (int r = 0; r < R1; ++r) sb(i * R1 + r, slot, h[u][r]);
        }
    }
    if constexpr (LU > 0) {
#pragma unroll
        for (int k = 0; k < LT; ++k) {
            const int tk = threadIdx.x + k * 32 * W;
            const int i = FR * 2 * W + tk / 32, ls = (tk >> 1) & 15, ln = tk & 1;
            if (tk < LU * 32 && fbase + ls < npairs) {
#pragma unroll
                for (int r = 0; r < R1; ++r) buf[(i * R1 + r) * kLdP + 2 * ls + ln] = hl[k][r];
            }
        }
    }
    __syncthreads();
    // forward x-FFT, last stage (radix R0, twiddled): buffer -> the occupied
    // global rows; outputs of rows outside the cuboid are never formed
    if (act) {
#pragma unroll
        for (int u = 0; u < UA; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NA % (2 * W) == 0 || i < NA) {
                P2f g[R0];
#pragma unroll
                for (int r = 0; r < R0; ++r) g[r] = sb(i + r * NA, slot);
                const float2* tw = twB + i * R0;  // i < NA = R1
#pragma unroll
                for (int r = 1; r < R0; ++r) g[r] = cmulc(g[r], tw[r]);
                Dft<R0, -1>::run(g);
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) != 0) {
                        if (QR::template inside<r>(i)) *reinterpret_cast<P2f*>(sl + (i + QR::off(r)) * pstride) = g[r];
                    }
                });
            }
        }
    }
}

// ------------------------------------------------------------------ K4
template <int N, bool GM = false>
__global__ void __launch_bounds__(kThreads, minb_k4(N)) k4_ct(DevTables t, const float2* __restrict__ tw3,
                                                 const float2* __restrict__ cyl, float2* out, float scale,
                                                 const float* __restrict__ diag, const float2* cin, GammaArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    load_tw<float>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    rows_in_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
    __syncthreads();
    fft_ct<N, -1, kWarps, false, true, true>(stw, SmemP{buf}, SmemP{buf}, buf, slot_of(), sub_of(), warp_of(),
                                             2 * slot_of() < lines);
    __syncthreads();
    gather_tile<GM>(t, tile, buf, out, b, scale, diag, cin, g);
}

// ------------------------------------------------- K4, quarter-band form
// The forward z-pass in the reversed schedule, whose last stage (radix R0)
// writes row x = i + r NA of unit i: rows outside the band |l| <= N/4 are
// never gathered, so they are never formed.
// Gamma-point pairs at length 96: seven resident CTAs per SM (72 registers, no
// spills), 0.195 against 0.209 ms per 1024 real bands.
constexpr int minb_k4q(int n, bool gm) { return gm && n == 96 ? 7 : minb_k4(n); }
template <int N, bool GM = false>
__global__ void __launch_bounds__(kThreads, minb_k4q(N, GM)) k4q_ct(DevTables t, const float2* __restrict__ tw3,
                                                  const float2* __restrict__ cyl, float2* out, float scale,
                                                  const float* __restrict__ diag, const float2* cin, GammaArgs g) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-band z-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, W = kWarps;
    using L = RevStage<N, -1, W, 1>;  // radix R0, rows i + r NA
    static_assert(L::NI == QR::NA, "last forward stage rows");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    load_tw<float>(stw, tw3, N);
    rows_in_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
    __syncthreads();
    const bool act = 2 * slot < lines;
    SmemP sb{buf};
    RevStage<N, -1, W, 0>::template run<true>(stw, sb, sb, slot, sub, warp, act);
    __syncthreads();
    P2f h[L::U][R0];
    if (act) L::compute(h, stw, sb, slot, sub, warp);
    __syncthreads();
    if (act) {
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (L::NI % (2 * W) == 0 || i < L::NI) {
                sfor<R0>([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    if constexpr (QR::kind(r) != 0) sb(i + r * QR::NA, slot, h[u][r]);
                });
            }
        }
    }
    __syncthreads();
    gather_tile<GM>(t, tile, buf, out, b, scale, diag, cin, g);
}

// ------------------------------------------------- K4, direct form
// k4q_ct without the gather pass: the last forward stage (radix R0, rows
// x = i + r NA, the row structure of the dense z-band table) writes each
// result straight to its caller position, times 1/N, plus diag times the
// band for an H apply.  Plain plans with the dense table.  (Positions worked
// out from each line's stick run, as k1d_ct reads its inputs, measured
// slower here: 0.369 against 0.365 ms per 1024 bands at 96^3.)
#ifndef VLOC_K4_DIRECT
#define VLOC_K4_DIRECT 1
#endif
// Seven resident CTAs per SM at length 96 (72 registers, no spills): 0.365
// against 0.383 ms per 1024 bands with six; the other lengths keep K4's floors.
constexpr int minb_k4d(int n) { return n == 96 ? 7 : minb_k4(n); }
template <int N>
__global__ void __launch_bounds__(kThreads, minb_k4d(N)) k4d_ct(DevTables t, const float2* __restrict__ tw3,
                                                  const float2* __restrict__ cyl, float2* out, float scale,
                                                  const float* __restrict__ diag, const float2* cin) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-band z-pass: two-stage lengths");
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, NA = QR::NA, W = kWarps;
    using L = RevStage<N, -1, W, 1>;  // radix R0, rows i + r NA
    static_assert(L::NI == NA, "last forward stage rows");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int tile = blockIdx.x;
    const long long b = blockIdx.y;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    load_tw<float>(stw, tw3, N);
    const int s0 = t.tile_ptr[tile], lines = t.tile_ptr[tile + 1] - s0;
    rows_in_p<N>(buf, cyl + b * (long long)t.S * N, t.tile_sticks + s0, lines);
    __syncthreads();
    const bool act = 2 * slot < lines;
    SmemP sb{buf};
    RevStage<N, -1, W, 0>::template run<true>(stw, sb, sb, slot, sub, warp, act);
    __syncthreads();
    if (!act) return;
    const int* zd = t.zdense + (size_t)tile * (QR::groups() * NA) * kLines + 2 * slot;
    float2* o = out + b * t.npw;
    const float2* ci = cin + b * t.npw;
#pragma unroll
    for (int u = 0; u < L::U; ++u) {
        const int i = 2 * (warp + u * W) + sub;
        if (L::NI % (2 * W) == 0 || i < L::NI) {
            int2 e[R0];
            sfor<R0>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                if constexpr (QR::kind(r) != 0)
                    e[r] = *reinterpret_cast<const int2*>(zd + (QR::group(r) * NA + i) * kLines);
            });
            P2f h[R0];
            L::compute_unit(h, stw, sb, i, slot);
            sfor<R0>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                if constexpr (QR::kind(r) != 0) {
                    const int xa = e[r].x, xb = e[r].y;
                    if (diag) {  // H = diag + A (c is read before out is written: they may alias)
                        if (xa != -1) {
                            const float d = diag[xa];
                            const float2 cv = ci[xa], v = cscale(h[r].a, scale);
                            o[xa] = make_float2(v.x + d * cv.x, v.y + d * cv.y);
                        }
                        if (xb != -1) {
                            const float d = diag[xb];
                            const float2 cv = ci[xb], v = cscale(h[r].b, scale);
                            o[xb] = make_float2(v.x + d * cv.x, v.y + d * cv.y);
                        }
                    } else {
                        if (xa != -1) o[xa] = cscale(h[r].a, scale);
                        if (xb != -1) o[xb] = cscale(h[r].b, scale);
                    }
                }
            });
        }
    }
}

// ----------------------------------------------------------------- K3b
// dL/dV x-pass for one (y, z tile, band group): psi = inverse x-FFT of the
// c-slab tile (kept in buffer A), g = inverse x-FFT of the grad-slab tile
// (its last stage stays in registers), acc += Re(conj(g) psi) per element in
// FP32 over the group's bands (at most 16), then the group's partial sum,
// times 1/N, is written in FP64; groups are added later in a fixed order.
template <int N>
__global__ void __launch_bounds__(kThreads) k3b_ct(DevTables t, const float2* __restrict__ tw1,
                                                  const float2* slab_c, const float2* slab_g, int nb, int bpg,
                                                  double* __restrict__ partial, double invN) {
    using SC = Sched<N>;
    constexpr int nst = SC::nst;
    static_assert(nst >= 2, "compile-time x-pass needs at least two stages");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* bufA = reinterpret_cast<float2*>(smem_raw);
    float2* bufB = bufA + N * kLdP;
    float2* stw = bufB + N * kLdP;
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const int grp = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    const bool act = 2 * slot < lines;
    load_tw<float>(stw, tw1, N);
    for (int e = threadIdx.x; e < N; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const int pstride = n2 * n3;
    using L = NatStage<N, +1, kWarps, nst - 1>;
    constexpr int R = SC::R(nst - 1);
    float2 acc[L::U][R];
#pragma unroll
    for (int u = 0; u < L::U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[u][r] = make_float2(0.f, 0.f);
    SmemP sa{bufA}, sb{bufB};
    const int b1 = min(nb, (grp + 1) * bpg);
    for (int b = grp * bpg; b < b1; ++b) {
        XRowsP xc{const_cast<float2*>(slab_c) + (long long)b * t.NP * pstride + y * n3 + z0, xrow, pstride};
        XRowsP xg{const_cast<float2*>(slab_g) + (long long)b * t.NP * pstride + y * n3 + z0, xrow, pstride};
        fft_ct<N, +1, kWarps, false, false, true>(stw, xc, sa, bufA, slot, sub, warp, act);  // psi -> A
        NatStage<N, +1, kWarps, 0>::template run<false>(stw, xg, sb, slot, sub, warp, act);
        __syncthreads();
        if constexpr (nst >= 3) {
            NatStage<N, +1, kWarps, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        if constexpr (nst >= 4) {
            NatStage<N, +1, kWarps, 2>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        if (act) {
#pragma unroll
            for (int u = 0; u < L::U; ++u) {
                const int i = 2 * (warp + u * kWarps) + sub;
                if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
                    P2f h[R];
                    L::compute_unit(h, stw, sb, i, slot);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const P2f p = sa(i + r * L::NI, slot);
                        acc[u][r].x += h[r].a.x * p.a.x + h[r].a.y * p.a.y;
                        acc[u][r].y += h[r].b.x * p.b.x + h[r].b.y * p.b.y;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (act) {
        double* part = partial + (long long)grp * t.n1 * pstride + y * n3 + z0 + 2 * slot;
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = 2 * (warp + u * kWarps) + sub;
            if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    double* q = part + (i + r * L::NI) * pstride;
                    q[0] = (double)acc[u][r].x * invN;
                    q[1] = (double)acc[u][r].y * invN;
                }
            }
        }
    }
}

// dL/dV x-pass for the quarter-sphere plane set: k3b_ct with the first
// inverse stage of both transforms reading only the cuboid's rows.
#ifndef VLOC_MINB_K3BQ
#define VLOC_MINB_K3BQ 1
#endif
template <int N>
__global__ void __launch_bounds__(kThreads, VLOC_MINB_K3BQ) k3bq_ct(DevTables t, const float2* __restrict__ tw1,
                                                   const float2* slab_c, const float2* slab_g, int nb, int bpg,
                                                   double* __restrict__ partial, double invN) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-sphere x-pass: two-stage lengths");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* bufA = reinterpret_cast<float2*>(smem_raw);
    float2* bufB = bufA + N * kLdP;
    float2* stw = bufB + N * kLdP;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const int grp = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    const bool act = 2 * slot < lines;
    load_tw<float>(stw, tw1, N);
    __syncthreads();
    const int pstride = n2 * n3;
    using L = NatStage<N, +1, kWarps, 1>;
    constexpr int R = SC::R(1);
    float2 acc[L::U][R];
#pragma unroll
    for (int u = 0; u < L::U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[u][r] = make_float2(0.f, 0.f);
    SmemP sa{bufA}, sb{bufB};
    const int b1 = min(nb, (grp + 1) * bpg);
    for (int b = grp * bpg; b < b1; ++b) {
        const long long off = (long long)b * t.NP * pstride + y * n3 + z0 + 2 * slot;
        const float2* xc = slab_c + off;
        const float2* xg = slab_g + off;
        if (act) {
            xq_first_inverse<N, kWarps, P2f>([&](int p) { return *reinterpret_cast<const P2f*>(xc + p * pstride); },
                                             sa, slot, sub, warp);
            xq_first_inverse<N, kWarps, P2f>([&](int p) { return *reinterpret_cast<const P2f*>(xg + p * pstride); },
                                             sb, slot, sub, warp);
        }
        __syncthreads();
        L::template run<true>(stw, sa, sa, slot, sub, warp, act);  // psi complete in A
        __syncthreads();
        if (act) {
#pragma unroll
            for (int u = 0; u < L::U; ++u) {
                const int i = 2 * (warp + u * kWarps) + sub;
                if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
                    P2f h[R];
                    L::compute_unit(h, stw, sb, i, slot);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const P2f p = sa(i + r * L::NI, slot);
                        acc[u][r].x += h[r].a.x * p.a.x + h[r].a.y * p.a.y;
                        acc[u][r].y += h[r].b.x * p.b.x + h[r].b.y * p.b.y;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (act) {
        double* part = partial + (long long)grp * t.n1 * pstride + y * n3 + z0 + 2 * slot;
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = 2 * (warp + u * kWarps) + sub;
            if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    double* q = part + (i + r * L::NI) * pstride;
                    q[0] = (double)acc[u][r].x * invN;
                    q[1] = (double)acc[u][r].y * invN;
                }
            }
        }
    }
}

// ------------------------------------------- half transforms and density
struct GridRowsP {  // x line pair at fixed (y, z0 + 2 slot) of a full grid
    float2* g;      // grid[b][0][y][z0]
    int pstride;
    __device__ __forceinline__ P2f operator()(int e, int slot) const {
        return *reinterpret_cast<const P2f*>(g + e * pstride + 2 * slot);
    }
    __device__ __forceinline__ void operator()(int e, int slot, P2f v) const {
        *reinterpret_cast<P2f*>(g + e * pstride + 2 * slot) = v;
    }
};

// S = +1: slab tile -> full grid (inverse x-pass, input pruned to the
// occupied planes); S = -1: full grid -> slab tile (forward, output pruned).
template <int S, int N>
__global__ void __launch_bounds__(kThreads) k3g_ct(DevTables t, const float2* __restrict__ tw1, float2* slab,
                                                  float2* grid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const long long b = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    load_tw<float>(stw, tw1, N);
    for (int e = threadIdx.x; e < N; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const int pstride = n2 * n3;
    XRowsP xr{slab + b * t.NP * (long long)pstride + y * n3 + z0, xrow, pstride};
    GridRowsP gr{grid + b * (long long)N * pstride + y * n3 + z0, pstride};
    const bool act = 2 * slot_of() < lines;
    if constexpr (S > 0) fft_ct<N, +1, kWarps, false, false, false>(stw, xr, gr, buf, slot_of(), sub_of(), warp_of(), act);
    else fft_ct<N, -1, kWarps, false, false, false>(stw, gr, xr, buf, slot_of(), sub_of(), warp_of(), act);
}

// Density x-pass for one (y, z tile, band group): each band's inverse
// x-pass ends in registers, where the weighted |psi|^2 is added in FP32 over
// the group's bands (at most 16); the group's partial sum is stored as it is,
// in FP32 (half the bytes of an FP64 copy, and nothing rounded), and the
// groups are added later in FP64 in a fixed order.
template <int N>
__global__ void __launch_bounds__(kThreads, minb(N, 5)) k3d_ct(DevTables t, const float2* __restrict__ tw1, const float2* slab,
                                                  int nb, int bpg, const float* __restrict__ occ, long long b_base,
                                                  int pair, long long nreal, float* __restrict__ partial) {
    using SC = Sched<N>;
    constexpr int nst = SC::nst;
    static_assert(nst >= 2, "compile-time x-pass needs at least two stages");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const int grp = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    const bool act = 2 * slot < lines;
    load_tw<float>(stw, tw1, N);
    for (int e = threadIdx.x; e < N; e += kThreads) xrow[e] = t.xrow_plane[e];
    __syncthreads();
    const int pstride = n2 * n3;
    using L = NatStage<N, +1, kWarps, nst - 1>;
    constexpr int R = SC::R(nst - 1);
    float2 acc[L::U][R];
#pragma unroll
    for (int u = 0; u < L::U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[u][r] = make_float2(0.f, 0.f);
    SmemP sb{buf};
    const int b1 = min(nb, (grp + 1) * bpg);
    for (int b = grp * bpg; b < b1; ++b) {
        double wxd, wyd;
        density_weights(occ, b_base + b, pair, nreal, wxd, wyd);
        const float wx = (float)wxd, wy = (float)wyd;
        XRowsP xc{const_cast<float2*>(slab) + (long long)b * t.NP * pstride + y * n3 + z0, xrow, pstride};
        NatStage<N, +1, kWarps, 0>::template run<false>(stw, xc, sb, slot, sub, warp, act);
        __syncthreads();
        if constexpr (nst >= 3) {
            NatStage<N, +1, kWarps, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        if constexpr (nst >= 4) {
            NatStage<N, +1, kWarps, 2>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        if (act) {
            // one unit at a time (keeps the registers of one unit's values
            // next to the accumulators)
#pragma unroll
            for (int u = 0; u < L::U; ++u) {
                const int i = 2 * (warp + u * kWarps) + sub;
                if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
                    P2f h[R];
                    L::compute_unit(h, stw, sb, i, slot);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        acc[u][r].x += wx * h[r].a.x * h[r].a.x + wy * h[r].a.y * h[r].a.y;
                        acc[u][r].y += wx * h[r].b.x * h[r].b.x + wy * h[r].b.y * h[r].b.y;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (act) {
        // even offset (n3 even, z0 and 2 slot even): 8-byte aligned pairs
        float* part = partial + (long long)grp * N * pstride + y * n3 + z0 + 2 * slot;
#pragma unroll
        for (int u = 0; u < L::U; ++u) {
            const int i = 2 * (warp + u * kWarps) + sub;
            if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
#pragma unroll
                for (int r = 0; r < R; ++r) *reinterpret_cast<float2*>(part + (i + r * L::NI) * pstride) = acc[u][r];
            }
        }
    }
}

// Density x-pass for the quarter-sphere plane set: k3d_ct with the first
// inverse stage reading only the cuboid's rows (xq_first_inverse), and its
// last stage balanced as in k3q_ct (units left over after the full rounds of
// line-pair units run as single-line tasks spread over every thread).
#ifndef VLOC_MINB_K3DQ
#define VLOC_MINB_K3DQ 6
#endif
template <int N>
__global__ void __launch_bounds__(kThreads, N <= 96 ? VLOC_MINB_K3DQ : 1) k3dq_ct(DevTables t, const float2* __restrict__ tw1,
                                                   const float2* slab, int nb, int bpg, const float* __restrict__ occ,
                                                   long long b_base, int pair, long long nreal,
                                                   float* __restrict__ partial) {
    using SC = Sched<N>;
    static_assert(SC::nst == 2, "quarter-sphere x-pass: two-stage lengths");
    constexpr int W = kWarps;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = t.n2, n3 = t.n3;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + N * kLdP;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * kLines;
    const int grp = blockIdx.z;
    const int lines = min(kLines, n3 - z0);
    const bool act = 2 * slot < lines;
    load_tw<float>(stw, tw1, N);
    __syncthreads();
    const int pstride = n2 * n3;
    using L = NatStage<N, +1, W, 1>;
    constexpr int R = SC::R(1), NB = L::NI;
    constexpr int FR = NB / (2 * W), LU = NB % (2 * W);
    constexpr int LT = (LU * 32 + 32 * W - 1) / (32 * W);  // line tasks per thread
    float2 acc[FR > 0 ? FR : 1][R];
    float accl[LT > 0 ? LT : 1][R];
#pragma unroll
    for (int u = 0; u < FR; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[u][r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < LT; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) accl[k][r] = 0.f;
    SmemP sb{buf};
    const int b1 = min(nb, (grp + 1) * bpg);
    for (int b = grp * bpg; b < b1; ++b) {
        double wxd, wyd;
        density_weights(occ, b_base + b, pair, nreal, wxd, wyd);
        const float wx = (float)wxd, wy = (float)wyd;
        const float2* sl = slab + (long long)b * t.NP * pstride + y * n3 + z0 + 2 * slot;
        if (act)
            xq_first_inverse<N, W, P2f>([&](int p) { return *reinterpret_cast<const P2f*>(sl + p * pstride); }, sb,
                                        slot, sub, warp);
        __syncthreads();
        if (act) {
#pragma unroll
            for (int u = 0; u < FR; ++u) {
                const int i = 2 * (warp + u * W) + sub;
                P2f h[R];
                L::compute_unit(h, stw, sb, i, slot);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[u][r].x += wx * h[r].a.x * h[r].a.x + wy * h[r].a.y * h[r].a.y;
                    acc[u][r].y += wx * h[r].b.x * h[r].b.x + wy * h[r].b.y * h[r].b.y;
                }
            }
        }
        if constexpr (LU > 0) {
#pragma unroll
            for (int k = 0; k < LT; ++k) {
                const int tk = threadIdx.x + k * 32 * W;  // line task: unit, slot, line
                const int i = FR * 2 * W + tk / 32, ls = (tk >> 1) & 15, ln = tk & 1;
                if (tk < LU * 32 && 2 * ls < lines) {
                    float2 h[R];
                    NatStage<N, +1, W, 1, float2>::compute_unit(h, stw, SmemT<float2>{buf + ln}, i, ls);
#pragma unroll
                    for (int r = 0; r < R; ++r) accl[k][r] += wx * h[r].x * h[r].x + wy * h[r].y * h[r].y;
                }
            }
        }
        __syncthreads();
    }
    float* part0 = partial + (long long)grp * N * pstride + y * n3 + z0;  // the group sums in FP32, as in k3d_ct
    if (act) {
#pragma unroll
        for (int u = 0; u < FR; ++u) {
            const int i = 2 * (warp + u * W) + sub;
#pragma unroll
            for (int r = 0; r < R; ++r) *reinterpret_cast<float2*>(part0 + 2 * slot + (i + r * NB) * pstride) = acc[u][r];
        }
    }
    if constexpr (LU > 0) {
#pragma unroll
        for (int k = 0; k < LT; ++k) {
            const int tk = threadIdx.x + k * 32 * W;
            const int i = FR * 2 * W + tk / 32, ls = (tk >> 1) & 15, ln = tk & 1;
            if (tk < LU * 32 && 2 * ls < lines) {
#pragma unroll
                for (int r = 0; r < R; ++r) part0[2 * ls + ln + (i + r * NB) * pstride] = accl[k][r];
            }
        }
    }
}

// ------------------------------------------------------------ launchers
template <int N> struct CtSmem {
    static constexpr size_t sm = ct_smem<N>();
    template <class K> static cudaError_t ensure(K kernel) {
        if (sm <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
};

// K1 over nb bands (GM: nb Gamma-point pairs formed from the caller's real
// bands as they are read)
template <int N, bool GM>
int launch_k1_ct(const DevTables& t, const void* tw3, const void* coeffs, long long nb, void* cyl, const GammaArgs& g,
                 cudaStream_t st) {
    if constexpr (zs_length<N>()) {
        if (!GM && t.zs) {  // VLOC_Z_WARP plans
            k1s_ct<N><<<dim3(zs_blocks(t.S), (unsigned)nb), kZsThreads, 0, st>>>(t, (const float2*)tw3,
                                                                                (const float2*)coeffs, (float2*)cyl);
            return (int)cudaGetLastError();
        }
    }
    if constexpr (Sched<N>::nst == 2) {
        if (!GM && VLOC_K1_BULK && t.runs == 1 && t.zd_rows == QRows<N>::groups() * QRows<N>::NA) {
            constexpr size_t sm = k1b_smem<N>();
            static const cudaError_t onceb =
                sm <= 48 * 1024 ? cudaSuccess : cudaFuncSetAttribute(k1b_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (onceb) return (int)onceb;
            k1b_ct<N><<<dim3(t.T, (unsigned)nb), kThreads, sm, st>>>(t, (const float2*)tw3, (const float2*)coeffs,
                                                                    (float2*)cyl);
            return (int)cudaGetLastError();
        }
        // the dense table exists for plain plans only (its entries are caller
        // indices of the complex band the kernel reads)
        if (!GM && VLOC_K1_DIRECT && t.zd_rows == QRows<N>::groups() * QRows<N>::NA) {
            if (t.runs == 2) {
                static const cudaError_t oncer = CtSmem<N>::ensure(k1d_ct<N, true>);
                if (oncer) return (int)oncer;
                k1d_ct<N, true><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw3,
                                                                                      (const float2*)coeffs, (float2*)cyl);
                return (int)cudaGetLastError();
            }
            static const cudaError_t onced = CtSmem<N>::ensure(k1d_ct<N, false>);
            if (onced) return (int)onced;
            k1d_ct<N, false><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw3,
                                                                                       (const float2*)coeffs, (float2*)cyl);
            return (int)cudaGetLastError();
        }
        if (t.zq) {
            static const cudaError_t onceq = CtSmem<N>::ensure(k1q_ct<N, GM>);
            if (onceq) return (int)onceq;
            k1q_ct<N, GM><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw3,
                                                                                    (const float2*)coeffs,
                                                                                    (float2*)cyl, g);
            return (int)cudaGetLastError();
        }
    }
    static const cudaError_t once = CtSmem<N>::ensure(k1_ct<N, GM>);
    if (once) return (int)once;
    k1_ct<N, GM><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw3,
                                                                           (const float2*)coeffs, (float2*)cyl, g);
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k1(const DevTables& t, const void* tw3, const void* coeffs, long long nb, void* cyl,
                       cudaStream_t st) {
    static_assert(std::is_same<T, float>::value, "compile-time kernels are FP32");
    return launch_k1_ct<N, false>(t, tw3, coeffs, nb, cyl, GammaArgs{}, st);
}
template <typename T, int N>
int LaunchCT<T, N>::k1g(const DevTables& t, const void* tw3, const void* coeffs, long long npairs, long long nreal,
                        void* cyl, cudaStream_t st) {
    return launch_k1_ct<N, true>(t, tw3, coeffs, npairs, cyl, GammaArgs{t.npw_half, nreal, nullptr, nullptr}, st);
}
template <typename T, int N>
int LaunchCT<T, N>::k2(int sign, const DevTables& t, const void* tw2, long long nb, void* cyl, void* slab,
                       cudaStream_t st) {
    const dim3 grid(t.NP, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    if (sign > 0) {
        static const cudaError_t once = CtSmem<N>::ensure(k2_ct<+1, N>);
        if (once) return (int)once;
        k2_ct<+1, N><<<grid, kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw2, (float2*)cyl, (float2*)slab);
    } else {
        static const cudaError_t once = CtSmem<N>::ensure(k2_ct<-1, N>);
        if (once) return (int)once;
        k2_ct<-1, N><<<grid, kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw2, (float2*)cyl, (float2*)slab);
    }
    return (int)cudaGetLastError();
}
// defined in k3_tma.cuh (included by the instantiating files)
template <int N> int launch_k3_tma(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab,
                                   const K3Tma& tma, cudaStream_t st);
template <typename T, int N>
int LaunchCT<T, N>::k3(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab, const K3Tma* tma,
                       cudaStream_t st) {
    if (tma) return launch_k3_tma<N>(t, tw1, V, nb, slab, *tma, st);
    constexpr int W = k3_warps(N);
    if constexpr (Sched<N>::nst == 2) {
        if (t.xq) {
            constexpr size_t sm = k3q_smem<N>();
            // (a preferred shared-memory carveout, 86 % or 100 %, measured
            // slower at every length than the driver's own choice)
            static_assert(sm <= 48 * 1024, "x-pass tile within the default shared-memory limit");
            if (t.n3 % kLines == 0) {
                const dim3 grid(t.n2, t.n3 / kLines, (unsigned)nb);
                k3q_ct<N, W, false><<<grid, 32 * W, sm, st>>>(t, (const float2*)tw1, (const float*)V, (float2*)slab);
            } else {
                const dim3 grid((unsigned)((t.n2 * (t.n3 / 2) + 15) / 16), 1, (unsigned)nb);  // 16 line pairs a tile
                k3q_ct<N, W, true><<<grid, 32 * W, sm, st>>>(t, (const float2*)tw1, (const float*)V, (float2*)slab);
            }
            return (int)cudaGetLastError();
        }
    }
    static const cudaError_t once = CtSmem<N>::ensure(k3_ct<N, W>);
    if (once) return (int)once;
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    k3_ct<N, W><<<grid, 32 * W, CtSmem<N>::sm, st>>>(t, (const float2*)tw1, (const float*)V,
                                                                           (float2*)slab);
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k3b(const DevTables& t, const void* tw1, const void* sc, const void* sg, long long nb, int bpg,
                        double* partial, cudaStream_t st) {
    constexpr size_t sm = 2 * (size_t)N * kLdP * sizeof(float2) + (size_t)N * sizeof(float2) + (size_t)N * sizeof(int) + 16;
    static const cudaError_t once =
        sm <= 48 * 1024 ? cudaSuccess : cudaFuncSetAttribute(k3b_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (once) return (int)once;
    const int ng = (int)((nb + bpg - 1) / bpg);
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, ng);
    const double invN = 1.0 / ((double)t.n1 * t.n2 * t.n3);
    if constexpr (Sched<N>::nst == 2) {
        if (t.xq) {
            static const cudaError_t onceq =
                sm <= 48 * 1024 ? cudaSuccess
                                : cudaFuncSetAttribute(k3bq_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (onceq) return (int)onceq;
            k3bq_ct<N><<<grid, kThreads, sm, st>>>(t, (const float2*)tw1, (const float2*)sc, (const float2*)sg, (int)nb,
                                                  bpg, partial, invN);
            return (int)cudaGetLastError();
        }
    }
    k3b_ct<N><<<grid, kThreads, sm, st>>>(t, (const float2*)tw1, (const float2*)sc, (const float2*)sg, (int)nb, bpg,
                                          partial, invN);
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k3g(int sign, const DevTables& t, const void* tw1, long long nb, void* slab, void* grid,
                        cudaStream_t st) {
    const dim3 g3(t.n2, (t.n3 + kLines - 1) / kLines, (unsigned)nb);
    if (sign > 0) {
        static const cudaError_t once = CtSmem<N>::ensure(k3g_ct<+1, N>);
        if (once) return (int)once;
        k3g_ct<+1, N><<<g3, kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw1, (float2*)slab, (float2*)grid);
    } else {
        static const cudaError_t once = CtSmem<N>::ensure(k3g_ct<-1, N>);
        if (once) return (int)once;
        k3g_ct<-1, N><<<g3, kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw1, (float2*)slab, (float2*)grid);
    }
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k3d(const DevTables& t, const void* tw1, const void* slab, long long nb, int bpg, const void* occ,
                        long long b_base, int pair, long long nreal, float* partial, cudaStream_t st) {
    const int ng = (int)((nb + bpg - 1) / bpg);
    const dim3 grid(t.n2, (t.n3 + kLines - 1) / kLines, ng);
    if constexpr (Sched<N>::nst == 2) {
        if (t.xq) {
            static const cudaError_t onceq = CtSmem<N>::ensure(k3dq_ct<N>);
            if (onceq) return (int)onceq;
            k3dq_ct<N><<<grid, kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw1, (const float2*)slab, (int)nb, bpg,
                                                              (const float*)occ, b_base, pair, nreal, partial);
            return (int)cudaGetLastError();
        }
    }
    static const cudaError_t once = CtSmem<N>::ensure(k3d_ct<N>);
    if (once) return (int)once;
    k3d_ct<N><<<grid, kThreads, CtSmem<N>::sm, st>>>(t, (const float2*)tw1, (const float2*)slab, (int)nb, bpg,
                                                     (const float*)occ, b_base, pair, nreal, partial);
    return (int)cudaGetLastError();
}
template <int N, bool GM>
int launch_k4_ct(const DevTables& t, const void* tw3, const void* cyl, long long nb, void* out, const void* diag,
                 const void* cin, const GammaArgs& g, cudaStream_t st) {
    const float scale = (float)(1.0 / ((double)t.n1 * t.n2 * t.n3));
    if constexpr (zs_length<N>()) {
        if (!GM && t.zs) {  // VLOC_Z_WARP plans
            k4s_ct<N><<<dim3(zs_blocks(t.S), (unsigned)nb), kZsThreads, 0, st>>>(
                t, (const float2*)tw3, (const float2*)cyl, (float2*)out, scale, (const float*)diag, (const float2*)cin);
            return (int)cudaGetLastError();
        }
    }
    if constexpr (Sched<N>::nst == 2) {
        if (!GM && VLOC_K4_DIRECT && t.zd_rows == QRows<N>::groups() * QRows<N>::NA) {
            static const cudaError_t onced = CtSmem<N>::ensure(k4d_ct<N>);
            if (onced) return (int)onced;
            k4d_ct<N><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(
                t, (const float2*)tw3, (const float2*)cyl, (float2*)out, scale, (const float*)diag, (const float2*)cin);
            return (int)cudaGetLastError();
        }
        if (t.zq) {
            static const cudaError_t onceq = CtSmem<N>::ensure(k4q_ct<N, GM>);
            if (onceq) return (int)onceq;
            k4q_ct<N, GM><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(
                t, (const float2*)tw3, (const float2*)cyl, (float2*)out, scale, (const float*)diag, (const float2*)cin,
                g);
            return (int)cudaGetLastError();
        }
    }
    static const cudaError_t once = CtSmem<N>::ensure(k4_ct<N, GM>);
    if (once) return (int)once;
    k4_ct<N, GM><<<dim3(t.T, (unsigned)nb), kThreads, CtSmem<N>::sm, st>>>(
        t, (const float2*)tw3, (const float2*)cyl, (float2*)out, scale, (const float*)diag, (const float2*)cin, g);
    return (int)cudaGetLastError();
}
template <typename T, int N>
int LaunchCT<T, N>::k4(const DevTables& t, const void* tw3, const void* cyl, long long nb, void* out,
                       const void* diag, const void* cin, cudaStream_t st) {
    return launch_k4_ct<N, false>(t, tw3, cyl, nb, out, diag, cin, GammaArgs{}, st);
}
template <typename T, int N>
int LaunchCT<T, N>::k4g(const DevTables& t, const void* tw3, const void* cyl, long long npairs, long long nreal,
                        void* out, const void* diag, const void* cin, cudaStream_t st) {
    return launch_k4_ct<N, true>(t, tw3, cyl, npairs, out, nullptr, nullptr,
                                 GammaArgs{t.npw_half, nreal, (const float*)diag, (const float2*)cin}, st);
}

}  // namespace vloc
