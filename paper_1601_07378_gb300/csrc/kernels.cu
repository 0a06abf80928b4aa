// kernels.cu -- precision dispatch of the V_loc kernel launchers.  The
// kernels are in kernels_impl.cuh, compiled once per precision in
// kernels_f32.cu and kernels_f64.cu (two translation units built in
// parallel).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"
#include "fft_core.cuh"

namespace vloc {

__global__ void k_zero_f64(double* p, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.0;
}

// ---- Gamma-point real mode: two real bands per complex band
template <typename V>
__global__ void k_gamma_pack(const V* __restrict__ c, long long nb, long long nh, const int* __restrict__ neg,
                             long long nfull, V* __restrict__ C) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long p = blockIdx.y;
    if (q >= nh) return;
    const V a = c[(2 * p) * nh + q];
    V b;
    b.x = 0; b.y = 0;
    if (2 * p + 1 < nb) b = c[(2 * p + 1) * nh + q];
    V* row = C + p * nfull;
    const int n = neg[q];
    V u, w;
    if (n == q) {  // G = 0 is its own partner: the real parts
        u.x = a.x; u.y = b.x;
        row[q] = u;
        return;
    }
    u.x = a.x - b.y; u.y = a.y + b.x;   // a + i b at G
    w.x = a.x + b.y; w.y = b.x - a.y;   // conj(a) + i conj(b) at -G
    row[q] = u;
    row[n] = w;
}
template <typename V, typename T>
__global__ void k_gamma_unpack(const V* __restrict__ U, long long nfull, const int* __restrict__ neg, long long nh,
                               V* out, long long nb, const T* __restrict__ diag, const V* c) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long p = blockIdx.y;
    if (q >= nh) return;
    const V* row = U + p * nfull;
    const V x = row[q], y = row[neg[q]];  // U(G) and U(-G)
    V a, b;
    a.x = (x.x + y.x) * 0.5f; a.y = (x.y - y.y) * 0.5f;   // (U(G) + conj U(-G)) / 2
    b.x = (x.y + y.y) * 0.5f; b.y = (y.x - x.x) * 0.5f;   // (U(G) - conj U(-G)) / 2i
    const bool has_b = 2 * p + 1 < nb;
    if (diag) {  // H = diag + A; c is read before out is written (they may alias)
        const T d = diag[q];
        const V ca = c[(2 * p) * nh + q];
        a.x += d * ca.x; a.y += d * ca.y;
        if (has_b) {
            const V cb = c[(2 * p + 1) * nh + q];
            b.x += d * cb.x; b.y += d * cb.y;
        }
    }
    out[(2 * p) * nh + q] = a;
    if (has_b) out[(2 * p + 1) * nh + q] = b;
}
int launch_gamma_pack(int dbl, const void* c, long long nb, long long nh, const int* neg, long long nfull, void* C,
                      long long np, cudaStream_t st) {
    const dim3 grid((unsigned)((nh + 255) / 256), (unsigned)np);
    if (dbl) k_gamma_pack<double2><<<grid, 256, 0, st>>>((const double2*)c, nb, nh, neg, nfull, (double2*)C);
    else k_gamma_pack<float2><<<grid, 256, 0, st>>>((const float2*)c, nb, nh, neg, nfull, (float2*)C);
    return (int)cudaGetLastError();
}
int launch_gamma_unpack(int dbl, const void* U, long long np, long long nfull, const int* neg, long long nh,
                        void* out, long long nb, const void* diag, const void* c, cudaStream_t st) {
    const dim3 grid((unsigned)((nh + 255) / 256), (unsigned)np);
    if (dbl)
        k_gamma_unpack<double2, double><<<grid, 256, 0, st>>>((const double2*)U, nfull, neg, nh, (double2*)out, nb,
                                                              (const double*)diag, (const double2*)c);
    else
        k_gamma_unpack<float2, float><<<grid, 256, 0, st>>>((const float2*)U, nfull, neg, nh, (float2*)out, nb,
                                                            (const float*)diag, (const float2*)c);
    return (int)cudaGetLastError();
}

int launch_zero_f64(double* p, long long n, cudaStream_t st) {
    k_zero_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n);
    return (int)cudaGetLastError();
}

size_t smem_bytes_for(int dbl, int n) { return dbl ? Launch<double>::smem(n) : Launch<float>::smem(n); }
size_t grad_smem_bytes(int dbl, int n) { return dbl ? Launch<double>::smem_grad(n) : Launch<float>::smem_grad(n); }
// The dynamic shared-memory limit is a per-kernel attribute of the current
// device's context, shared by every plan on that device, so it only ever
// grows; the largest length set so far is kept per device.
int set_smem_limits(int dbl, int nmax, int optin) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static int cur[kMaxDevices][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < kMaxDevices && nmax <= cur[dev][dbl]) return 0;
    const int rc = dbl ? Launch<double>::set_limits(nmax, optin) : Launch<float>::set_limits(nmax, optin);
    if (rc == 0 && dev >= 0 && dev < kMaxDevices) cur[dev][dbl] = nmax;
    return rc;
}
int launch_twiddles(int dbl, void* tw, int n, cudaStream_t st) {
    return dbl ? Launch<double>::twiddles(tw, n, st) : Launch<float>::twiddles(tw, n, st);
}
bool has_ct(int n);
bool has_df(int n) { return has_ct(n); }

__global__ void k_twiddles_df(const double2* __restrict__ tw, TwDF* __restrict__ out, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = twdf_make(tw[j].x, tw[j].y);
}
int launch_twiddles_df(const void* tw64, void* twdf, int n, cudaStream_t st) {
    k_twiddles_df<<<(n + 127) / 128, 128, 0, st>>>((const double2*)tw64, (TwDF*)twdf, n);
    return (int)cudaGetLastError();
}
__global__ void k_v_to_df(const double* __restrict__ V, float2* __restrict__ out, long long N) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < N) out[i] = df_split(V[i]);
}
int launch_v_to_df(const void* V, void* Vdf, long long N, cudaStream_t st) {
    k_v_to_df<<<(unsigned)((N + 255) / 256), 256, 0, st>>>((const double*)V, (float2*)Vdf, N);
    return (int)cudaGetLastError();
}

bool has_ct(int n) {
    switch (n) {
#define VLOC_CASE(N) case N:
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        return true;
        default: return false;
    }
}

int launch_k1_scatter_zpass(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw3,
                            const void* coeffs, long long nb, void* cyl, cudaStream_t st) {
    if (dbl && fast == 2) switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchF64<0, N>::k1(t, tw3, coeffs, nb, cyl, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: return (int)cudaErrorInvalidValue;
    }
    if (dbl && fast == 1) switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchF64<1, N>::k1(t, tw3, coeffs, nb, cyl, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    if (!dbl && fast) switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k1(t, tw3, coeffs, nb, cyl, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k1(t, ax, tw3, coeffs, nb, cyl, st) : Launch<float>::k1(t, ax, tw3, coeffs, nb, cyl, st);
}
int launch_k1_gamma(const DevTables& t, const void* tw3, const void* c, long long npairs, long long nreal, void* cyl,
                    cudaStream_t st) {
    switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k1g(t, tw3, c, npairs, nreal, cyl, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: return (int)cudaErrorInvalidValue;
    }
}
int launch_k4_gamma(const DevTables& t, const void* tw3, const void* cyl, long long npairs, long long nreal, void* out,
                    const void* diag, const void* cin, cudaStream_t st) {
    switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k4g(t, tw3, cyl, npairs, nreal, out, diag, cin, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: return (int)cudaErrorInvalidValue;
    }
}
int launch_k2_ypass(int dbl, int fast, int sign, const DevTables& t, const LaunchAxes& ax, const void* tw2,
                    long long nb, void* cyl, void* slab, cudaStream_t st) {
    if (dbl && fast == 2) switch (t.n2) {
#define VLOC_CASE(N) case N: return LaunchF64<0, N>::k2(sign, t, tw2, nb, cyl, slab, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: return (int)cudaErrorInvalidValue;
    }
    if (dbl && fast == 1) switch (t.n2) {
#define VLOC_CASE(N) case N: return LaunchF64<1, N>::k2(sign, t, tw2, nb, cyl, slab, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    // the compile-time y- and x-passes move line pairs along z as 16-byte
    // vectors, which needs an even n3 (every pair then starts on an even
    // element); odd n3 takes the runtime-radix kernels
    if (!dbl && fast && (t.n3 & 1) == 0) switch (t.n2) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k2(sign, t, tw2, nb, cyl, slab, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k2(sign, t, ax, tw2, nb, cyl, slab, st)
               : Launch<float>::k2(sign, t, ax, tw2, nb, cyl, slab, st);
}
int launch_k3_xpass_v(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* V,
                      long long nb, void* slab, cudaStream_t st, const K3Tma* tma) {
    if (dbl && fast == 2) switch (t.n1) {  // V: hi + lo pairs
#define VLOC_CASE(N) case N: return LaunchF64<0, N>::k3(t, tw1, V, nb, slab, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: return (int)cudaErrorInvalidValue;
    }
    if (dbl && fast == 1) switch (t.n1) {
#define VLOC_CASE(N) case N: return LaunchF64<1, N>::k3(t, tw1, V, nb, slab, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    // the compile-time x-pass reads V two lines at a time (8-byte loads)
    if (!dbl && fast && (t.n3 & 1) == 0 && ((uintptr_t)V & 7) == 0) switch (t.n1) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k3(t, tw1, V, nb, slab, tma, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k3(t, ax, tw1, V, nb, slab, st) : Launch<float>::k3(t, ax, tw1, V, nb, slab, st);
}
int launch_k4_zpass_gather(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw3,
                           const void* cyl, long long nb, void* out, const void* diag, const void* cin,
                           cudaStream_t st) {
    if (dbl && fast == 2) switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchF64<0, N>::k4(t, tw3, cyl, nb, out, diag, cin, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: return (int)cudaErrorInvalidValue;
    }
    if (dbl && fast == 1) switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchF64<1, N>::k4(t, tw3, cyl, nb, out, diag, cin, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    if (!dbl && fast) switch (t.n3) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k4(t, tw3, cyl, nb, out, diag, cin, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k4(t, ax, tw3, cyl, nb, out, diag, cin, st)
               : Launch<float>::k4(t, ax, tw3, cyl, nb, out, diag, cin, st);
}
int launch_k3b_grad_v(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab_c,
                      const void* slab_g, long long nb, int bpg, double* partial, int* used, cudaStream_t st) {
    const int ng = (int)((nb + bpg - 1) / bpg);
    *used = ng;
    if (!dbl && fast && (t.n3 & 1) == 0) switch (t.n1) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k3b(t, tw1, slab_c, slab_g, nb, bpg, partial, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k3b(t, ax, tw1, slab_c, slab_g, nb, ng, partial, st)
               : Launch<float>::k3b(t, ax, tw1, slab_c, slab_g, nb, ng, partial, st);
}

int launch_k3_grid(int dbl, int fast, int sign, const DevTables& t, const LaunchAxes& ax, const void* tw1,
                   long long nb, void* slab, void* grid, cudaStream_t st) {
    // the compile-time x-pass moves z line pairs as 16-byte vectors
    if (!dbl && fast && (t.n3 & 1) == 0 && ((uintptr_t)grid & 15) == 0) switch (t.n1) {
#define VLOC_CASE(N) case N: return LaunchCT<float, N>::k3g(sign, t, tw1, nb, slab, grid, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k3g(sign, t, ax, tw1, nb, slab, grid, st)
               : Launch<float>::k3g(sign, t, ax, tw1, nb, slab, grid, st);
}
int launch_k3d_density(int dbl, int fast, const DevTables& t, const LaunchAxes& ax, const void* tw1, const void* slab,
                       long long nb, int bpg, const void* occ, long long b_base, int pair, long long nreal,
                       double* partial, int* used, cudaStream_t st) {
    *used = (int)((nb + bpg - 1) / bpg);
    if (density_partials_f32(dbl, fast, t)) switch (t.n1) {
#define VLOC_CASE(N) \
    case N: return LaunchCT<float, N>::k3d(t, tw1, slab, nb, bpg, occ, b_base, pair, nreal, (float*)partial, st);
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        default: break;
    }
    return dbl ? Launch<double>::k3d(t, ax, tw1, slab, nb, bpg, occ, b_base, pair, nreal, partial, st)
               : Launch<float>::k3d(t, ax, tw1, slab, nb, bpg, occ, b_base, pair, nreal, partial, st);
}
int density_partials_f32(int dbl, int fast, const DevTables& t) {
    if (dbl || !fast || (t.n3 & 1)) return 0;
    switch (t.n1) {
#define VLOC_CASE(N) case N:
        VLOC_CT_SIZES(VLOC_CASE)
#undef VLOC_CASE
        return 1;
        default: return 0;
    }
}
size_t density_smem_bytes(int dbl, int n) { return dbl ? Launch<double>::smem_dens(n) : Launch<float>::smem_dens(n); }

__global__ void k_reduce_partials(const double* __restrict__ partial, int ng, long long N, double* __restrict__ acc) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = acc[i];
    for (int g = 0; g < ng; ++g) s += partial[(long long)g * N + i];
    acc[i] = s;
}
int launch_reduce_partials(const double* partial, int ngroups, long long N, double* acc, cudaStream_t st) {
    k_reduce_partials<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(partial, ngroups, N, acc);
    return (int)cudaGetLastError();
}
// FP32 partials, added in group order by compensated summation in FP32: an
// error-free two-sum (Knuth) per group, the rounding errors gathered in a
// second word c (Ogita, Rump and Oishi's Sum2).  s + c is then as accurate as
// a sum in twice FP32's precision: its error is at most ((ng - 1) u)^2 times
// the sum of |partial|, u = 2^-24 (1.4e-11 for 64 groups), far below the
// FP32 result's own rounding.  The groups so cost FP32 adds rather than FP64
// conversions and adds (a slow pipe on this part); s + c then joins the FP64
// accumulator.
__global__ void k_reduce_partials_f32(const float* __restrict__ partial, int ng, long long N, double* __restrict__ acc,
                                      int first, float* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float s = 0.f, c = 0.f;
#pragma unroll 8
    for (int g = 0; g < ng; ++g) {
        const float p = partial[(long long)g * N + i];
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);  // the part of p that t took
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
        s = t;
    }
    const double tot = (first ? 0.0 : acc[i]) + ((double)s + (double)c);
    if (out) out[i] = (float)tot;
    else acc[i] = tot;
}
int launch_reduce_partials_f32(const float* partial, int ngroups, long long N, double* acc, int first, float* out,
                               cudaStream_t st) {
    k_reduce_partials_f32<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(partial, ngroups, N, acc, first, out);
    return (int)cudaGetLastError();
}

int launch_finish_grad_v(int dbl, const double* acc, void* gradV, long long N, cudaStream_t st) {
    return dbl ? Launch<double>::finish_grad(acc, gradV, N, st) : Launch<float>::finish_grad(acc, gradV, N, st);
}

}  // namespace vloc
