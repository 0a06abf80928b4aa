// k3_tma.cuh -- persistent x-pass kernel (FP32, compile-time length) whose
// slab tiles move by TMA tensor copies between global and shared memory,
// double-buffered with mbarriers (the VLOC_X_TMA plan option).
//
// Same arithmetic as k3_ct (inverse x-FFT, x V(r), forward x-FFT with the
// chained middle stage), bit for bit.  A CTA loops over (y, 32-z tile, band)
// tiles with a grid stride; while it transforms one tile, one TMA tensor load
// brings the next tile (NP occupied-plane rows of 32 z) into the other
// landing buffer, and one TMA tensor store writes the finished tile back.
// Measured on GB300 at 96^3: 2.27 ms per 1024 bands against 1.82 ms for
// k3_ct (128 registers and two landing buffers leave 4 CTAs per SM against
// 5, and the transforms, not the loads, bound the kernel), so it is opt-in.
//
// Every wait is bounded: a copy that has not landed within about a second
// (clock64) sets the plan's error flag, the CTA waits (bounded) for its own
// copies in flight and returns.
#pragma once

#include <algorithm>

#include "kernels_ct.cuh"

namespace vloc {

constexpr int kLandRow = kLines;  // landing rows: 32 z (float2), 256 bytes

// rows of a landing buffer [NP][32] (dense; row = plane), read through the
// x -> plane map like XRowsP
struct LandRowsP {
    float2* land;
    const int* xrow;
    __device__ __forceinline__ P2f operator()(int e, int slot) const {
        const int p = xrow[e];
        return p >= 0 ? *reinterpret_cast<const P2f*>(land + p * kLandRow + 2 * slot) : czero<P2f>();
    }
    __device__ __forceinline__ void operator()(int e, int slot, P2f v) const {
        const int p = xrow[e];
        if (p >= 0) *reinterpret_cast<P2f*>(land + p * kLandRow + 2 * slot) = v;
    }
};

inline size_t k3_tma_smem(int N, int NP) {
    return 128 + 2 * (size_t)NP * kLandRow * 8 + (size_t)N * kLdP * 8 + (size_t)N * 8 + (size_t)N * 4;
}

__device__ __forceinline__ void tma_load_tile(float2* dst, const CUtensorMap* map, int c0, int c1, int c3,
                                              unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(0), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_tile(const CUtensorMap* map, int c0, int c1, int c3, const float2* src) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(c0), "r"(c1), "r"(0), "r"(c3), "r"(smem_u32(src))
                 : "memory");
}

// Persistent x-pass: tiles (y, 32-z tile, band) with a grid stride; one TMA
// load brings a tile's NP plane rows into a landing buffer while the
// previous tile is transformed, one TMA store writes the result back.
template <int N>
__global__ void __launch_bounds__(kThreads, 4) k3_tma(DevTables t, const float2* __restrict__ tw1,
                                                     const float* __restrict__ Vr, const __grid_constant__ CUtensorMap map,
                                                     int band0, int nb, int* err, int skip_first) {
    using SC = Sched<N>;
    constexpr int nst = SC::nst;
    static_assert(nst >= 2, "compile-time x-pass needs at least two stages");
    extern __shared__ __align__(128) unsigned char smem_bulk[];
    const int n2 = t.n2, n3 = t.n3, NP = t.NP;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_bulk);  // [2]
    float2* land0 = reinterpret_cast<float2*>(smem_bulk + 128);                   // [2][NP][32]
    float2* buf = land0 + 2 * NP * kLandRow;                                      // [N][kLdP]
    float2* stw = buf + N * kLdP;
    int* xrow = reinterpret_cast<int*>(stw + N);
    const int tid = threadIdx.x;
    const int slot = slot_of(), sub = sub_of(), warp = warp_of();
    const int ztiles = (n3 + kLines - 1) / kLines;
    const int ntiles = n2 * ztiles * nb;
    const int pstride = n2 * n3;
    const unsigned tile_bytes = (unsigned)NP * kLandRow * 8u;  // the whole box, zero-filled past n3

    for (int e = tid; e < N; e += kThreads) {
        stw[e] = tw1[e];
        xrow[e] = t.xrow_plane[e];
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // tile T = (b * ztiles + zt) * n2 + y
    unsigned pending = 0;  // thread 0: bit s set while buffer s has a load in flight
    auto issue_load = [&](int T, int s) {  // thread 0
        const int y = T % n2, r = T / n2;
        pending |= 1u << s;
        mbar_expect_tx(&bars[s], tile_bytes);
        tma_load_tile(land0 + s * NP * kLandRow, &map, 2 * (r % ztiles) * kLines, y, band0 + r / ztiles, &bars[s]);
    };
    // (skip_first: a test aid -- block 0's first tile is never requested, so
    // its bounded wait below runs out with no copy of that buffer in flight)
    if (tid == 0 && (int)blockIdx.x < ntiles && !(skip_first && blockIdx.x == 0)) issue_load(blockIdx.x, 0);
    SmemP sb{buf};
    int k = 0;
    for (int T = blockIdx.x; T < ntiles; T += gridDim.x, ++k) {
        const int s = k & 1;
        float2* land = land0 + s * NP * kLandRow;
        if (tid == 0) {
            bulk_wait_read0();  // the other buffer's store has read it
            if (T + (int)gridDim.x < ntiles) issue_load(T + gridDim.x, s ^ 1);
        }
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bars[s], (unsigned)(k >> 1) & 1u));
        if (!ok) {
            // record the failure, then wait (bounded) for every load of this
            // block still in flight and for its stores, and leave
            if (tid == 0) {
                atomicExch(err, 1);
                if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (unsigned)(k >> 1) & 1u);
                if (pending & (1u << (s ^ 1))) mbar_wait_bounded(&bars[s ^ 1], (unsigned)((k + 1) >> 1) & 1u);
                bulk_wait0();
            }
            __syncthreads();
            return;
        }
        if (tid == 0) pending &= ~(1u << s);
        const int y = T % n2, r = T / n2;
        const int zt = r % ztiles, b = r / ztiles;
        const int z0 = zt * kLines;
        const int lines = min(kLines, n3 - z0);
        const bool act = 2 * slot < lines;
        const float* vrow = Vr + (long long)y * n3 + z0 + 2 * slot;
        LandRowsP lr{land, xrow};

        NatStage<N, +1, kWarps, 0>::template run<false>(stw, lr, sb, slot, sub, warp, act);
        __syncthreads();
        if constexpr (nst >= 3) {
            NatStage<N, +1, kWarps, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        if constexpr (nst >= 4) {
            NatStage<N, +1, kWarps, 2>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        using L = NatStage<N, +1, kWarps, nst - 1>;
        using F = RevStage<N, -1, kWarps, 0>;
        constexpr int R = SC::R(nst - 1);
        static_assert(F::NI == L::NI && SC::RR(0) == R, "chained stages must share units");
        P2f h[L::U][R];
        if (act) {
            L::compute(h, stw, sb, slot, sub, warp);
#pragma unroll
            for (int u = 0; u < L::U; ++u) {
                const int i = 2 * (warp + u * kWarps) + sub;
                if (L::NI % (2 * kWarps) == 0 || i < L::NI) {
#pragma unroll
                    for (int rr = 0; rr < R; ++rr) {
                        const float2 w = *reinterpret_cast<const float2*>(vrow + (i + rr * L::NI) * pstride);
                        h[u][rr].a = cscale(h[u][rr].a, w.x);
                        h[u][rr].b = cscale(h[u][rr].b, w.y);
                    }
                    Dft<R, -1>::run(h[u]);
                }
            }
        }
        __syncthreads();
        if (act) F::store(h, sb, slot, sub, warp);
        __syncthreads();
        if constexpr (nst >= 3) {
            RevStage<N, -1, kWarps, 1>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        if constexpr (nst >= 4) {
            RevStage<N, -1, kWarps, 2>::template run<true>(stw, sb, sb, slot, sub, warp, act);
            __syncthreads();
        }
        RevStage<N, -1, kWarps, nst - 1>::template run<false>(stw, sb, lr, slot, sub, warp, act);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_tile(&map, 2 * z0, y, band0 + b, land);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait0();
}

template <int N>
int launch_k3_tma(const DevTables& t, const void* tw1, const void* V, long long nb, void* slab, const K3Tma& tma,
                  cudaStream_t st) {
    static const cudaError_t once =
        cudaFuncSetAttribute(k3_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k3_tma_smem(N, N));
    if (once) return (int)once;
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    const size_t sm = k3_tma_smem(N, t.NP);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_tma<N>, kThreads, sm);
    if (e) return (int)e;
    const long long ntiles = (long long)t.n2 * ((t.n3 + kLines - 1) / kLines) * nb;
    const long long grid = std::min<long long>(ntiles, (long long)nsm * std::max(per_sm, 1));
    const int band0 = (int)(((const char*)slab - (const char*)tma.base) / (long long)tma.band_bytes);
    k3_tma<N><<<(unsigned)grid, kThreads, sm, st>>>(t, (const float2*)tw1, (const float*)V, tma.map, band0, (int)nb,
                                                    tma.err, tma.skip_first);
    return (int)cudaGetLastError();
}

}  // namespace vloc
