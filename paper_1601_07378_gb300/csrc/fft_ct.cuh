// fft_ct.cuh -- compile-time-sized Stockham stages (the fast path).
//
// Same algorithm as fft_core.cuh's runtime stages, but the transform length
// N, each stage's radix R and stride Ns are template constants, so the index
// arithmetic folds into immediates and every unit's registers are known at
// compile time.  FP32 only.  Three further differences:
//  * each lane carries two adjacent lines as one 16-byte vector (P2f), so a
//    shared or global access moves two elements and the address and
//    predicate work per element halves, while tiles stay 32 lines wide;
//  * one shared-memory buffer per tile: a stage that reads and writes the
//    buffer first computes all of its warp's units into registers, waits at a
//    barrier, then stores (halves the footprint, doubling resident CTAs);
//  * `ct_stage<...>::compute` / `store` are separate so a kernel can chain
//    the last inverse stage, a pointwise product and the first forward stage
//    of the reverse schedule in registers (the forward's first radix equals
//    the inverse's last, so a unit holds exactly the same elements).
#pragma once

#include "fft_core.cuh"

namespace vloc {

struct Radices {
    int nst;
    int r[kMaxStages];
};

// Compile-time copy of the host planner: fewest stages, then the smallest
// largest radix, then larger radices first (radix set of fft_core.cuh).
constexpr int kRadixSet[11] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
constexpr bool radices_better(const int* a, const int* b, int k) {
    int ma = 0, mb = 0;
    for (int i = 0; i < k; ++i) { ma = a[i] > ma ? a[i] : ma; mb = b[i] > mb ? b[i] : mb; }
    if (ma != mb) return ma < mb;
    for (int i = 0; i < k; ++i)
        if (a[i] != b[i]) return a[i] > b[i];
    return false;
}
constexpr Radices plan_ct(int n) {
    Radices best{0, {0, 0, 0, 0}};
    for (int i = 0; i < 11; ++i)
        if (kRadixSet[i] == n) { best.nst = 1; best.r[0] = n; return best; }
    for (int k = 2; k <= 4; ++k) {
        int idx[4] = {0, 0, 0, 0};
        bool found = false;
        while (true) {
            long long prod = 1;
            int c[4] = {0, 0, 0, 0};
            for (int i = 0; i < k; ++i) { c[i] = kRadixSet[idx[i]]; prod *= c[i]; }
            if (prod == n && (!found || radices_better(c, best.r, k))) {
                found = true;
                best.nst = k;
                for (int i = 0; i < 4; ++i) best.r[i] = i < k ? c[i] : 0;
            }
            int i = k - 1;
            while (i >= 0 && ++idx[i] == 11) { idx[i] = 0; --i; }
            if (i < 0) break;
        }
        if (found) return best;
    }
    return best;
}

template <int N> struct Sched {
    static constexpr Radices P = plan_ct(N);
    static constexpr int nst = P.nst;
    static_assert(P.nst > 0, "length must be 2/3/5-smooth and <= 4 stages");
    // radix and stride of stage s of the inverse (natural) schedule
    static constexpr int R(int s) { return P.r[s]; }
    static constexpr int NS(int s) { int p = 1; for (int i = 0; i < s; ++i) p *= P.r[i]; return p; }
    // reversed schedule (used for the forward transform chained after the inverse)
    static constexpr int RR(int s) { return P.r[P.nst - 1 - s]; }
    static constexpr int NSR(int s) { int p = 1; for (int i = 0; i < s; ++i) p *= P.r[P.nst - 1 - i]; return p; }
};

// ---- x rows of the quarter-sphere plane set
// When the occupied x-planes are exactly x = 0..Q and N - Q .. N - 1 (Q =
// N / 4: a cut-off sphere of radius N/4 grid units, the cuboid of Fig. 5)
// every row the x-pass touches is known at compile time.  Row r of unit i
// of the first inverse stage (and of the last forward stage) is x = i + r NA
// (NA = N / R0); its kind says whether it is always outside the cuboid
// (a known-zero input, an output that is never stored), always inside it,
// or on its edge (inside for some units i only), and where its plane sits.
template <int N> struct QRows {
    static constexpr int Q = N / 4;
    static constexpr int NP = 2 * Q + 1;
    static constexpr int R0 = Sched<N>::R(0);
    static constexpr int NA = N / R0;
    static_assert(NA - 1 < N - 2 * Q, "a row cannot touch both edges");
    // 0: outside for every unit; 1: low rows, always inside; 2: high rows,
    // always inside; 3: low edge (inside iff i <= Q - r NA); 4: high edge
    // (inside iff i >= N - Q - r NA)
    static constexpr int kind(int r) {
        const int lo = r * NA, hi = r * NA + NA - 1;
        return hi <= Q ? 1 : lo >= N - Q ? 2 : lo <= Q ? 3 : hi >= N - Q ? 4 : 0;
    }
    // plane of row r for unit i: i + off(r)
    static constexpr int off(int r) { return (kind(r) == 1 || kind(r) == 3) ? r * NA : r * NA - N + NP; }
    static constexpr unsigned mask() {
        unsigned m = 0;
        for (int r = 0; r < R0; ++r) m |= (kind(r) ? 1u : 0u) << r;
        return m;
    }
    // index of row group r among the groups that meet the cuboid
    static constexpr int group(int r) {
        int j = 0;
        for (int q = 0; q < r; ++q) j += kind(q) ? 1 : 0;
        return j;
    }
    static constexpr int groups() { return group(R0); }
    template <int r> __device__ __forceinline__ static bool inside(int i) {
        constexpr int k = kind(r);
        if constexpr (k == 1 || k == 2) return true;
        else if constexpr (k == 3) return i <= Q - r * NA;
        else if constexpr (k == 4) return i >= N - Q - r * NA;
        else return false;
    }
};
// First stage of an inverse x-transform (radix R0, no twiddles) read from
// the quarter-sphere rows: `load(p)` returns the value of plane p for this
// lane's line(s); rows outside the cuboid are known zeros; results go to
// rows i R0 + r of `dst`.  W warps share the NA units.
template <int N, int W, class V, class Load, class Dst>
__device__ __forceinline__ void xq_first_inverse(const Load& load, const Dst& dst, int slot, int sub, int warp) {
    using QR = QRows<N>;
    constexpr int R0 = QR::R0, NA = QR::NA, UA = (NA + 2 * W - 1) / (2 * W);
#pragma unroll
    for (int u = 0; u < UA; ++u) {
        const int i = 2 * (warp + u * W) + sub;
        if (NA % (2 * W) == 0 || i < NA) {
            V h[R0];
            sfor<R0>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                if constexpr (QR::kind(r) == 0) h[r] = czero<V>();
                else h[r] = QR::template inside<r>(i) ? load(i + QR::off(r)) : czero<V>();
            });
            DftZ<R0, +1, QR::mask()>::run(h);
#pragma unroll
            for (int r = 0; r < R0; ++r) dst(i * R0 + r, slot, h[r]);
        }
    }
}

// Rows x of a length-N line that the first inverse stage of the natural
// schedule may read when every nonzero input lies in the quarter band (row
// x is read by unit x % NA as row x / NA)
template <int N> __device__ __forceinline__ bool xq_row_read(int x) {
    return (QRows<N>::mask() >> (x / QRows<N>::NA)) & 1u;
}

// Shared line buffer for lane pairs: [N][kLdP] FP32 complex, pitch even so a
// pair of adjacent lines is one aligned 16-byte vector.
constexpr int kLdP = kLines + 2;
template <class V> struct SmemT {  // [N][kLdP] float2 slots; V is 16 bytes per slot
    float2* p;
    __device__ __forceinline__ V operator()(int e, int slot) const {
        return *reinterpret_cast<const V*>(p + e * kLdP + 2 * slot);
    }
    __device__ __forceinline__ void operator()(int e, int slot, V v) const {
        *reinterpret_cast<V*>(p + e * kLdP + 2 * slot) = v;
    }
};
using SmemP = SmemT<P2f>;

// One compile-time Stockham stage over a tile of 16 slots.  Each lane carries
// one 16-byte value V per element of its slot (slot = lane % 16): a pair of
// FP32 lines (P2f, 32-line tiles) or one double-float line (DFc, 16-line
// tiles); a warp works on two units at once (sub = lane / 16) and the CTA's
// W warps share the units.  TW is the twiddle type of V.
template <int N, int R, int NS, int S, int W, class V = P2f, class TW = float2> struct CtStage {
    static constexpr int NI = N / R;
    static constexpr int U = (NI + 2 * W - 1) / (2 * W);
    static constexpr int TWS = N / (NS * R);

    // unit i (caller checks i < NI): load, twiddle, R-point DFT
    template <class Src>
    __device__ __forceinline__ static void compute_unit(V (&h)[R], const TW* __restrict__ tw, const Src& src, int i,
                                                       int slot) {
#pragma unroll
        for (int r = 0; r < R; ++r) h[r] = src(i + r * NI, slot);
        if constexpr (NS > 1) {
            const int base = (i % NS) * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const TW w = tw[r * base];
                h[r] = S > 0 ? cmul(h[r], w) : cmulc(h[r], w);
            }
        }
        Dft<R, S>::run(h);
    }

    template <class Src>
    __device__ __forceinline__ static void compute(V (&h)[U][R], const TW* __restrict__ tw, const Src& src, int slot,
                                                  int sub, int warp) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NI % (2 * W) == 0 || i < NI) compute_unit(h[u], tw, src, i, slot);
        }
    }

    template <class Dst>
    __device__ __forceinline__ static void store(const V (&h)[U][R], const Dst& dst, int slot, int sub, int warp) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = 2 * (warp + u * W) + sub;
            if (NI % (2 * W) == 0 || i < NI) {
                const int k = i % NS;
                const int j = (i - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) dst(j + r * NS, slot, h[u][r]);
            }
        }
    }

    // compute + store; HOLD puts a CTA barrier between them (the stage reads
    // and writes the same shared buffer).
    template <bool HOLD, class Src, class Dst>
    __device__ __forceinline__ static void run(const TW* __restrict__ tw, const Src& src, const Dst& dst, int slot,
                                              int sub, int warp, bool act) {
        V h[U][R];
        if (act) compute(h, tw, src, slot, sub, warp);
        if constexpr (HOLD) __syncthreads();
        if (act) store(h, dst, slot, sub, warp);
    }
};

// Stage s of the natural (sign S) schedule of length N.
template <int N, int S, int W, int s, class V = P2f, class TW = float2>
using NatStage = CtStage<N, Sched<N>::R(s), Sched<N>::NS(s), S, W, V, TW>;
// Stage s of the reversed schedule.
template <int N, int S, int W, int s, class V = P2f, class TW = float2>
using RevStage = CtStage<N, Sched<N>::RR(s), Sched<N>::NSR(s), S, W, V, TW>;

// Full transform with one shared buffer `buf` ([N][kLdP] FP32 complex).
// `in` may be global or `buf` itself (IN_BUF), `out` may be global or `buf`
// (OUT_BUF).  The caller provides a barrier before the call if `buf` was in
// use; the call ends without a barrier.
template <int N, int S, int W, bool REV, bool IN_BUF, bool OUT_BUF, class V = P2f, class TW = float2, class In,
          class Out>
__device__ __forceinline__ void fft_ct(const TW* __restrict__ tw, const In& in, const Out& out, float2* buf, int slot,
                                       int sub, int warp, bool act) {
    constexpr int nst = Sched<N>::nst;
    SmemT<V> sb{buf};
    auto stage = [&](auto sc, const auto& src, const auto& dst, auto hold) {
        constexpr int s = decltype(sc)::value;
        using St = std::conditional_t<REV, RevStage<N, S, W, s, V, TW>, NatStage<N, S, W, s, V, TW>>;
        St::template run<decltype(hold)::value>(tw, src, dst, slot, sub, warp, act);
    };
    if constexpr (nst == 1) {
        stage(std::integral_constant<int, 0>{}, in, out, std::integral_constant<bool, IN_BUF && OUT_BUF>{});
    } else {
        stage(std::integral_constant<int, 0>{}, in, sb, std::integral_constant<bool, IN_BUF>{});
        __syncthreads();
        if constexpr (nst >= 3) {
            stage(std::integral_constant<int, 1>{}, sb, sb, std::true_type{});
            __syncthreads();
        }
        if constexpr (nst >= 4) {
            stage(std::integral_constant<int, 2>{}, sb, sb, std::true_type{});
            __syncthreads();
        }
        stage(std::integral_constant<int, nst - 1>{}, sb, out, std::integral_constant<bool, OUT_BUF>{});
    }
}

}  // namespace vloc
