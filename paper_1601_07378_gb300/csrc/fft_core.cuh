// fft_core.cuh -- batched, line-parallel mixed-radix 1-D FFT building blocks
// for the compact 3-D FFT of the V_loc action (Sec. 4.3, Fig. 5: three sets
// of 1-D FFTs, each run only on the lines that can hold nonzero data).
//
// Design (GB300 / sm_103a, CUDA cores -- the transforms are not a dense
// contraction, so there is no tensor-core form of them worth its accuracy):
//  * A CTA owns a tile of up to 32 independent lines; lane l of every warp
//    works on line l, so every shared-memory access is 32 consecutive
//    elements (bank-conflict free) and every global access of a line tile
//    whose lines are contiguous in memory is fully coalesced.
//  * A length-n transform is a Stockham autosort sequence of radix-R stages
//    (R in {2,3,4,5,6,8,9,10,12,15,16}, at most 4 stages for any 2/3/5-smooth
//    n <= 256).  A stage reads R elements spaced n/R apart, applies the
//    inter-stage twiddles, runs an R-point DFT fully in registers and writes R
//    elements spaced Ns apart (Ns = product of the earlier radices).  The
//    first stage may read straight from global memory and the last may write
//    straight to it, so a two-stage transform touches shared memory once.
//  * The small DFTs are unrolled at compile time; their internal twiddles are
//    compile-time constants (Taylor series below).  Inter-stage twiddles come
//    from a per-axis table exp(+2 pi i j / n), made once per plan in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace vloc {

// ------------------------------------------------------------------ complex
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using c2 = typename Cplx<T>::type;

template <typename V> struct ScalarOf { using type = decltype(V{}.x); };
template <typename V> using scalar_t = typename ScalarOf<V>::type;

template <typename V> __device__ __forceinline__ V cmk(scalar_t<V> re, scalar_t<V> im) {
    V r; r.x = re; r.y = im; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cneg(V a) { return cmk<V>(-a.x, -a.y); }
// a * b and a * conj(b) for a twiddle b of the scalar complex type
template <typename V, typename W> __device__ __forceinline__ V cmul(V a, W b) {
    return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V, typename W> __device__ __forceinline__ V cmulc(V a, W b) {
    return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, scalar_t<V> s) { return cmk<V>(a.x * s, a.y * s); }
// a + s * b, s real
template <typename V> __device__ __forceinline__ V cfma(V a, scalar_t<V> s, V b) {
    return cmk<V>(a.x + s * b.x, a.y + s * b.y);
}
// x * (c + i s), c and s real constants
template <typename V> __device__ __forceinline__ V cmul_cs(V x, scalar_t<V> c, scalar_t<V> s) {
    return cmk<V>(x.x * c - x.y * s, x.x * s + x.y * c);
}
// multiply by S*i (S = +1 or -1)
template <int S, typename V> __device__ __forceinline__ V mul_si(V a) {
    return S > 0 ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
}
template <typename V> __device__ __forceinline__ V czero() { return cmk<V>(0, 0); }

// FP32 complex values are one float2: their componentwise operations (add,
// subtract, scale by a real) map onto the paired FP32 instructions of
// sm_100+ (one instruction for both components).  Declared before the DFT
// templates so that unqualified calls with float2 arguments find them.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 cfma(float2 a, float s, float2 b) { return __ffma2_rn(make_float2(s, s), b, a); }

// Two FP32 complex values of adjacent lines carried by one lane (one 16-byte
// vector): every operation applies to both; twiddles are shared.
struct __align__(16) P2f {
    float2 a, b;
};
template <> struct ScalarOf<P2f> { using type = float; };
__device__ __forceinline__ P2f cadd(P2f x, P2f y) { return {cadd(x.a, y.a), cadd(x.b, y.b)}; }
__device__ __forceinline__ P2f csub(P2f x, P2f y) { return {csub(x.a, y.a), csub(x.b, y.b)}; }
__device__ __forceinline__ P2f cneg(P2f x) { return {cneg(x.a), cneg(x.b)}; }
__device__ __forceinline__ P2f cmul(P2f x, float2 w) { return {cmul(x.a, w), cmul(x.b, w)}; }
__device__ __forceinline__ P2f cmulc(P2f x, float2 w) { return {cmulc(x.a, w), cmulc(x.b, w)}; }
__device__ __forceinline__ P2f cscale(P2f x, float s) { return {cscale(x.a, s), cscale(x.b, s)}; }
__device__ __forceinline__ P2f cfma(P2f x, float s, P2f y) { return {cfma(x.a, s, y.a), cfma(x.b, s, y.b)}; }
__device__ __forceinline__ P2f cmul_cs(P2f x, float c, float s) { return {cmul_cs(x.a, c, s), cmul_cs(x.b, c, s)}; }
template <int S> __device__ __forceinline__ P2f mul_si(P2f x) { return {mul_si<S>(x.a), mul_si<S>(x.b)}; }
template <> __device__ __forceinline__ P2f czero<P2f>() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// ---------------------------------------------- double-float arithmetic
// A real value held as hi + lo, two FP32 (about 48 significant bits).  Sums
// use the two-sum of Knuth / Moller, products an FMA for the rounding error
// of hi * hi (Dekker's product with a fused multiply-add); errors stay within
// a few units of 2^-48 relative to the operands' magnitudes, the bound an
// FFT's norm-wise error analysis needs.
__device__ __forceinline__ float2 fneg2_(float2 a) { return make_float2(-a.x, -a.y); }
// hi + lo split of a double (hi = nearest FP32, lo = nearest FP32 of the rest)
__host__ __device__ __forceinline__ float2 df_split(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// Complex double-float value held as a pair of high parts and a pair of low
// parts, hi = (re.hi, im.hi), lo = (re.lo, im.lo): the real and imaginary
// double-float operations then run side by side as paired FP32 instructions
// (sm_100+).  16 bytes, the size of an FP64 complex.  Scalar constants of the
// DFTs arrive as doubles and are split at compile time.
struct __align__(16) DFc {
    float2 hi, lo;
};
template <> struct ScalarOf<DFc> { using type = double; };
// twiddle w = c + i s as broadcast pairs: (c.hi, c.hi), (c.lo, c.lo),
// (-s.hi, s.hi), (-s.lo, s.lo)
struct __align__(16) TwDF {
    float2 ch, cl, sh, sl;
};
__host__ __device__ __forceinline__ TwDF twdf_make(double c, double s) {
    const float2 cc = df_split(c), ss = df_split(s);
    return TwDF{make_float2(cc.x, cc.x), make_float2(cc.y, cc.y), make_float2(-ss.x, ss.x), make_float2(-ss.y, ss.y)};
}
__device__ __forceinline__ DFc df2_neg(DFc x) { return {fneg2_(x.hi), fneg2_(x.lo)}; }
// Paired double-float sum: the exact two-sum of the high parts, plus the
// low parts.  The pair is left unnormalised (no final fast two-sum): the
// next two-sum is exact whatever the size of the low part, and each low part
// stays within a few ulps of its high part, so errors stay a few units of
// 2^-48 relative to the operands (the norm-wise bound of an FFT).
__device__ __forceinline__ DFc cadd(DFc x, DFc y) {
    const float2 s = __fadd2_rn(x.hi, y.hi);
    const float2 bb = __fadd2_rn(s, fneg2_(x.hi));
    const float2 e = __fadd2_rn(__fadd2_rn(__fadd2_rn(x.hi, fneg2_(__fadd2_rn(s, fneg2_(bb)))),
                                           __fadd2_rn(y.hi, fneg2_(bb))),
                                __fadd2_rn(x.lo, y.lo));
    return {s, e};
}
__device__ __forceinline__ DFc csub(DFc x, DFc y) { return cadd(x, df2_neg(y)); }
// renormalise (fast two-sum; |lo| is a few ulps of hi at most): applied when a
// value is written to global memory, so low parts do not grow over passes
__device__ __forceinline__ DFc df2_norm(DFc x) {
    const float2 hi = __fadd2_rn(x.hi, x.lo);
    return {hi, __fadd2_rn(x.lo, fneg2_(__fadd2_rn(hi, fneg2_(x.hi))))};
}
__device__ __forceinline__ DFc cneg(DFc x) { return df2_neg(x); }
// componentwise double-float product of x with the pair (bh + bl): the exact
// product of the high parts (an FMA gives its rounding error) plus the cross
// terms; the result (p, e) has |e| of a few ulps of p, so it needs no
// renormalisation either
__device__ __forceinline__ DFc df2_mul(DFc x, float2 bh, float2 bl) {
    const float2 p = __fmul2_rn(x.hi, bh);
    float2 e = __ffma2_rn(x.hi, bh, fneg2_(p));
    e = __ffma2_rn(x.hi, bl, e);
    e = __ffma2_rn(x.lo, bh, e);
    return {p, e};
}
__device__ __forceinline__ DFc df2_swap(DFc x) {  // (re, im) -> (im, re)
    return {make_float2(x.hi.y, x.hi.x), make_float2(x.lo.y, x.lo.x)};
}
__device__ __forceinline__ DFc cmul(DFc x, TwDF w) {  // x * w = x c + (im, re) (-s, s)
    return cadd(df2_mul(x, w.ch, w.cl), df2_mul(df2_swap(x), w.sh, w.sl));
}
__device__ __forceinline__ DFc cmulc(DFc x, TwDF w) {  // x * conj(w) = x c - (im, re) (-s, s)
    return cadd(df2_mul(x, w.ch, w.cl), df2_neg(df2_mul(df2_swap(x), w.sh, w.sl)));
}
__device__ __forceinline__ DFc cscale(DFc x, double s) {
    const float2 d = df_split(s);
    return df2_mul(x, make_float2(d.x, d.x), make_float2(d.y, d.y));
}
__device__ __forceinline__ DFc cfma(DFc x, double s, DFc y) { return cadd(x, cscale(y, s)); }  // x + s y
__device__ __forceinline__ DFc cmul_cs(DFc x, double c, double s) { return cmul(x, twdf_make(c, s)); }
template <int S> __device__ __forceinline__ DFc mul_si(DFc x) {  // x * (S i): (re, im) -> (-S im, S re)
    const DFc w = df2_swap(x);
    return S > 0 ? DFc{make_float2(-w.hi.x, w.hi.y), make_float2(-w.lo.x, w.lo.y)}
                 : DFc{make_float2(w.hi.x, -w.hi.y), make_float2(w.lo.x, -w.lo.y)};
}
template <> __device__ __forceinline__ DFc czero<DFc>() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
// FP64 complex <-> DFc
__device__ __forceinline__ DFc df_from(double2 v) {
    const float2 a = df_split(v.x), b = df_split(v.y);
    return {make_float2(a.x, b.x), make_float2(a.y, b.y)};
}
__device__ __forceinline__ double2 df_to(DFc v) {
    return make_double2((double)v.hi.x + (double)v.lo.x, (double)v.hi.y + (double)v.lo.y);
}

// ------------------------------------------------- compile-time cos / sin
// exp(2 pi i m / R) from Taylor series on the first octant (|x| <= pi/4,
// truncation below 1e-21), with exact integer quadrant reduction.
namespace ct {
constexpr double kHalfPi = 1.57079632679489661923132169163975144;
constexpr double sin_oct(double x) {
    double x2 = x * x;
    double s = 1.0 - x2 / (18.0 * 19.0);
    s = 1.0 - x2 / (16.0 * 17.0) * s;
    s = 1.0 - x2 / (14.0 * 15.0) * s;
    s = 1.0 - x2 / (12.0 * 13.0) * s;
    s = 1.0 - x2 / (10.0 * 11.0) * s;
    s = 1.0 - x2 / (8.0 * 9.0) * s;
    s = 1.0 - x2 / (6.0 * 7.0) * s;
    s = 1.0 - x2 / (4.0 * 5.0) * s;
    s = 1.0 - x2 / (2.0 * 3.0) * s;
    return x * s;
}
constexpr double cos_oct(double x) {
    double x2 = x * x;
    double c = 1.0 - x2 / (19.0 * 20.0);
    c = 1.0 - x2 / (17.0 * 18.0) * c;
    c = 1.0 - x2 / (15.0 * 16.0) * c;
    c = 1.0 - x2 / (13.0 * 14.0) * c;
    c = 1.0 - x2 / (11.0 * 12.0) * c;
    c = 1.0 - x2 / (9.0 * 10.0) * c;
    c = 1.0 - x2 / (7.0 * 8.0) * c;
    c = 1.0 - x2 / (5.0 * 6.0) * c;
    c = 1.0 - x2 / (3.0 * 4.0) * c;
    return 1.0 - x2 / (1.0 * 2.0) * c;
}
// cos(2 pi m / R) and sin(2 pi m / R)
constexpr double cos_turn(int m, int R) {
    int t = ((m % R) + R) % R;
    int q = (4 * t) / R, r = 4 * t - q * R;  // angle = (q + r/R) * pi/2, 0 <= r < R
    double c0 = 2 * r <= R ? cos_oct(kHalfPi * r / R) : sin_oct(kHalfPi * (R - r) / R);
    double s0 = 2 * r <= R ? sin_oct(kHalfPi * r / R) : cos_oct(kHalfPi * (R - r) / R);
    return q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;
}
constexpr double sin_turn(int m, int R) {
    int t = ((m % R) + R) % R;
    int q = (4 * t) / R, r = 4 * t - q * R;
    double c0 = 2 * r <= R ? cos_oct(kHalfPi * r / R) : sin_oct(kHalfPi * (R - r) / R);
    double s0 = 2 * r <= R ? sin_oct(kHalfPi * r / R) : cos_oct(kHalfPi * (R - r) / R);
    return q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;
}
}  // namespace ct

// compile-time unrolled loop: f(std::integral_constant<int, i>) for i < N
template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F> __device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// x * exp(S 2 pi i M / R), M and R compile-time; trivial angles cost no multiply.
template <int R, int S, int M, typename V> __device__ __forceinline__ V tw_const(V x) {
    constexpr int m = ((M % R) + R) % R;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (2 * m == R) {
        return cneg(x);
    } else if constexpr (4 * m == R) {
        return mul_si<S>(x);
    } else if constexpr (4 * m == 3 * R) {
        return mul_si<-S>(x);
    } else {
        using T = scalar_t<V>;
        constexpr T c = (T)ct::cos_turn(m, R);
        constexpr T s = (T)(S * ct::sin_turn(m, R));
        return cmul_cs(x, c, s);
    }
}

// ------------------------------------------------------------ small DFTs
// X[k] = sum_n x[n] exp(S 2 pi i n k / R), in place on registers.
template <int R, int S> struct Dft;

template <int S> struct Dft<1, S> {
    template <typename V> __device__ __forceinline__ static void run(V*) {}
};
template <int S> struct Dft<2, S> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <int S> struct Dft<3, S> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        using T = scalar_t<V>;
        constexpr T h = (T)0.866025403784438646763723170752936183;  // sqrt(3)/2
        V t = cadd(v[1], v[2]);
        V d = csub(v[1], v[2]);
        V m = cfma(v[0], (T)-0.5, t);
        V r = mul_si<S>(cscale(d, h));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};
template <int S> struct Dft<4, S> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        V t2 = cadd(v[1], v[3]), t3 = mul_si<S>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};
template <int S> struct Dft<5, S> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        using T = scalar_t<V>;
        constexpr T c1 = (T)ct::cos_turn(1, 5), c2 = (T)ct::cos_turn(2, 5);
        constexpr T s1 = (T)ct::sin_turn(1, 5), s2 = (T)ct::sin_turn(2, 5);
        V a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        V a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        V x0 = v[0];
        V p1 = cfma(cfma(x0, c1, a1), c2, a2);
        V p2 = cfma(cfma(x0, c2, a1), c1, a2);
        V q1 = mul_si<S>(cfma(cscale(b1, s1), s2, b2));
        V q2 = mul_si<S>(cfma(cscale(b1, s2), -s1, b2));
        v[0] = cadd(cadd(x0, a1), a2);
        v[1] = cadd(p1, q1);
        v[4] = csub(p1, q1);
        v[2] = cadd(p2, q2);
        v[3] = csub(p2, q2);
    }
};
// composite R = A * B: n = B n1 + n2, k = k1 + A k2.
template <int A, int B, int S> struct DftAB {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        constexpr int R = A * B;
        V y[R];
        sfor<B>([&](auto n2) {
            V t[A];
            sfor<A>([&](auto n1) { t[n1] = v[B * n1 + n2]; });
            Dft<A, S>::run(t);
            sfor<A>([&](auto k1) { y[n2 * A + k1] = tw_const<R, S, n2 * k1>(t[k1]); });
        });
        sfor<A>([&](auto k1) {
            V t[B];
            sfor<B>([&](auto n2) { t[n2] = y[n2 * A + k1]; });
            Dft<B, S>::run(t);
            sfor<B>([&](auto k2) { v[k1 + A * k2] = t[k2]; });
        });
    }
};
template <int S> struct Dft<6, S> : DftAB<2, 3, S> {};
template <int S> struct Dft<8, S> : DftAB<4, 2, S> {};
template <int S> struct Dft<9, S> : DftAB<3, 3, S> {};
template <int S> struct Dft<10, S> : DftAB<2, 5, S> {};
template <int S> struct Dft<12, S> : DftAB<4, 3, S> {};
template <int S> struct Dft<15, S> : DftAB<3, 5, S> {};
template <int S> struct Dft<16, S> : DftAB<4, 4, S> {};

// ------------------------------------- small DFTs with known-zero inputs
// A pruned stage (Sec. 4.3, Fig. 5: only the cuboid's planes hold data)
// knows at compile time which inputs of a unit are zero.  ZV<Z, V> carries
// that knowledge in its type: Z = true means "known zero", and the helpers
// below skip every operation with a known-zero operand, so a DFT over such
// inputs costs only the adds and products its nonzero inputs need.  Outputs
// a caller never stores are left to dead-code elimination.
template <bool Z, class V> struct ZV {
    V v;
};
template <bool Z, class V> __device__ __forceinline__ V zget(const ZV<Z, V>& a) {
    if constexpr (Z) return czero<V>();
    else return a.v;
}
template <bool A, bool B, class V> __device__ __forceinline__ ZV<A && B, V> zadd(const ZV<A, V>& a, const ZV<B, V>& b) {
    if constexpr (A && B) return {};
    else if constexpr (A) return {b.v};
    else if constexpr (B) return {a.v};
    else return {cadd(a.v, b.v)};
}
template <bool A, bool B, class V> __device__ __forceinline__ ZV<A && B, V> zsub(const ZV<A, V>& a, const ZV<B, V>& b) {
    if constexpr (A && B) return {};
    else if constexpr (A) return {cneg(b.v)};
    else if constexpr (B) return {a.v};
    else return {csub(a.v, b.v)};
}
template <int S, bool A, class V> __device__ __forceinline__ ZV<A, V> zmul_si(const ZV<A, V>& a) {
    if constexpr (A) return {};
    else return {mul_si<S>(a.v)};
}
template <bool A, class V> __device__ __forceinline__ ZV<A, V> zscale(const ZV<A, V>& a, scalar_t<V> s) {
    if constexpr (A) return {};
    else return {cscale(a.v, s)};
}
// a + s b
template <bool A, bool B, class V>
__device__ __forceinline__ ZV<A && B, V> zfma(const ZV<A, V>& a, scalar_t<V> s, const ZV<B, V>& b) {
    if constexpr (B) return {a.v};
    else if constexpr (A) return {cscale(b.v, s)};
    else return {cfma(a.v, s, b.v)};
}

constexpr bool zbit(unsigned m, int i) { return ((m >> i) & 1u) == 0; }  // true: input i known zero

// X[k] = sum_n x[n] exp(S 2 pi i n k / R) where bit n of M is clear for the
// inputs known to be zero (their values are ignored).  M = all ones is the
// plain Dft.
template <int R, int S, unsigned M> struct DftZ {
    template <typename V> __device__ __forceinline__ static void run(V* v) { Dft<R, S>::run(v); }
};
template <int S, unsigned M> struct DftZ<2, S, M> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        const ZV<zbit(M, 0), V> a{v[0]};
        const ZV<zbit(M, 1), V> b{v[1]};
        v[0] = zget(zadd(a, b));
        v[1] = zget(zsub(a, b));
    }
};
template <int S, unsigned M> struct DftZ<3, S, M> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        using T = scalar_t<V>;
        constexpr T h = (T)0.866025403784438646763723170752936183;  // sqrt(3)/2
        const ZV<zbit(M, 0), V> x0{v[0]};
        const ZV<zbit(M, 1), V> x1{v[1]};
        const ZV<zbit(M, 2), V> x2{v[2]};
        const auto t = zadd(x1, x2);
        const auto d = zsub(x1, x2);
        const auto m = zfma(x0, (T)-0.5, t);
        const auto r = zmul_si<S>(zscale(d, h));
        v[0] = zget(zadd(x0, t));
        v[1] = zget(zadd(m, r));
        v[2] = zget(zsub(m, r));
    }
};
template <int S, unsigned M> struct DftZ<4, S, M> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        const ZV<zbit(M, 0), V> x0{v[0]};
        const ZV<zbit(M, 1), V> x1{v[1]};
        const ZV<zbit(M, 2), V> x2{v[2]};
        const ZV<zbit(M, 3), V> x3{v[3]};
        const auto t0 = zadd(x0, x2), t1 = zsub(x0, x2);
        const auto t2 = zadd(x1, x3), t3 = zmul_si<S>(zsub(x1, x3));
        v[0] = zget(zadd(t0, t2));
        v[2] = zget(zsub(t0, t2));
        v[1] = zget(zadd(t1, t3));
        v[3] = zget(zsub(t1, t3));
    }
};
template <int S, unsigned M> struct DftZ<5, S, M> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        using T = scalar_t<V>;
        constexpr T c1 = (T)ct::cos_turn(1, 5), c2 = (T)ct::cos_turn(2, 5);
        constexpr T s1 = (T)ct::sin_turn(1, 5), s2 = (T)ct::sin_turn(2, 5);
        const ZV<zbit(M, 0), V> x0{v[0]};
        const ZV<zbit(M, 1), V> x1{v[1]};
        const ZV<zbit(M, 2), V> x2{v[2]};
        const ZV<zbit(M, 3), V> x3{v[3]};
        const ZV<zbit(M, 4), V> x4{v[4]};
        const auto a1 = zadd(x1, x4), b1 = zsub(x1, x4);
        const auto a2 = zadd(x2, x3), b2 = zsub(x2, x3);
        const auto p1 = zfma(zfma(x0, c1, a1), c2, a2);
        const auto p2 = zfma(zfma(x0, c2, a1), c1, a2);
        const auto q1 = zmul_si<S>(zfma(zscale(b1, s1), s2, b2));
        const auto q2 = zmul_si<S>(zfma(zscale(b1, s2), -s1, b2));
        v[0] = zget(zadd(zadd(x0, a1), a2));
        v[1] = zget(zadd(p1, q1));
        v[4] = zget(zsub(p1, q1));
        v[2] = zget(zadd(p2, q2));
        v[3] = zget(zsub(p2, q2));
    }
};
// composite R = A * B as in DftAB: a first-pass group whose inputs are all
// known zero is skipped (its outputs stay zero), and the second pass knows
// which groups those were.
template <int A, int B, unsigned M> struct ZMaskAB {
    static constexpr unsigned group(int n2) {
        unsigned g = 0;
        for (int n1 = 0; n1 < A; ++n1) g |= ((M >> (B * n1 + n2)) & 1u) << n1;
        return g;
    }
    static constexpr unsigned second() {
        unsigned m = 0;
        for (int n2 = 0; n2 < B; ++n2) m |= (group(n2) ? 1u : 0u) << n2;
        return m;
    }
};
template <int A, int B, int S, unsigned M> struct DftABZ {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        constexpr int R = A * B;
        using MK = ZMaskAB<A, B, M>;
        V y[R];
        sfor<B>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            constexpr unsigned g = MK::group(n2);
            if constexpr (g != 0) {
                V t[A];
                sfor<A>([&](auto n1) { t[n1] = v[B * n1 + n2]; });
                DftZ<A, S, g>::run(t);
                sfor<A>([&](auto k1) { y[n2 * A + k1] = tw_const<R, S, n2 * k1>(t[k1]); });
            } else {
                sfor<A>([&](auto k1) { y[n2 * A + k1] = czero<V>(); });
            }
        });
        constexpr unsigned m2 = MK::second();
        sfor<A>([&](auto k1) {
            V t[B];
            sfor<B>([&](auto n2) { t[n2] = y[n2 * A + k1]; });
            DftZ<B, S, m2>::run(t);
            sfor<B>([&](auto k2) { v[k1 + A * k2] = t[k2]; });
        });
    }
};
template <int R> constexpr unsigned zfull() { return R >= 32 ? ~0u : (1u << R) - 1u; }
#define VLOC_DFTZ_AB(RR, AA, BB)                                                              \
    template <int S, unsigned M> struct DftZ<RR, S, M> {                                    \
        template <typename V> __device__ __forceinline__ static void run(V* v) {            \
            if constexpr ((M & zfull<RR>()) == zfull<RR>()) Dft<RR, S>::run(v);             \
            else DftABZ<AA, BB, S, M>::run(v);                                               \
        }                                                                                    \
    };
VLOC_DFTZ_AB(6, 2, 3)
VLOC_DFTZ_AB(8, 4, 2)
VLOC_DFTZ_AB(9, 3, 3)
VLOC_DFTZ_AB(10, 2, 5)
VLOC_DFTZ_AB(12, 4, 3)
VLOC_DFTZ_AB(15, 3, 5)
VLOC_DFTZ_AB(16, 4, 4)
#undef VLOC_DFTZ_AB

// ------------------------------------------------------------ per-axis plan
constexpr int kMaxStages = 4;
constexpr int kLines = 32;          // lines per tile (one per lane)
constexpr int kLd = kLines + 1;     // shared-memory row pitch (elements)
constexpr int kThreads = 128;       // threads per CTA
constexpr int kWarps = kThreads / 32;

struct AxisPlan {
    int n;
    int nst;
    int radix[kMaxStages];
};

// shared-memory line buffer [n][kLd]
template <typename V> struct Smem {
    V* p;
    __device__ __forceinline__ V operator()(int e, int l) const { return p[e * kLd + l]; }
    __device__ __forceinline__ void operator()(int e, int l, V v) const { p[e * kLd + l] = v; }
};

// One Stockham stage of radix R over `lines` lines held across lanes.
template <int R, int S, typename V, class Src, class Dst>
__device__ __forceinline__ void fft_stage(int n, int Ns, const V* __restrict__ tw, const Src& src,
                                         const Dst& dst, int lines) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nI = n / R;
    const int twstep = n / (Ns * R);
    if (lane >= lines) return;
    for (int i = warp; i < nI; i += kWarps) {
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src(i + r * nI, lane);
        const int k = i % Ns;
        if (Ns > 1) {
            const int base = k * twstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                V w = tw[r * base];
                v[r] = S > 0 ? cmul(v[r], w) : cmulc(v[r], w);
            }
        }
        Dft<R, S>::run(v);
        const int j = (i - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst(j + r * Ns, lane, v[r]);
    }
}

template <int S, typename V, class Src, class Dst>
__device__ __forceinline__ void stage_dispatch(int R, int n, int Ns, const V* tw, const Src& src, const Dst& dst,
                                               int lines) {
    switch (R) {
        case 2: fft_stage<2, S>(n, Ns, tw, src, dst, lines); break;
        case 3: fft_stage<3, S>(n, Ns, tw, src, dst, lines); break;
        case 4: fft_stage<4, S>(n, Ns, tw, src, dst, lines); break;
        case 5: fft_stage<5, S>(n, Ns, tw, src, dst, lines); break;
        case 6: fft_stage<6, S>(n, Ns, tw, src, dst, lines); break;
        case 8: fft_stage<8, S>(n, Ns, tw, src, dst, lines); break;
        case 9: fft_stage<9, S>(n, Ns, tw, src, dst, lines); break;
        case 10: fft_stage<10, S>(n, Ns, tw, src, dst, lines); break;
        case 12: fft_stage<12, S>(n, Ns, tw, src, dst, lines); break;
        case 15: fft_stage<15, S>(n, Ns, tw, src, dst, lines); break;
        case 16: fft_stage<16, S>(n, Ns, tw, src, dst, lines); break;
        default: break;  // the host planner only emits the radices above
    }
}

// Buffer that receives the transform when the output is a shared-memory
// buffer and stages ping-pong P -> Q -> P ...: stage 0 writes P.
template <typename V> __device__ __forceinline__ V* final_buf(int nst, V* P, V* Q) { return (nst & 1) ? P : Q; }

// Full length-n transform of `lines` lines: stage 0 reads `in` (global or
// shared, must not be P), intermediate results ping-pong between P and Q,
// the last stage writes `out`.  Ends without a barrier.
template <int S, typename V, class In, class Out>
__device__ __forceinline__ void fft_lines(const AxisPlan& ap, const V* tw, const In& in, const Out& out, V* P, V* Q,
                                          int lines) {
    if (ap.nst == 1) {
        stage_dispatch<S>(ap.radix[0], ap.n, 1, tw, in, out, lines);
        return;
    }
    stage_dispatch<S>(ap.radix[0], ap.n, 1, tw, in, Smem<V>{P}, lines);
    __syncthreads();
    int Ns = ap.radix[0];
    V* cur = P;
    V* oth = Q;
    for (int s = 1; s < ap.nst - 1; ++s) {
        stage_dispatch<S>(ap.radix[s], ap.n, Ns, tw, Smem<V>{cur}, Smem<V>{oth}, lines);
        __syncthreads();
        Ns *= ap.radix[s];
        V* t = cur; cur = oth; oth = t;
    }
    stage_dispatch<S>(ap.radix[ap.nst - 1], ap.n, Ns, tw, Smem<V>{cur}, out, lines);
}

}  // namespace vloc
