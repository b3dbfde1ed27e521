// ibf_device.cuh -- device building blocks of the projection kernels:
//   * complex arithmetic,
//   * float-float ("df32", an unevaluated sum hi + lo of two fp32 numbers) arithmetic
//     after Dekker (1971) and Knuth's TwoSum, with FMA-based exact products,
//   * fp64 <-> df32 / fp32 conversions done with integer bit operations only
//     (GB300 runs fp64 arithmetic and F2F conversions at ~1/72 of the fp32 rate),
//   * register DFTs of length 1..32 (mixed radix 2/3/4 Stockham autosort stages,
//     Govindaraju et al., SC 2008) and a two-level shared-memory FFT built on them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ibf_internal.h"

namespace ibf {

// ------------------------------------------------------------------ complex
template <typename T> struct cx { T x, y; };

template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
// fp32: one packed two-lane instruction (sm_100 family) per complex add or subtract,
// each lane rounded exactly as the scalar operation (a - b as fma(b, -1, a))
template <> __device__ __forceinline__ cx<float> cadd<float>(cx<float> a, cx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return {r.x, r.y};
}
template <> __device__ __forceinline__ cx<float> csub<float>(cx<float> a, cx<float> b) {
    const float2 r = __ffma2_rn(make_float2(b.x, b.y), make_float2(-1.f, -1.f), make_float2(a.x, a.y));
    return {r.x, r.y};
}
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {  // a * conj(b)
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.x * s, a.y * s}; }
template <typename T> __device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.x, -a.y}; }

// ------------------------------------------------------------------ float-float
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ df df_make(float a) { return {a, 0.f}; }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_addf(df a, float b) {
    df s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ float df_to_f(df a) { return __fadd_rn(a.hi, a.lo); }
// a + b + c of three floats as a normalised pair (error below 2^-47 of the largest term)
__device__ __forceinline__ df sum3(float a, float b, float c) {
    const df s = two_sum(a, b);
    const df t = two_sum(s.hi, c);
    return two_sum(t.hi, __fadd_rn(t.lo, s.lo));
}

// hi + lo + v for a possibly unnormalised pair (hi, lo) as a normalised pair: hi + v
// and its error, that error plus lo and its error, all without rounding, then the
// leading float renormalised against the collected remainder (error below 2^-47 of the
// sum, whatever the relative sizes of lo and v)
__device__ __forceinline__ df df_add3(float hi, float lo, float v) {
    const df s = two_sum(hi, v);
    const df t = two_sum(s.lo, lo);
    const df u = two_sum(s.hi, t.hi);
    return quick_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

// the same sum as an unnormalised pair: hi the rounded sum, lo its error (rounded once)
__device__ __forceinline__ df sum3u(float a, float b, float c) {
    const df s = two_sum(a, b);
    const df t = two_sum(s.hi, c);
    return {t.hi, __fadd_rn(t.lo, s.lo)};
}

// c1 d1 + c2 d2 + c3 d3 of float-float operands as a normalised pair: each product
// is its leading float and one FMA-collected error term (the lo x lo part, below
// 2^-46 of the product, is dropped), the three leading floats are added without
// error, and every error term is collected in one float that is added once at the
// end (the compensated dot product of Ogita, Rump and Oishi, SIAM J. Sci. Comput.
// 26 (2005), "Dot2", on float-float inputs).  Error below about 2^-45 of
// |c1 d1| + |c2 d2| + |c3 d3|, as for a chain of df_mul / df_add.
__device__ __forceinline__ df df_dot3(df c1, df d1, df c2, df d2, df c3, df d3) {
    const float p1 = __fmul_rn(c1.hi, d1.hi);
    float e1 = __fmaf_rn(c1.hi, d1.hi, -p1);
    e1 = __fmaf_rn(c1.hi, d1.lo, e1);
    e1 = __fmaf_rn(c1.lo, d1.hi, e1);
    const float p2 = __fmul_rn(c2.hi, d2.hi);
    float e2 = __fmaf_rn(c2.hi, d2.hi, -p2);
    e2 = __fmaf_rn(c2.hi, d2.lo, e2);
    e2 = __fmaf_rn(c2.lo, d2.hi, e2);
    const float p3 = __fmul_rn(c3.hi, d3.hi);
    float e3 = __fmaf_rn(c3.hi, d3.hi, -p3);
    e3 = __fmaf_rn(c3.hi, d3.lo, e3);
    e3 = __fmaf_rn(c3.lo, d3.hi, e3);
    const df s = two_sum(p1, p2);
    const df t = two_sum(s.hi, p3);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, s.lo)), t.lo);
    return two_sum(t.hi, lo);
}

// b - c0 - (c1 d1 + c2 d2 + c3 d3 - c4 d4) as a normalised pair: products as in
// df_dot3, the six leading floats added without error, one collected error term.
__device__ __forceinline__ df df_resid4(df b, df c0, df c1, df d1, df c2, df d2, df c3, df d3, df c4, df d4) {
    const float p1 = __fmul_rn(c1.hi, d1.hi);
    float e1 = __fmaf_rn(c1.hi, d1.hi, -p1);
    e1 = __fmaf_rn(c1.hi, d1.lo, e1);
    e1 = __fmaf_rn(c1.lo, d1.hi, e1);
    const float p2 = __fmul_rn(c2.hi, d2.hi);
    float e2 = __fmaf_rn(c2.hi, d2.hi, -p2);
    e2 = __fmaf_rn(c2.hi, d2.lo, e2);
    e2 = __fmaf_rn(c2.lo, d2.hi, e2);
    const float p3 = __fmul_rn(c3.hi, d3.hi);
    float e3 = __fmaf_rn(c3.hi, d3.hi, -p3);
    e3 = __fmaf_rn(c3.hi, d3.lo, e3);
    e3 = __fmaf_rn(c3.lo, d3.hi, e3);
    const float p4 = __fmul_rn(c4.hi, d4.hi);
    float e4 = __fmaf_rn(c4.hi, d4.hi, -p4);
    e4 = __fmaf_rn(c4.hi, d4.lo, e4);
    e4 = __fmaf_rn(c4.lo, d4.hi, e4);
    df s = two_sum(b.hi, -c0.hi);
    float lo = __fadd_rn(__fsub_rn(b.lo, c0.lo), s.lo);
    s = two_sum(s.hi, -p1);
    lo = __fadd_rn(lo, s.lo);
    s = two_sum(s.hi, -p2);
    lo = __fadd_rn(lo, s.lo);
    s = two_sum(s.hi, -p3);
    lo = __fadd_rn(lo, s.lo);
    s = two_sum(s.hi, p4);
    lo = __fadd_rn(lo, s.lo);
    lo = __fadd_rn(lo, __fsub_rn(__fsub_rn(e4, e1), __fadd_rn(e2, e3)));
    return two_sum(s.hi, lo);
}

// ------------------------------------------------------------------ float-float, two lanes
// The sequences above on two independent values at once, in the packed fp32x2
// instructions of the sm_100 family: every lane rounds exactly as the scalar operation
// (a - b as fma(b, -1, a)), so each lane of a result equals the scalar result bit for bit.
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
struct df2 { float2 hi, lo; };
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
    const float2 s = p2add(a, b), bb = p2sub(s, a);
    return {s, p2add(p2sub(a, p2sub(s, bb)), p2sub(b, bb))};
}
__device__ __forceinline__ df2 quick_two_sum2(float2 a, float2 b) {
    const float2 s = p2add(a, b);
    return {s, p2sub(b, p2sub(s, a))};
}
__device__ __forceinline__ df2 df_addf2(df2 a, float2 b) {
    const df2 s = two_sum2(a.hi, b);
    return quick_two_sum2(s.hi, p2add(s.lo, a.lo));
}
__device__ __forceinline__ df2 sum3u2(float2 a, float2 b, float2 c) {
    const df2 s = two_sum2(a, b);
    const df2 t = two_sum2(s.hi, c);
    return {t.hi, p2add(t.lo, s.lo)};
}
// the leading float of c d negated (-p) and the FMA-collected error of p, as in df_resid4
__device__ __forceinline__ void prod_neg(df c, float dh, float dl, float &pn, float &e) {
    pn = __fmul_rn(-c.hi, dh);
    e = __fmaf_rn(c.hi, dh, pn);
    e = __fmaf_rn(c.hi, dl, e);
    e = __fmaf_rn(c.lo, dh, e);
}
__device__ __forceinline__ void prod_pos(df c, float dh, float dl, float &p, float &e) {
    p = __fmul_rn(c.hi, dh);
    e = __fmaf_rn(c.hi, dh, -p);
    e = __fmaf_rn(c.hi, dl, e);
    e = __fmaf_rn(c.lo, dh, e);
}
__device__ __forceinline__ df2 df_add2(df2 a, df2 b) {
    const df2 s = two_sum2(a.hi, b.hi);
    return quick_two_sum2(s.hi, p2add(s.lo, p2add(a.lo, b.lo)));
}
// df_sub on two values: lane for lane the scalar df_sub (df_add of the negation).  The
// negation is folded into the subtractions: with round-to-nearest, x + (-y) and
// -(y + z) round exactly as x - y and the negated sum.
__device__ __forceinline__ df2 df_sub2(df2 a, df2 b) {
    const float2 s = p2sub(a.hi, b.hi), bb = p2sub(s, a.hi);
    const float2 e = p2sub(p2sub(a.hi, p2sub(s, bb)), p2add(b.hi, bb));
    return quick_two_sum2(s, p2add(e, p2sub(a.lo, b.lo)));
}
// a - b for float-float pairs that need not be normalised (phi = hi + lo during the
// refinement), to the pairs' precision: the leading words' difference exactly (a two-sum),
// the trailing words' difference rounded once to a float, and that float added to the
// exact pair by a second two-sum.  The one rounding that is not at the pair's precision
// is fl(a.lo - b.lo), which the refinement residual reproduces (k_xfwd, XM_RESID1), so that
// it cancels in the divergence of the corrected velocity.
__device__ __forceinline__ df df_sub_acc(df a, df b) {
    const df s = two_sum(a.hi, -b.hi);
    const df t = two_sum(s.hi, __fsub_rn(a.lo, b.lo));
    return quick_two_sum(t.hi, __fadd_rn(t.lo, s.lo));
}
__device__ __forceinline__ df2 df_sub2_acc(df2 a, df2 b) {  // lane for lane df_sub_acc
    const float2 s = p2sub(a.hi, b.hi), bb = p2sub(s, a.hi);
    const float2 e = p2sub(p2sub(a.hi, p2sub(s, bb)), p2add(b.hi, bb));
    const df2 t = two_sum2(s, p2sub(a.lo, b.lo));
    return quick_two_sum2(t.hi, p2add(t.lo, e));
}
// df_mul of one float-float c by two values: lane for lane the scalar df_mul(c, d) (the
// leading product formed negated, which rounds as its negation)
__device__ __forceinline__ df2 df_mul2(df c, df2 d) {
    const float2 ch = make_float2(c.hi, c.hi), cl = make_float2(c.lo, c.lo);
    const float2 pn = p2mul(make_float2(-c.hi, -c.hi), d.hi);
    float2 e = __ffma2_rn(ch, d.hi, pn);
    e = __ffma2_rn(ch, d.lo, e);
    e = __ffma2_rn(cl, d.hi, e);
    const float2 s = p2sub(e, pn);                 // p + e
    return {s, p2sub(e, p2add(s, pn))};            // e - (s - p)
}
// df_dot3 on two values: products per lane, every sum in two-lane operations
__device__ __forceinline__ df2 df_dot3_2(df c1, df2 d1, df c2, df2 d2, df c3, df2 d3) {
    float2 p1, p2, p3, e1, e2, e3;
    prod_pos(c1, d1.hi.x, d1.lo.x, p1.x, e1.x);
    prod_pos(c1, d1.hi.y, d1.lo.y, p1.y, e1.y);
    prod_pos(c2, d2.hi.x, d2.lo.x, p2.x, e2.x);
    prod_pos(c2, d2.hi.y, d2.lo.y, p2.y, e2.y);
    prod_pos(c3, d3.hi.x, d3.lo.x, p3.x, e3.x);
    prod_pos(c3, d3.hi.y, d3.lo.y, p3.y, e3.y);
    const df2 s = two_sum2(p1, p2);
    const df2 t = two_sum2(s.hi, p3);
    const float2 lo = p2add(p2add(p2add(e1, e2), p2add(e3, s.lo)), t.lo);
    return two_sum2(t.hi, lo);
}
// df_resid4 on two values: products per lane, every sum in two-lane operations
__device__ __forceinline__ df2 df_resid4_2(df2 b, df c0, df c1, df2 d1, df c2, df2 d2, df c3, df2 d3, df c4,
                                           df2 d4) {
    float2 n1, n2, n3, p4, e1, e2, e3, e4;
    prod_neg(c1, d1.hi.x, d1.lo.x, n1.x, e1.x);
    prod_neg(c1, d1.hi.y, d1.lo.y, n1.y, e1.y);
    prod_neg(c2, d2.hi.x, d2.lo.x, n2.x, e2.x);
    prod_neg(c2, d2.hi.y, d2.lo.y, n2.y, e2.y);
    prod_neg(c3, d3.hi.x, d3.lo.x, n3.x, e3.x);
    prod_neg(c3, d3.hi.y, d3.lo.y, n3.y, e3.y);
    prod_pos(c4, d4.hi.x, d4.lo.x, p4.x, e4.x);
    prod_pos(c4, d4.hi.y, d4.lo.y, p4.y, e4.y);
    df2 s = two_sum2(b.hi, make_float2(-c0.hi, -c0.hi));
    float2 lo = p2add(p2sub(b.lo, make_float2(c0.lo, c0.lo)), s.lo);
    s = two_sum2(s.hi, n1);
    lo = p2add(lo, s.lo);
    s = two_sum2(s.hi, n2);
    lo = p2add(lo, s.lo);
    s = two_sum2(s.hi, n3);
    lo = p2add(lo, s.lo);
    s = two_sum2(s.hi, p4);
    lo = p2add(lo, s.lo);
    lo = p2add(lo, p2sub(p2sub(e4, e1), p2add(e2, e3)));
    return two_sum2(s.hi, lo);
}

// fp64 -> df32 without fp64 arithmetic.  hi takes the sign, the exponent and the
// top 23 fraction bits (truncated); lo = x - hi is formed from the remaining 29
// bits (rounded to 24 by the integer->float conversion), so hi + lo == x within
// 2^-48 relative.  |x| < 2^-74 loses lo, |x| < 2^-126 flushes to 0, |x| >= 2^128
// maps to +-inf, NaN stays NaN.  The general routine; f64_to_df below takes a shorter
// path for the common exponents and calls this one (out of line) for the rest.
__device__ __forceinline__ df f64_to_df_general(double x) {
    const unsigned long long X = (unsigned long long)__double_as_longlong(x);
    const unsigned h = (unsigned)(X >> 32), l = (unsigned)X;
    const unsigned e = (h >> 20) & 0x7FFu;
    const unsigned s = h & 0x80000000u;
    unsigned hbits = __funnelshift_l(l, (h & 0x7FFFFFFFu) - (896u << 20), 3);
    float scale = __uint_as_float(s | ((e - 948u) << 23));
    float lo = __fmul_rn(__uint2float_rn(l & 0x1FFFFFFFu), scale);
    if (e < 949u) {
        lo = 0.f;
        if (e < 897u) hbits = 0u;
    }
    if (e > 1150u) {
        hbits = 0x7F800000u | (((e == 2047u) && ((h & 0xFFFFFu) | l)) ? 0x400000u : 0u);
        lo = 0.f;
    }
    return {__uint_as_float(s | hbits), lo};
}

// df32 -> fp64 without fp64 arithmetic.  For a normalised pair (|lo| <= ulp(hi),
// which every df_* operation returns; hi = 0 implies lo = 0) hi + lo is exactly an
// fp64 number in hi's binade, so it is hi's fp64 bit pattern plus lo's significand
// aligned to hi's fp64 ulp (a shift by el - eh + 29 <= 6, so 32-bit arithmetic
// suffices); the only binade change possible is a borrow below a power of two (hi's
// fraction zero, lo of opposite sign), where the ulp halves.  lo bits below 2^-52 of
// hi are truncated, a subnormal lo (|hi| below 2^-102) is dropped.  hi zero or
// subnormal gives a signed zero; hi inf / nan stays inf / nan.  The general routine;
// df_to_f64 below takes a shorter path for the common case.
__device__ __forceinline__ double df_to_f64_general(df a) {
    const unsigned hb = __float_as_uint(a.hi), lb = __float_as_uint(a.lo);
    const unsigned ha = hb & 0x7FFFFFFFu, sgn = hb & 0x80000000u;
    const bool special = ha >= 0x7F800000u;
    // hi as fp64: sign, exponent + 896 (all ones for inf / nan), fraction << 29
    const unsigned hw = sgn | ((ha >> 3) + 0x38000000u) | (special ? 0x7FF00000u : 0u);
    const unsigned lw = hb << 29;
    const unsigned el = (lb >> 23) & 0xFFu;
    const int sh = (int)el - (int)(ha >> 23) + 29;
    // L 2^sh with the bits below 2^0 truncated (shift amounts of 32 and more give 0)
    unsigned Li = __funnelshift_rc(((lb & 0x7FFFFFu) | 0x800000u) << 8, 0u, (unsigned)(8 - sh));
    if (el == 0u || special) Li = 0u;
    const bool neg = ((hb ^ lb) & 0x80000000u) != 0u;
    if (neg && (ha & 0x7FFFFFu) == 0u) Li <<= 1;
    unsigned long long H = ((unsigned long long)hw << 32) | lw;
    H = neg ? H - Li : H + Li;
    if (ha < 0x00800000u) H = (unsigned long long)sgn << 32;
    return __longlong_as_double((long long)H);
}

static __device__ __noinline__ df f64_to_df_slow(double x) { return f64_to_df_general(x); }
static __device__ __noinline__ double df_to_f64_slow(df a) { return df_to_f64_general(a); }

// fp64 -> df32, the same result as f64_to_df_general.  Exponents 949..1150 (|x| in
// [2^-74, 2^128)), where neither part is flushed nor overflows, take the short path:
// hi is x truncated to 24 bits, and the weight of the 29 remaining fraction bits' unit
// (x's fp64 ulp) is read off hi's exponent field, 52 binades below it.  Everything else
// goes to the general routine, out of line, so that the common path carries no
// special-case selects.
__device__ __forceinline__ df f64_to_df(double x) {
    const unsigned long long X = (unsigned long long)__double_as_longlong(x);
    const unsigned h = (unsigned)(X >> 32), l = (unsigned)X;
    const unsigned ha = h & 0x7FFFFFFFu;
    if (ha - (949u << 20) >= ((1151u - 949u) << 20)) return f64_to_df_slow(x);
    const unsigned hb = __funnelshift_l(l, ha - (896u << 20), 3) | (h & 0x80000000u);
    const float scale = __uint_as_float((hb & 0xFF800000u) - (52u << 23));
    return {__uint_as_float(hb), __fmul_rn(__uint2float_rn(l & 0x1FFFFFFFu), scale)};
}

// df32 -> fp64 for a normalised pair, the same value as df_to_f64_general.  Short path
// when hi is normal with exponent field 52..254 and a nonzero fraction (so that hi + lo
// stays in hi's binade): lo, times a power of two that carries hi's sign and makes hi's
// fp64 ulp the unit, is exactly a float below 2^29 in magnitude; its truncation toward
// zero is the number of fp64 ulps to add to hi's fp64 bit pattern (hi's own pattern has
// 29 zero low bits, so the sum never carries out of them or borrows past them).  Other
// pairs (zero, tiny, huge, special, or hi a power of two) take the general routine.
__device__ __forceinline__ double df_to_f64(df a) {
    const unsigned hb = __float_as_uint(a.hi);
    const unsigned ef = hb & 0x7F800000u;
    if (ef - (52u << 23) >= ((254u - 52u + 1u) << 23) || (hb & 0x7FFFFFu) == 0u) return df_to_f64_slow(a);
    const unsigned hw = ((unsigned)((int)hb >> 3) & 0x8FFFFFFFu) + 0x38000000u;
    const float sc = __uint_as_float(((306u << 23) - ef) | (hb & 0x80000000u));
    const long long li = (long long)__float2int_rz(__fmul_rn(a.lo, sc));
    const unsigned long long H = (((unsigned long long)hw << 32) | (unsigned long long)(hb << 29)) + (unsigned long long)li;
    return __longlong_as_double((long long)H);
}

// ------------------------------------------------------------------ precision policies
// FP64 path: everything in double.  MIXED path: transforms in float, stencils in df32.
struct F64Arith {
    typedef double V;      // high-precision value
    __device__ __forceinline__ static V load(double x) { return x; }
    __device__ __forceinline__ static double store(V v) { return v; }
    __device__ __forceinline__ static double store_once(V v) { return v; }
    __device__ __forceinline__ static V add(V a, V b) { return a + b; }
    __device__ __forceinline__ static V sub(V a, V b) { return a - b; }
    __device__ __forceinline__ static V sub_acc(V a, V b) { return a - b; }
    __device__ __forceinline__ static V mul(V a, V b) { return a * b; }
    __device__ __forceinline__ static V from_f(float a) { return (double)a; }
    __device__ __forceinline__ static V zero() { return 0.0; }
    __device__ __forceinline__ static V norm(V a) { return a; }
};
struct DFArith {
    typedef df V;
    __device__ __forceinline__ static V load(double x) { return f64_to_df(x); }
    __device__ __forceinline__ static double store(V v) { return df_to_f64(v); }
    // a value stored once per CTA (a block sum): the general conversion, in line
    __device__ __forceinline__ static double store_once(V v) { return df_to_f64_general(v); }
    __device__ __forceinline__ static V add(V a, V b) { return df_add(a, b); }
    __device__ __forceinline__ static V sub(V a, V b) { return df_sub(a, b); }
    // differences of a refined phi (unnormalised pairs): see df_sub_acc
    __device__ __forceinline__ static V sub_acc(V a, V b) { return df_sub_acc(a, b); }
    __device__ __forceinline__ static V mul(V a, V b) { return df_mul(a, b); }
    __device__ __forceinline__ static V from_f(float a) { return df_make(a); }
    __device__ __forceinline__ static V zero() { return df_make(0.f); }
    __device__ __forceinline__ static V norm(V a) { return quick_two_sum(a.hi, a.lo); }
};

// ------------------------------------------------------------------ twiddle constants
// exp(-2 pi i r / 96): every twiddle inside a register DFT of length dividing 96.
__constant__ double c_tw96d[96][2] = {
#include "tw96.inc"
};
__constant__ float c_tw96f[96][2] = {
#include "tw96.inc"
};

template <typename T> struct Tw96;
template <> struct Tw96<double> {
    __device__ __forceinline__ static cx<double> get(int r) { return {c_tw96d[r][0], c_tw96d[r][1]}; }
};
template <> struct Tw96<float> {
    __device__ __forceinline__ static cx<float> get(int r) { return {c_tw96f[r][0], c_tw96f[r][1]}; }
};

// ------------------------------------------------------------------ butterflies
// DIR = -1: forward (exp(-i ...)), DIR = +1: inverse (unnormalised).
template <typename T, int R, int DIR> struct Bfly;
template <typename T, int DIR> struct Bfly<T, 2, DIR> {
    __device__ __forceinline__ static void run(cx<T> *v) {
        cx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <typename T, int DIR> struct Bfly<T, 3, DIR> {
    __device__ __forceinline__ static void run(cx<T> *v) {
        const T c = (T)0.86602540378443864676;  // sin(2 pi / 3)
        cx<T> s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        cx<T> t = {v[0].x - (T)0.5 * s.x, v[0].y - (T)0.5 * s.y};
        v[0] = cadd(v[0], s);
        // v1 = t + DIR*i*c*d, v2 = t - DIR*i*c*d  with i*d = (-d.y, d.x)
        v[1] = {t.x - (T)DIR * c * d.y, t.y + (T)DIR * c * d.x};
        v[2] = {t.x + (T)DIR * c * d.y, t.y - (T)DIR * c * d.x};
    }
};
template <typename T, int DIR> struct Bfly<T, 4, DIR> {
    __device__ __forceinline__ static void run(cx<T> *v) {
        cx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        cx<T> t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
        cx<T> it3 = {(T)(-DIR) * t3.y, (T)DIR * t3.x};  // (DIR*i) * t3
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, it3);
        v[3] = csub(t1, it3);
    }
};

// In-place register DFT of the P elements x[s * STRIDE], s < P (P a divisor of 96
// built from radices 2, 3, 4): P = P1 * P2 with P1 the first radix, DFT_P1 on the
// P2 strided subsets, twiddles w_P^(n2 k1), DFT_P2 on the P1 contiguous groups
// (the "four-step" factorisation applied inside the registers).  No second array
// is needed; output k is left at x[ip_rev(P, k) * STRIDE], a digit permutation
// that the callers apply when they store.
__host__ __device__ constexpr int ip_first(int P) { return P == 6 ? 2 : (P % 4 == 0 ? 4 : (P % 2 == 0 ? 2 : 3)); }
__host__ __device__ constexpr int ip_rev(int P, int k) {
    return P <= 4 ? k : (P / ip_first(P)) * (k % ip_first(P)) + ip_rev(P / ip_first(P), k / ip_first(P));
}

template <typename T, int N, int P, int OFF, int STRIDE, int DIR> struct IPDFT {
    __device__ __forceinline__ static void run(cx<T> (&x)[N]) {
        constexpr int P1 = ip_first(P), P2 = P / P1;
        IPDFT_subsets<0, P2>(x);
#pragma unroll
        for (int n2 = 1; n2 < P2; ++n2) {
#pragma unroll
            for (int k1 = 1; k1 < P1; ++k1) {
                cx<T> w = Tw96<T>::get((n2 * k1 * (96 / P)) % 96);
                if (DIR > 0) w.y = -w.y;
                const int e = OFF + (n2 + P2 * ip_rev(P1, k1)) * STRIDE;
                x[e] = cmul(x[e], w);
            }
        }
        IPDFT_groups<0, P1>(x);
    }
    // DFT_P1 on the P2 strided subsets n2 + P2 n1
    template <int n2, int P2> __device__ __forceinline__ static void IPDFT_subsets(cx<T> (&x)[N]) {
        if constexpr (n2 < P2) {
            IPDFT<T, N, ip_first(P), OFF + n2 * STRIDE, STRIDE * P2, DIR>::run(x);
            IPDFT_subsets<n2 + 1, P2>(x);
        }
    }
    // DFT_P2 on the P1 contiguous groups
    template <int r, int P1> __device__ __forceinline__ static void IPDFT_groups(cx<T> (&x)[N]) {
        if constexpr (r < P1) {
            IPDFT<T, N, P / P1, OFF + (P / P1) * r * STRIDE, STRIDE, DIR>::run(x);
            IPDFT_groups<r + 1, P1>(x);
        }
    }
};
template <typename T, int N, int OFF, int STRIDE, int DIR> struct IPDFT<T, N, 1, OFF, STRIDE, DIR> {
    __device__ __forceinline__ static void run(cx<T> (&)[N]) {}
};
template <typename T, int N, int OFF, int STRIDE, int DIR> struct IPDFT<T, N, 2, OFF, STRIDE, DIR> {
    __device__ __forceinline__ static void run(cx<T> (&x)[N]) {
        cx<T> v[2] = {x[OFF], x[OFF + STRIDE]};
        Bfly<T, 2, DIR>::run(v);
        x[OFF] = v[0];
        x[OFF + STRIDE] = v[1];
    }
};
template <typename T, int N, int OFF, int STRIDE, int DIR> struct IPDFT<T, N, 3, OFF, STRIDE, DIR> {
    __device__ __forceinline__ static void run(cx<T> (&x)[N]) {
        cx<T> v[3] = {x[OFF], x[OFF + STRIDE], x[OFF + 2 * STRIDE]};
        Bfly<T, 3, DIR>::run(v);
        x[OFF] = v[0];
        x[OFF + STRIDE] = v[1];
        x[OFF + 2 * STRIDE] = v[2];
    }
};
template <typename T, int N, int OFF, int STRIDE, int DIR> struct IPDFT<T, N, 4, OFF, STRIDE, DIR> {
    __device__ __forceinline__ static void run(cx<T> (&x)[N]) {
        cx<T> v[4] = {x[OFF], x[OFF + STRIDE], x[OFF + 2 * STRIDE], x[OFF + 3 * STRIDE]};
        Bfly<T, 4, DIR>::run(v);
        x[OFF] = v[0];
        x[OFF + STRIDE] = v[1];
        x[OFF + 2 * STRIDE] = v[2];
        x[OFF + 3 * STRIDE] = v[3];
    }
};

// ------------------------------------------------------------------ two-level smem FFT
// A length-N sequence (N = N1 * N2) lives in shared memory as an N1 x (N2+1)
// padded matrix: element (row r, col c) at base + r*(N2+1) + c.  The padding
// keeps the strided row-pass accesses free of bank conflicts.
//   forward:  input x[p] at (p / N2, p % N2)  [natural]
//             column pass: DFT_N1 down each column, multiply (q1, p2) by w_N^(p2 q1)
//             row pass:    DFT_N2 along each row
//             output X[q] at (q % N1, q / N1)  ["transposed"]
//   inverse:  input at the transposed positions, row pass (DFT_N2^-1), multiply by
//             w_N^-(p2 q1), column pass (DFT_N1^-1); output natural, unnormalised.
// tw: the four-step twiddles w_N^(a b), w_N = exp(-2 pi i / N), as two tables laid out
// so that the lanes of a pass read consecutive entries: forward F[q1 N2 + p2] (column
// pass, lanes over columns p2), then inverse I[p2 N1 + q1] at tw + N (row pass, lanes
// over rows q1).  Global memory, read through the L1 cache.
__host__ __device__ __forceinline__ int fft_pos_nat(int p, int N2) { return (p / N2) * (N2 + 1) + (p % N2); }
__host__ __device__ __forceinline__ int fft_pos_tr(int q, int N1, int N2) { return (q % N1) * (N2 + 1) + (q / N1); }
__host__ __device__ __forceinline__ int fft_seq_len(int N1, int N2) { return N1 * (N2 + 1); }

template <typename T> __device__ __forceinline__ cx<T> ld_tw(const cx<T> *tw, int r);
template <> __device__ __forceinline__ cx<float> ld_tw<float>(const cx<float> *tw, int r) {
    float2 v = __ldg(reinterpret_cast<const float2 *>(tw) + r);
    return {v.x, v.y};
}
template <> __device__ __forceinline__ cx<double> ld_tw<double>(const cx<double> *tw, int r) {
    double2 v = __ldg(reinterpret_cast<const double2 *>(tw) + r);
    return {v.x, v.y};
}

// store DFT outputs q = Q..P-1 (held at x[ip_rev(P, q)]) to base[q * ld], optionally
// multiplied by tw[q * tstep] (conjugated when CONJ); compile-time recursion so that
// every register index is a constant
template <typename T, int P, int Q, bool TWID, bool CONJ>
__device__ __forceinline__ void ip_store(cx<T> (&x)[P], cx<T> *base, int ld, const cx<T> *tw, int tstep) {
    if constexpr (Q < P) {
        cx<T> v = x[ip_rev(P, Q)];
        if constexpr (TWID && Q > 0) {
            const cx<T> t = ld_tw<T>(tw, Q * tstep);
            v = CONJ ? cmulc(v, t) : cmul(v, t);
        }
        base[Q * ld] = v;
        ip_store<T, P, Q + 1, TWID, CONJ>(x, base, ld, tw, tstep);
    }
}

// column task: DFT_N1 down column c of one sequence (P == N1); forward multiplies output
// q1 by w_N^(q1 c) = F[q1 N2 + c] (ld = N2 + 1)
template <typename T, int P, int DIR>
__device__ __forceinline__ void fft_col_task(cx<T> *seq, int c, int ld, const cx<T> *tw) {
    cx<T> x[P];
#pragma unroll
    for (int r = 0; r < P; ++r) x[r] = seq[r * ld + c];
    IPDFT<T, P, P, 0, 1, DIR>::run(x);
    if (DIR < 0 && c > 0) ip_store<T, P, 0, true, false>(x, seq + c, ld, tw + c, ld - 1);
    else ip_store<T, P, 0, false, false>(x, seq + c, ld, tw, 0);
}
// row task: DFT_N2 along row q1 of one sequence (P == N2); inverse then multiplies output
// p2 by w_N^-(p2 q1) = conj(I[p2 N1 + q1]), I at tw + N1 N2
template <typename T, int P, int DIR>
__device__ __forceinline__ void fft_row_task(cx<T> *seq, int q1, int ld, const cx<T> *tw, int N1) {
    cx<T> x[P];
    cx<T> *row = seq + q1 * ld;
#pragma unroll
    for (int c = 0; c < P; ++c) x[c] = row[c];
    IPDFT<T, P, P, 0, 1, DIR>::run(x);
    if (DIR > 0 && q1 > 0) ip_store<T, P, 0, true, true>(x, row, 1, tw + N1 * P + q1, N1);
    else ip_store<T, P, 0, false, false>(x, row, 1, tw, 0);
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FDiv &f) { return (__umulhi(n, f.m) + n) >> f.s; }

template <typename T, int P, int DIR>
__device__ __forceinline__ void fft_col_pass_P(cx<T> *buf, int nseq, int sstride, int N2, const FDiv &fN2,
                                               const cx<T> *tw, int tid, int nthr) {
    const int ntask = nseq * N2;
    for (int t = tid; t < ntask; t += nthr) {
        const int s = (int)fdiv((unsigned)t, fN2), c = t - s * N2;
        fft_col_task<T, P, DIR>(buf + s * sstride, c, N2 + 1, tw);
    }
}
template <typename T, int P, int DIR>
__device__ __forceinline__ void fft_row_pass_P(cx<T> *buf, int nseq, int sstride, int N1, int N2, const FDiv &fN1,
                                               const cx<T> *tw, int tid, int nthr) {
    const int ntask = nseq * N1;
    for (int t = tid; t < ntask; t += nthr) {
        const int s = (int)fdiv((unsigned)t, fN1), q1 = t - s * N1;
        fft_row_task<T, P, DIR>(buf + s * sstride, q1, N2 + 1, tw, N1);
    }
}

#define IBF_FFT_SIZES(X) X(1) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32)

template <typename T, int DIR>
__device__ __forceinline__ void fft_col_pass(cx<T> *buf, int nseq, int sstride, int N1, int N2, const FDiv &fN2,
                                             const cx<T> *tw, int tid, int nthr) {
    switch (N1) {
#define IBF_CASE(P) case P: fft_col_pass_P<T, P, DIR>(buf, nseq, sstride, N2, fN2, tw, tid, nthr); break;
        IBF_FFT_SIZES(IBF_CASE)
#undef IBF_CASE
        default: break;
    }
}
template <typename T, int DIR>
__device__ __forceinline__ void fft_row_pass(cx<T> *buf, int nseq, int sstride, int N1, int N2, const FDiv &fN1,
                                             const cx<T> *tw, int tid, int nthr) {
    switch (N2) {
#define IBF_CASE(P) case P: fft_row_pass_P<T, P, DIR>(buf, nseq, sstride, N1, N2, fN1, tw, tid, nthr); break;
        IBF_FFT_SIZES(IBF_CASE)
#undef IBF_CASE
        default: break;
    }
}

// One warp, one sequence whose input arrives dense (row stride N2, as a contiguous copy
// leaves it): the column pass reads that layout and writes its outputs to the padded one
// (row stride N2 + 1) in the same buffer.  One column task per lane (N2 <= 32), and every
// lane's reads come before any lane's writes (a __syncwarp between), so the in-place
// change of layout is safe; the row pass then runs on the padded layout as usual.
template <typename T, int P, int DIR>
__device__ __forceinline__ void fft_col_task_dense_in(cx<T> *seq, int c, bool active, int N2, const cx<T> *tw) {
    cx<T> x[P];
#pragma unroll
    for (int r = 0; r < P; ++r) x[r] = active ? seq[r * N2 + c] : cx<T>{(T)0, (T)0};
    __syncwarp();
    if (!active) return;
    IPDFT<T, P, P, 0, 1, DIR>::run(x);
    if (DIR < 0 && c > 0) ip_store<T, P, 0, true, false>(x, seq + c, N2 + 1, tw + c, N2);
    else ip_store<T, P, 0, false, false>(x, seq + c, N2 + 1, tw, 0);
}
template <typename T, int DIR>
__device__ __forceinline__ void fft_col_pass_dense_in(cx<T> *buf, int N1, int N2, const cx<T> *tw, int lane) {
    const bool active = lane < N2;
    switch (N1) {
#define IBF_CASE(P) case P: fft_col_task_dense_in<T, P, DIR>(buf, lane, active, N2, tw); break;
        IBF_FFT_SIZES(IBF_CASE)
#undef IBF_CASE
        default: break;
    }
}

// Batch of nseq sequences at buf + s * sstride.  Ends with a __syncthreads().
template <typename T, int DIR>
__device__ __forceinline__ void fft_batch(cx<T> *buf, int nseq, int sstride, int N1, int N2, const FDiv &fN1,
                                          const FDiv &fN2, const cx<T> *tw) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (DIR < 0) {
        fft_col_pass<T, DIR>(buf, nseq, sstride, N1, N2, fN2, tw, tid, nthr);
        __syncthreads();
        fft_row_pass<T, DIR>(buf, nseq, sstride, N1, N2, fN1, tw, tid, nthr);
    } else {
        fft_row_pass<T, DIR>(buf, nseq, sstride, N1, N2, fN1, tw, tid, nthr);
        __syncthreads();
        fft_col_pass<T, DIR>(buf, nseq, sstride, N1, N2, fN2, tw, tid, nthr);
    }
    __syncthreads();
}

// natural position p -> (p / N2) (N2+1) + p % N2 = p + p / N2
__device__ __forceinline__ int pos_nat(int p, const FDiv &fN2) { return p + (int)fdiv((unsigned)p, fN2); }
// transposed position of mode q: (q % N1) (N2+1) + q / N1
__device__ __forceinline__ int pos_tr(int q, int N1, int N2, const FDiv &fN1) {
    const int a = (int)fdiv((unsigned)q, fN1);
    return (q - a * N1) * (N2 + 1) + a;
}

}  // namespace ibf
