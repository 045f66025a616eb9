// Double-float arithmetic on GB300: values are unevaluated sums hi + lo of two
// floats (about 48 significant bits), operated on with the error-free
// transformations TwoSum (Knuth) and FMA-based TwoProd (Dekker) on the FP32
// pipe.  GB300 executes FP64 arithmetic and FP64 <-> FP32 conversions at 1/58
// of its FP32 rate, so the kernels that read or write FP64 arrays convert with
// integer bit operations: splitting a double costs one FP64 subtraction, and
// forming a double from a pair one FP64 addition.
#pragma once

#include <cuda_runtime.h>

struct dfloat {
    float h, l;
};

__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float &s, float &e) {  // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}

// The rare paths by conversion, kept out of line: inlined, the compiler
// predicates them and the predicated-off conversions still occupy the narrow
// FP64 pipe on every call.
static __device__ __noinline__ dfloat df_split_slow(double x) {
    dfloat r;
    r.h = __double2float_rn(x);
    r.l = __double2float_rn(x - double(r.h));
    return r;
}
static __device__ __noinline__ double df_f2d_slow(float f) { return double(f); }

// The pair of the double with bit pattern b, taken with exponent field E (E equal
// to b's own field, or shifted to scale the value by a power of two); E must lie in
// [950, 1150].  hi keeps the top 24 significand bits (truncated), lo the next 24 of
// the remaining 29 (the pair is exact to 2^-48 relative).
__device__ __forceinline__ dfloat df_split_bits(unsigned long long b, unsigned E) {
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    dfloat r;
    const unsigned sgn = hi32 & 0x80000000u;
    const unsigned mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);  // top 23 fraction bits
    r.h = __uint_as_float(sgn | ((E - 896u) << 23) | mh);
    const unsigned L = lo32 & 0x1fffffffu;  // the low 29 fraction bits: L 2^(E-1075)
    r.l = 0.f;
    if (L) {
        const int k = 31 - __clz(L);  // leading one
        const unsigned sig = k >= 23 ? (L >> (k - 23)) : (L << (23 - k));
        r.l = __uint_as_float(sgn | ((unsigned)(k + (int)E - 948) << 23) | (sig & 0x7fffffu));
    }
    return r;
}

// x = hi + lo from the bit pattern with integer operations; zero gives (0, 0) and
// other exponents outside [2^-73, 2^127) (tiny, huge, non-finite) take the
// conversion path.
__device__ __forceinline__ dfloat df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
    if (E < 950u || E > 1150u) {
        if ((b << 1) == 0ull) return dfloat{__uint_as_float((unsigned)(b >> 32) & 0x80000000u), 0.f};  // +-0
        return df_split_slow(x);
    }
    return df_split_bits(b, E);
}

// the float's value as a double, from its bit pattern (normal floats; zero,
// subnormal and non-finite values take the conversion path)
__device__ __forceinline__ double df_f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
        return df_f2d_slow(f);
    }
    const unsigned hi32 = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    const unsigned lo32 = u << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi32 << 32) | lo32));
}
__device__ __forceinline__ double df_to_double(dfloat a) { return df_f2d(a.h) + df_f2d(a.l); }

__device__ __forceinline__ dfloat df_norm(float h, float l) {
    dfloat r;
    df_fast_two_sum(h, l, r.h, r.l);
    return r;
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    float s, e;
    df_two_sum(a.h, b.h, s, e);
    e += a.l + b.l;
    return df_norm(s, e);
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat{-a.h, -a.l}; }
__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_norm(p, e);
}
// a / b: q1 = a_h / b_h, then the remainder a - q1 b (exact product by FMA)
// divided once more
__device__ __forceinline__ dfloat df_div(dfloat a, dfloat b) {
    const float q1 = a.h / b.h;
    const float p = q1 * b.h;
    const float pe = fmaf(q1, b.h, -p);
    const float r = (((a.h - p) - pe) + a.l) - q1 * b.l;
    return df_norm(q1, r / b.h);
}

// m = the larger of m and |v| (by hi, then lo), both double-float; NaN propagates
__device__ __forceinline__ void df_absmax(dfloat &m, dfloat v) {
    const bool neg = v.h < 0.f || (v.h == 0.f && v.l < 0.f);
    const dfloat a = neg ? dfloat{-v.h, -v.l} : v;
    // a NaN value wins and then stays (every comparison with it is false)
    const bool gt = a.h > m.h || (a.h == m.h && a.l > m.l) || a.h != a.h;
    m = gt ? a : m;
}
