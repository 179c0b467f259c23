// Double-FP32 ("df") arithmetic for the FP64 operator.
//
// GB300 executes FP64 arithmetic at about 1/64 of its FP32 rate, so the FP64
// Wilson-Clover operator is bound by the FP64 pipe, not by memory.  A df
// value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi),
// about 47 significant bits, and every operation runs on the FP32 pipes
// (roughly 7 instructions per product, 11 per sum, 15 per fused
// multiply-add).  The building blocks are the classical error-free
// transformations:
//   TwoSum (Knuth, TAOCP vol. 2, sec. 4.2.2): s + e = a + b exactly;
//   Fast2Sum (Dekker 1971): the same in 3 operations when |a| >= |b|;
//   the FMA product error: a * b - fl(a * b) = fma(a, b, -fl(a * b)) exactly.
// Sums use the short ("sloppy") double-word addition: its error is below
// ~2^-45 (|a| + |b|), i.e. relative to the operands rather than to the
// result, which is what a stencil sum needs.  Every step uses the _rn
// intrinsics, which the compiler never contracts into an FMA, so that each
// error term is computed exactly.
//
// Conversions from and to FP64 use integer operations and one FP64 addition
// per stored value (FP64 conversions would also run at the reduced rate).
// Range: FP64 values with |x| < 2^-126 read as zero, values with
// |x| < 2^-103 keep 24 bits, |x| >= 2^128 read as infinity; NaN and
// infinity are carried through.
#pragma once

#include <cuda_runtime.h>

namespace wc {

// keep the float and double fma overloads visible next to the df one
using ::fma;

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __device__ explicit df(double x);
};

__device__ __forceinline__ df df_fast2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df df_2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

__device__ __forceinline__ df operator+(df a, df b)
{
    const df s = df_2sum(a.hi, b.hi);
    return df_fast2sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast2sum(p, e);
}

// a * b + c with one final normalisation
__device__ __forceinline__ df fma(df a, df b, df c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df s = df_2sum(p, c.hi);
    return df_fast2sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// FP64 -> df with integer operations: hi = x truncated to 24 significant
// bits, lo = the next 23 bits (truncated), both with the sign of x.
__device__ __forceinline__ df df_from_double(double x)
{
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const unsigned sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu);            // biased FP64 exponent
    const unsigned top = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const int fe = e - 896;                              // biased FP32 exponent of hi
    unsigned hb;
    if (e == 0x7FF) hb = sign | 0x7F800000u | ((top | (lw & 0x1FFFFFFFu)) ? 0x400000u : 0u);   // inf / NaN
    else if (fe >= 255) hb = sign | 0x7F800000u;
    else if (fe <= 0) hb = sign;
    else hb = sign | ((unsigned)fe << 23) | top;
    float lo = 0.0f;
    const int se = e - 919;                              // biased FP32 exponent of 2^(e - 1046)
    if (se > 0 && e != 0x7FF && fe < 255) {
        const unsigned t = (lw & 0x1FFFFFFFu) >> 6;      // top 23 of the 29 remaining bits
        const float f = __fsub_rn(__uint_as_float(0x3F800000u | t), 1.0f);   // t * 2^-23, exact
        lo = __fmul_rn(f, __uint_as_float((unsigned)se << 23));
        lo = __uint_as_float(__float_as_uint(lo) | sign);
    }
    return df(__uint_as_float(hb), lo);
}

__device__ __forceinline__ df::df(double x) : df(df_from_double(x)) {}

// float -> double, exact, with integer operations (subnormal floats read as 0)
__device__ __forceinline__ double df_f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    if (e == 0) return __hiloint2double((int)sign, 0);
    const unsigned de = e == 0xFFu ? 0x7FFu : e + 896u;
    return __hiloint2double((int)(sign | (de << 20) | (m >> 3)), (int)(m << 29));
}

__device__ __forceinline__ double df_to_double(df a) { return __dadd_rn(df_f2d(a.hi), df_f2d(a.lo)); }

// (re, im) of an FP64 complex as df pairs, packed (hi re, lo re, hi im, lo im)
__device__ __forceinline__ float4 df_pack(double2 v)
{
    const df a = df_from_double(v.x), b = df_from_double(v.y);
    return make_float4(a.hi, a.lo, b.hi, b.lo);
}

}  // namespace wc
