// Complex double-FP32 arithmetic on packed float pairs.
//
// A complex df value z = (re.hi + re.lo) + i (im.hi + im.lo) is operated on
// as two 64-bit registers of two floats each, H = (re.hi, im.hi) and
// L = (re.lo, im.lo), with the sm_100-family paired instructions
// add/sub/mul/fma.rn.f32x2: one instruction does the same IEEE operation
// with round-to-nearest on both lanes, so every error-free transformation
// of wc_df.cuh (TwoSum, Fast2Sum, the FMA product error) runs for the real
// and the imaginary part at once.  The lane-wise operations and their order
// are exactly those of the scalar df operators (a - b is computed as
// a + (-b) would be: IEEE subtraction equals addition of the negation), so
// results are bit-identical to the scalar forms; only the instruction count
// changes (a complex df add 11 instead of 22 issues, a complex df
// multiply-add about 37 instead of 60).
//
// These overloads of the complex operators for cx<df> are found by
// argument-dependent lookup from the templated stencil code.
#pragma once

#include <cuda_runtime.h>

namespace wc {

namespace f2 {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float a, float b)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(u64 r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ u64 add(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// sign flips: both lanes, lane 0 only (the real part), lane 1 only
__device__ __forceinline__ u64 neg(u64 a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ u64 neg0(u64 a) { return a ^ 0x0000000080000000ull; }
__device__ __forceinline__ u64 neg1(u64 a) { return a ^ 0x8000000000000000ull; }

// a packed complex df
struct z2 {
    u64 h, l;
};

__device__ __forceinline__ z2 to2(const cx<df> &z) { return z2{pk(z.re.hi, z.im.hi), pk(z.re.lo, z.im.lo)}; }
__device__ __forceinline__ cx<df> from2(const z2 &z)
{
    float rh, ih, rl, il;
    upk(z.h, rh, ih);
    upk(z.l, rl, il);
    return cx<df>{df(rh, rl), df(ih, il)};
}
// both lanes carry the real (or the imaginary) part of z
__device__ __forceinline__ z2 bcast(df x) { return z2{pk(x.hi, x.hi), pk(x.lo, x.lo)}; }
// (im, re)
__device__ __forceinline__ z2 swap(const cx<df> &z) { return z2{pk(z.im.hi, z.re.hi), pk(z.im.lo, z.re.lo)}; }

// lane-wise df sum (the scalar operator+ of wc_df.cuh on both lanes)
__device__ __forceinline__ z2 dadd(const z2 &a, const z2 &b)
{
    const u64 s = add(a.h, b.h);
    const u64 bb = sub(s, a.h);
    const u64 e = add(sub(a.h, sub(s, bb)), sub(b.h, bb));
    const u64 t = add(e, add(a.l, b.l));
    const u64 hi = add(s, t);
    return z2{hi, sub(t, sub(hi, s))};
}
// lane-wise df product (operator* of wc_df.cuh)
__device__ __forceinline__ z2 dmul(const z2 &a, const z2 &b)
{
    const u64 p = mul(a.h, b.h);
    u64 e = fma(a.h, b.h, neg(p));
    e = fma(a.h, b.l, e);
    e = fma(a.l, b.h, e);
    const u64 hi = add(p, e);
    return z2{hi, sub(e, sub(hi, p))};
}
// lane-wise a * b + c (fma of wc_df.cuh)
__device__ __forceinline__ z2 dfma(const z2 &a, const z2 &b, const z2 &c)
{
    const u64 p = mul(a.h, b.h);
    u64 e = fma(a.h, b.h, neg(p));
    e = fma(a.h, b.l, e);
    e = fma(a.l, b.h, e);
    const u64 s = add(p, c.h);
    const u64 bb = sub(s, p);
    const u64 se = add(sub(p, sub(s, bb)), sub(c.h, bb));
    const u64 t = add(se, add(e, c.l));
    const u64 hi = add(s, t);
    return z2{hi, sub(t, sub(hi, s))};
}

}  // namespace f2

__device__ __forceinline__ cx<df> operator+(cx<df> a, cx<df> b) { return f2::from2(f2::dadd(f2::to2(a), f2::to2(b))); }
__device__ __forceinline__ cx<df> operator-(cx<df> a)
{
    return cx<df>{df(-a.re.hi, -a.re.lo), df(-a.im.hi, -a.im.lo)};
}
__device__ __forceinline__ cx<df> operator-(cx<df> a, cx<df> b)
{
    const f2::z2 nb = f2::to2(b);
    return f2::from2(f2::dadd(f2::to2(a), f2::z2{f2::neg(nb.h), f2::neg(nb.l)}));
}
// (a.re b.re - a.im b.im, a.re b.im + a.im b.re)
__device__ __forceinline__ cx<df> operator*(cx<df> a, cx<df> b)
{
    const f2::z2 p = f2::dmul(f2::bcast(a.re), f2::to2(b));   // (a.re b.re, a.re b.im)
    const f2::z2 q = f2::dmul(f2::bcast(a.im), f2::swap(b));  // (a.im b.im, a.im b.re)
    return f2::from2(f2::dadd(p, f2::z2{f2::neg0(q.h), f2::neg0(q.l)}));
}
__device__ __forceinline__ cx<df> operator*(df s, cx<df> a) { return f2::from2(f2::dmul(f2::bcast(s), f2::to2(a))); }
// acc + a * b: lanes (re, im) take a.re (b.re, b.im), then (-a.im b.im, a.im b.re)
__device__ __forceinline__ cx<df> cfma(cx<df> a, cx<df> b, cx<df> acc)
{
    f2::z2 r = f2::dfma(f2::bcast(a.re), f2::to2(b), f2::to2(acc));
    const f2::z2 ai = f2::bcast(a.im);
    r = f2::dfma(f2::z2{f2::neg0(ai.h), f2::neg0(ai.l)}, f2::swap(b), r);
    return f2::from2(r);
}
// acc + conj(a) * b: a.re (b.re, b.im), then (a.im b.im, -a.im b.re)
__device__ __forceinline__ cx<df> cfma_conj(cx<df> a, cx<df> b, cx<df> acc)
{
    f2::z2 r = f2::dfma(f2::bcast(a.re), f2::to2(b), f2::to2(acc));
    const f2::z2 ai = f2::bcast(a.im);
    r = f2::dfma(f2::z2{f2::neg1(ai.h), f2::neg1(ai.l)}, f2::swap(b), r);
    return f2::from2(r);
}

}  // namespace wc
