// Device-side types of libwc: complex arithmetic, lattice geometry, the
// device layouts of links and clover, and the per-precision load/store
// traits shared by all kernels.
//
// Device layouts (V = lattice volume, every array plane-major so that one
// warp's 16-byte loads of one component plane are contiguous):
//   spinor  F64: double2 [12][V]       component k = 3*spin + colour
//           F32: float4  [6][V]        chunk j = components 2j, 2j+1
//           F16: uint4   [3][V]        chunk j = components 4j..4j+3 (half2
//                each), times float scale[V] (max |real| of the site)
//   links   FP32/FP16: rows 0 and 1 of U_mu(x) (6 complex, row-major); row 2
//           is rebuilt in registers as conj(row0 x row1) (paper Sec. 2,
//           SU(3) reconstruction) -- these kernels are bandwidth-bound.
//           FP64: all three rows, the third computed once at load time by
//           the same formula: on GB300 the FP64 operator is bound by the
//           FP64 pipe, not by bandwidth, so the rebuild is not repeated.
//           F64: double2 [4][9][V]     F32: float4 [4][3][V]
//           F16: uint4 [4][V] (complex 0..3) + uint2 [4][V] (complex 4, 5)
//   clover  A = 1 + T as two Hermitian 6x6 blocks (spins {0,1} and {2,3},
//           index 3*s_local + colour): per block 6 real diagonal entries then
//           the 15 complex entries below the diagonal in row order
//           (1,0) (2,0) (2,1) (3,0) ... (5,4); 72 reals per site
//           F64: double2 [36][V]       F32: float4 [18][V]    F16: uint4 [9][V]
//   FP64 links and clover are also kept split into double-FP32 pairs (same
//   planes, float4 = hi, lo of the real part, hi, lo of the imaginary part)
//   for the double-FP32 operator (wc_df.cuh).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "wc_check.cuh"
#include "wc_df.cuh"

namespace wc {

// ------------------------------------------------------------------------
// complex arithmetic
// ------------------------------------------------------------------------

template <class R>
struct cx {
    R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) { return cx<R>{a, b}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
// i * a
template <class R>
__host__ __device__ __forceinline__ cx<R> times_i(cx<R> a) { return {-a.im, a.re}; }
// conj(a) * b
template <class R>
__host__ __device__ __forceinline__ cx<R> cmul_conj(cx<R> a, cx<R> b)
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc + a * b
template <class R>
__host__ __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a) * b
template <class R>
__host__ __device__ __forceinline__ cx<R> cfma_conj(cx<R> a, cx<R> b, cx<R> acc)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}

}  // namespace wc

// the same operators for complex double-FP32 values, on packed float pairs
#include "wc_df2.cuh"

namespace wc {

// ------------------------------------------------------------------------
// geometry
// ------------------------------------------------------------------------

// Division of a non-negative index n < 2^31 by a fixed divisor d without
// the integer-divide instruction sequence: q = floor(n m / 2^k) with
// k = 31 + ceil(log2 d) and m = ceil(2^k / d) < 2^32 is floor(n / d) for
// every such n (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994: m d - 2^k < d <= 2^(k - 31)).
struct FastDiv {
    unsigned m;
    int k;
};

inline FastDiv make_fastdiv(int d)
{
    int l = 0;
    while ((1LL << l) < d) ++l;
    const int k = 31 + l;
    const unsigned long long p = 1ULL << k;
    return FastDiv{(unsigned)((p + (unsigned long long)d - 1) / (unsigned long long)d), k};
}

__host__ __device__ __forceinline__ int fast_div(int n, FastDiv f)
{
    return (int)(((unsigned long long)(unsigned)n * f.m) >> f.k);
}

struct Geom {
    int L[4];
    int stride[4];  // 1, Lx, Lx*Ly, Lx*Ly*Lz
    int V;
    int tbc;        // +1 or -1
    FastDiv div[3]; // by L[0], L[1], L[2]
};

// the fast divisors of g.L (host, after L is set)
inline void geom_set_div(Geom &g)
{
    for (int m = 0; m < 3; ++m) g.div[m] = make_fastdiv(g.L[m]);
}

__device__ __forceinline__ void site_coords(const Geom &g, int s, int c[4])
{
    c[0] = s % g.L[0];
    s /= g.L[0];
    c[1] = s % g.L[1];
    s /= g.L[1];
    c[2] = s % g.L[2];
    c[3] = s / g.L[2];
}

// site_coords with the divisions by multiplication.  Measured per operator:
// the FP16 kernel (bound by instruction issue) gains 3 %, the FP32 kernel
// (at 80 registers, bandwidth-bound) loses 2 %, so only the FP16 path uses it.
__device__ __forceinline__ void site_coords_fast(const Geom &g, int s, int c[4])
{
    int q = fast_div(s, g.div[0]);
    c[0] = s - q * g.L[0];
    s = q;
    q = fast_div(s, g.div[1]);
    c[1] = s - q * g.L[1];
    s = q;
    q = fast_div(s, g.div[2]);
    c[2] = s - q * g.L[2];
    c[3] = q;
}

// ------------------------------------------------------------------------
// raw device stores of a lattice
// ------------------------------------------------------------------------

struct GaugeStore {
    double2 *u64 = nullptr;   // [4][9][V]
    float4 *udf = nullptr;    // [4][9][V] u64 as double-FP32 pairs
    float4 *u32 = nullptr;    // [4][3][V]
    uint4 *u16a = nullptr;    // [4][V]  row 0, row 1 entry 0
    uint2 *u16b = nullptr;    // [4][V]  row 1 entries 1, 2
};

struct CloverStore {
    double2 *c64 = nullptr;   // [36][V]
    float4 *cdf = nullptr;    // [36][V] c64 as double-FP32 pairs
    float4 *c32 = nullptr;    // [18][V]
    uint4 *c16 = nullptr;     // [9][V]
};

// Scalars of one BiCGStab solve, resident on the device.
struct SolverScalars {
    double2 rho, rho0, alpha, omega, beta;
    double rr;       // |r|^2
    double pp, ss;   // |p|^2, |s|^2 (scales of the defect correction)
    double tt;
    int flags;       // bit 0: breakdown, bit 1: non-finite value
    int skip;        // lockstep batch: 1 = this right-hand side has stopped, and
                     // the low-precision step kernels return at once (0 otherwise)
};

enum { FLAG_BREAKDOWN = 1, FLAG_NAN = 2 };

// Reduction scratch: per-block partial sums and a completion ticket.
struct ReduceScratch {
    double *partials = nullptr;   // [max_blocks][8]
    unsigned *ticket = nullptr;
    double *result = nullptr;     // [8] final sums (device)
    double *host_result = nullptr;  // [8] pinned host mirror
    int max_blocks = 0;
};

// ------------------------------------------------------------------------
// precision traits: loads and stores of the device layouts
// ------------------------------------------------------------------------

__device__ __forceinline__ cx<float> h2c(unsigned v)
{
    __half2 h = *reinterpret_cast<__half2 *>(&v);
    float2 f = __half22float2(h);
    return {f.x, f.y};
}

__device__ __forceinline__ unsigned c2h(float re, float im)
{
    __half2 h = __floats2half2_rn(re, im);
    return *reinterpret_cast<unsigned *>(&h);
}

// max(a, b, c) in one instruction (three-input max.f32)
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// third row of an SU(3) matrix from its first two: c = conj(a x b)
template <class R>
__device__ __forceinline__ void reconstruct_row2(const cx<R> u[6], cx<R> c[3])
{
    c[0] = conj(u[1] * u[5] - u[2] * u[4]);
    c[1] = conj(u[2] * u[3] - u[0] * u[5]);
    c[2] = conj(u[0] * u[4] - u[1] * u[3]);
}

struct P64 {
    using real = double;
    // register caps of the operator's launch shapes (bit 0: cap 1, bit 1:
    // cap 2) and the minimum resident 256-thread CTAs that cap 1 stands for
    static constexpr int kCaps = 0;   // ALU-bound on the FP64 pipe: no cap
    static constexpr int kCap1MinBlocks = 1;
    static constexpr int kEoMinBlocks = 1;   // even-odd kernel: minimum resident CTAs of 128
    static __device__ __forceinline__ void load_spinor(const void *d, const float *, int V, int x,
                                                       cx<double> s[12])
    {
        const double2 *p = static_cast<const double2 *>(d);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = __ldg(p + (size_t)k * V + x);
            s[k] = {v.x, v.y};
        }
    }
    // the stored values and the factor they must be multiplied by (1 here)
    static __device__ __forceinline__ double load_spinor_raw(const void *d, const float *n, int V, int x,
                                                             cx<double> s[12])
    {
        load_spinor(d, n, V, x, s);
        return 1.0;
    }
    static __device__ __forceinline__ void store_spinor(void *d, float *, int V, int x,
                                                        const cx<double> s[12])
    {
        double2 *p = static_cast<double2 *>(d);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + x] = make_double2(s[k].re, s[k].im);
    }
    // s as a store_spinor followed by a load_spinor returns it (computed in
    // registers: load_spinor reads through the non-coherent path, which need
    // not see a write of the same kernel)
    static __device__ __forceinline__ void as_stored(cx<double> s[12]) {}
    // U_mu(x): a[0..2] = row 0, a[3..5] = row 1, c[0..2] = row 2
    static __device__ __forceinline__ void load_link(const GaugeStore &g, int V, int mu, int x,
                                                     cx<double> a[6], cx<double> c[3])
    {
        const double2 *p = g.u64 + (size_t)mu * 9 * V + x;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 v = __ldg(p + (size_t)k * V);
            a[k] = {v.x, v.y};
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double2 v = __ldg(p + (size_t)(6 + k) * V);
            c[k] = {v.x, v.y};
        }
    }
    // the 36 reals of clover block b
    static __device__ __forceinline__ void load_clover(const CloverStore &c, int V, int x, int b,
                                                       double r[36])
    {
        const double2 *p = c.c64 + (size_t)b * 18 * V + x;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            double2 v = __ldg(p + (size_t)k * V);
            r[2 * k] = v.x;
            r[2 * k + 1] = v.y;
        }
    }
};

struct P32 {
    using real = float;
    static constexpr int kCaps = 3;   // cap 1: 64 registers, cap 2: 85
    static constexpr int kCap1MinBlocks = 4;
    static constexpr int kEoMinBlocks = 1;
    static __device__ __forceinline__ void load_spinor(const void *d, const float *, int V, int x,
                                                       cx<float> s[12])
    {
        const float4 *p = static_cast<const float4 *>(d);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float4 v = __ldg(p + (size_t)j * V + x);
            s[2 * j] = {v.x, v.y};
            s[2 * j + 1] = {v.z, v.w};
        }
    }
    static __device__ __forceinline__ float load_spinor_raw(const void *d, const float *n, int V, int x,
                                                            cx<float> s[12])
    {
        load_spinor(d, n, V, x, s);
        return 1.f;
    }
    static __device__ __forceinline__ void store_spinor(void *d, float *, int V, int x,
                                                        const cx<float> s[12])
    {
        float4 *p = static_cast<float4 *>(d);
#pragma unroll
        for (int j = 0; j < 6; ++j)
            p[(size_t)j * V + x] = make_float4(s[2 * j].re, s[2 * j].im, s[2 * j + 1].re, s[2 * j + 1].im);
    }
    // s as a store_spinor followed by a load_spinor returns it
    static __device__ __forceinline__ void as_stored(cx<float> s[12]) {}
    static __device__ __forceinline__ void load_link(const GaugeStore &g, int V, int mu, int x,
                                                     cx<float> a[6], cx<float> c[3])
    {
        const float4 *p = g.u32 + (size_t)mu * 3 * V + x;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float4 v = __ldg(p + (size_t)j * V);
            a[2 * j] = {v.x, v.y};
            a[2 * j + 1] = {v.z, v.w};
        }
        reconstruct_row2(a, c);
    }
    static __device__ __forceinline__ void load_clover(const CloverStore &c, int V, int x, int b,
                                                       float r[36])
    {
        const float4 *p = c.c32 + (size_t)b * 9 * V + x;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float4 v = __ldg(p + (size_t)k * V);
            r[4 * k] = v.x;
            r[4 * k + 1] = v.y;
            r[4 * k + 2] = v.z;
            r[4 * k + 3] = v.w;
        }
    }
};

// FP64 storage, double-FP32 arithmetic (the operator's FP64 path when the
// lattice selects it): spinors are converted on load and store, links and
// clover come from their pre-split copies.
struct PDF {
    using real = df;
    static constexpr int kCaps = 1;   // cap 1: 128 registers (2 CTAs of 256)
    static constexpr int kCap1MinBlocks = 2;
    static constexpr int kEoMinBlocks = 4;   // 128 registers: latency-bound, occupancy pays
    static __device__ __forceinline__ void load_spinor(const void *d, const float *, int V, int x, cx<df> s[12])
    {
        const double2 *p = static_cast<const double2 *>(d);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 v = __ldg(p + (size_t)k * V + x);
            s[k] = {df_from_double(v.x), df_from_double(v.y)};
        }
    }
    static __device__ __forceinline__ df load_spinor_raw(const void *d, const float *n, int V, int x, cx<df> s[12])
    {
        load_spinor(d, n, V, x, s);
        return df(1.0f, 0.0f);
    }
    static __device__ __forceinline__ void store_spinor(void *d, float *, int V, int x, const cx<df> s[12])
    {
        double2 *p = static_cast<double2 *>(d);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + x] = make_double2(df_to_double(s[k].re), df_to_double(s[k].im));
    }
    // s as a store_spinor followed by a load_spinor returns it
    static __device__ __forceinline__ void as_stored(cx<df> s[12])
    {
#pragma unroll
        for (int k = 0; k < 12; ++k)
            s[k] = {df_from_double(df_to_double(s[k].re)), df_from_double(df_to_double(s[k].im))};
    }
    static __device__ __forceinline__ void load_link(const GaugeStore &g, int V, int mu, int x, cx<df> a[6],
                                                     cx<df> c[3])
    {
        const float4 *p = g.udf + (size_t)mu * 9 * V + x;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = __ldg(p + (size_t)k * V);
            a[k] = {df(v.x, v.y), df(v.z, v.w)};
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = __ldg(p + (size_t)(6 + k) * V);
            c[k] = {df(v.x, v.y), df(v.z, v.w)};
        }
    }
    // real entry t (0..5: the diagonal) and complex lower entry m (0..14) of
    // block b at position x
    static __device__ __forceinline__ df clover_real(const CloverStore &c, int V, int x, int b, int t)
    {
        const float4 v = __ldg(c.cdf + (size_t)(b * 18 + (t >> 1)) * V + x);
        return (t & 1) ? df(v.z, v.w) : df(v.x, v.y);
    }
    static __device__ __forceinline__ cx<df> clover_lower(const CloverStore &c, int V, int x, int b, int m)
    {
        const float4 v = __ldg(c.cdf + (size_t)(b * 18 + 3 + m) * V + x);
        return {df(v.x, v.y), df(v.z, v.w)};
    }
    static __device__ __forceinline__ void load_clover(const CloverStore &c, int V, int x, int b, df r[36])
    {
        const float4 *p = c.cdf + (size_t)b * 18 * V + x;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const float4 v = __ldg(p + (size_t)k * V);
            r[2 * k] = df(v.x, v.y);
            r[2 * k + 1] = df(v.z, v.w);
        }
    }
};

struct P16 {
    using real = float;
    static constexpr int kCaps = 3;   // cap 1: 64 registers, cap 2: 85
    static constexpr int kCap1MinBlocks = 4;
    static constexpr int kEoMinBlocks = 1;
    // stored (unit-scaled) values; returns the site's scale, to be folded
    // into a later coefficient instead of multiplying all 24 components
    static __device__ __forceinline__ float load_spinor_raw(const void *d, const float *nrm, int V, int x,
                                                            cx<float> s[12])
    {
        const uint4 *p = static_cast<const uint4 *>(d);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 v = __ldg(p + (size_t)j * V + x);
            s[4 * j] = h2c(v.x);
            s[4 * j + 1] = h2c(v.y);
            s[4 * j + 2] = h2c(v.z);
            s[4 * j + 3] = h2c(v.w);
        }
        return __ldg(nrm + x);
    }
    static __device__ __forceinline__ void load_spinor(const void *d, const float *nrm, int V, int x,
                                                       cx<float> s[12])
    {
        const uint4 *p = static_cast<const uint4 *>(d);
        const float sc = __ldg(nrm + x);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 v = __ldg(p + (size_t)j * V + x);
            s[4 * j] = sc * h2c(v.x);
            s[4 * j + 1] = sc * h2c(v.y);
            s[4 * j + 2] = sc * h2c(v.z);
            s[4 * j + 3] = sc * h2c(v.w);
        }
    }
    static __device__ __forceinline__ void store_spinor(void *d, float *nrm, int V, int x,
                                                        const cx<float> s[12])
    {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmax3(m, fabsf(s[k].re), fabsf(s[k].im));
        const float inv = m > 0.f ? 1.f / m : 0.f;
        uint4 *p = static_cast<uint4 *>(d);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 v;
            v.x = c2h(s[4 * j].re * inv, s[4 * j].im * inv);
            v.y = c2h(s[4 * j + 1].re * inv, s[4 * j + 1].im * inv);
            v.z = c2h(s[4 * j + 2].re * inv, s[4 * j + 2].im * inv);
            v.w = c2h(s[4 * j + 3].re * inv, s[4 * j + 3].im * inv);
            p[(size_t)j * V + x] = v;
        }
        nrm[x] = m;
    }
    // s as a store_spinor followed by a load_spinor returns it
    static __device__ __forceinline__ void as_stored(cx<float> s[12])
    {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmax3(m, fabsf(s[k].re), fabsf(s[k].im));
        const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = m * h2c(c2h(s[k].re * inv, s[k].im * inv));
    }
    static __device__ __forceinline__ void load_link(const GaugeStore &g, int V, int mu, int x,
                                                     cx<float> a[6], cx<float> c[3])
    {
        uint4 v = __ldg(g.u16a + (size_t)mu * V + x);
        uint2 w = __ldg(g.u16b + (size_t)mu * V + x);
        a[0] = h2c(v.x);
        a[1] = h2c(v.y);
        a[2] = h2c(v.z);
        a[3] = h2c(v.w);
        a[4] = h2c(w.x);
        a[5] = h2c(w.y);
        reconstruct_row2(a, c);
    }
    static __device__ __forceinline__ void load_clover(const CloverStore &c, int V, int x, int b,
                                                       float r[36])
    {
        // block b occupies reals 36b .. 36b+35 = chunks 4.5b ... : load all 9
        // chunks' halves that belong to it
        const uint4 *p = c.c16 + x;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const int q = 18 * b + k;           // half2 index among 36 per site
            uint4 v = __ldg(p + (size_t)(q >> 2) * V);
            const unsigned w = (q & 3) == 0 ? v.x : (q & 3) == 1 ? v.y : (q & 3) == 2 ? v.z : v.w;
            cx<float> f = h2c(w);
            r[2 * k] = f.re;
            r[2 * k + 1] = f.im;
        }
    }
};

// Hermitian 6x6 block (packed) times a 6-vector: y = B v
template <class R>
__device__ __forceinline__ void clover_block_mul(const R r[36], const cx<R> v[6], cx<R> y[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = r[i] * v[i];
    int k = 6;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const cx<R> l = mkc(r[k], r[k + 1]);
            k += 2;
            y[i] = cfma(l, v[j], y[i]);        // lower entry (i, j)
            y[j] = cfma_conj(l, v[i], y[j]);   // its mirror (j, i) = conj(l)
        }
    }
}

}  // namespace wc
