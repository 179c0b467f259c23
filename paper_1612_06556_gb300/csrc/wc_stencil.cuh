// Spin projection, SU(3) two-spinor products and reconstruction shared by
// the operator kernels and the RAS block solver.
//
// Projector algebra in the chiral basis, for P = 1 + s gamma_mu acting on
// psi = (u0, u1, d0, d1) (spins, each a colour 3-vector): the upper half
// h = u + s B_mu d determines the lower half as C_mu h, with
//   mu = x: B = i sigma_1,  C = -s i sigma_1
//   mu = y: B = i sigma_2,  C = -s i sigma_2
//   mu = z: B = i sigma_3,  C = -s i sigma_3
//   mu = t: B = 1,          C = s
// M uses s = -1 for forward hops and s = +1 for backward hops; M^+ =
// gamma5 M gamma5 swaps the two (gamma5 anticommutes with gamma_mu and
// commutes with the block-diagonal clover term).
#pragma once

#include <type_traits>

#include "wc_internal.cuh"

namespace wc {

// S * a for S = +-1, without a multiplication (exact in every arithmetic)
template <int S, class T>
__device__ __forceinline__ T sgn(T a)
{
    return S > 0 ? a : -a;
}

// Two-spinor h of (1 + S gamma_mu) psi, reading the four spin components of
// one colour at a time through ldc(c, u0, u1, d0, d1) (spins 0..3 of
// colour c).
template <int MU, int S, class R, class LoadColour>
__device__ __forceinline__ void project_from(LoadColour ldc, cx<R> h[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<R> u0, u1, d0, d1;
        ldc(c, u0, u1, d0, d1);
        if (MU == 0) {
            h[c] = u0 + sgn<S>(times_i(d1));
            h[3 + c] = u1 + sgn<S>(times_i(d0));
        } else if (MU == 1) {
            h[c] = u0 + sgn<S>(d1);
            h[3 + c] = u1 - sgn<S>(d0);
        } else if (MU == 2) {
            h[c] = u0 + sgn<S>(times_i(d0));
            h[3 + c] = u1 - sgn<S>(times_i(d1));
        } else {
            h[c] = u0 + sgn<S>(d0);
            h[3 + c] = u1 + sgn<S>(d1);
        }
    }
}

template <int MU, int S, class R>
__device__ __forceinline__ void project(const cx<R> p[12], cx<R> h[6])
{
    project_from<MU, S, R>(
        [&](int c, cx<R> &u0, cx<R> &u1, cx<R> &d0, cx<R> &d1) {
            u0 = p[c];
            u1 = p[3 + c];
            d0 = p[6 + c];
            d1 = p[9 + c];
        },
        h);
}

template <int MU, int S, class R>
__device__ __forceinline__ void reconstruct_add(cx<R> acc[12], const cx<R> w[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<R> w0 = w[c], w1 = w[3 + c];
        acc[c] = acc[c] + w0;
        acc[3 + c] = acc[3 + c] + w1;
        if (MU == 0) {
            acc[6 + c] = acc[6 + c] - sgn<S>(times_i(w1));
            acc[9 + c] = acc[9 + c] - sgn<S>(times_i(w0));
        } else if (MU == 1) {
            acc[6 + c] = acc[6 + c] - sgn<S>(w1);
            acc[9 + c] = acc[9 + c] + sgn<S>(w0);
        } else if (MU == 2) {
            acc[6 + c] = acc[6 + c] - sgn<S>(times_i(w0));
            acc[9 + c] = acc[9 + c] + sgn<S>(times_i(w1));
        } else {
            acc[6 + c] = acc[6 + c] + sgn<S>(w0);
            acc[9 + c] = acc[9 + c] + sgn<S>(w1);
        }
    }
}

// w = coef * U h  (per spin of the two-spinor)
template <class R>
__device__ __forceinline__ void su3_mul(const cx<R> u[6], const cx<R> r2[3], const cx<R> h[6], R coef,
                                        cx<R> w[6])
{
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const cx<R> a = h[3 * s], b = h[3 * s + 1], c = h[3 * s + 2];
        cx<R> y0 = u[0] * a, y1 = u[3] * a, y2 = r2[0] * a;
        y0 = cfma(u[1], b, y0);
        y1 = cfma(u[4], b, y1);
        y2 = cfma(r2[1], b, y2);
        y0 = cfma(u[2], c, y0);
        y1 = cfma(u[5], c, y1);
        y2 = cfma(r2[2], c, y2);
        w[3 * s] = coef * y0;
        w[3 * s + 1] = coef * y1;
        w[3 * s + 2] = coef * y2;
    }
}

// w = coef * U^+ h
template <class R>
__device__ __forceinline__ void su3_adj_mul(const cx<R> u[6], const cx<R> r2[3], const cx<R> h[6], R coef,
                                            cx<R> w[6])
{
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const cx<R> a = h[3 * s], b = h[3 * s + 1], c = h[3 * s + 2];
        cx<R> y0 = mkc(R(0), R(0)), y1 = y0, y2 = y0;
        y0 = cfma_conj(u[0], a, y0);
        y1 = cfma_conj(u[1], a, y1);
        y2 = cfma_conj(u[2], a, y2);
        y0 = cfma_conj(u[3], b, y0);
        y1 = cfma_conj(u[4], b, y1);
        y2 = cfma_conj(u[5], b, y2);
        y0 = cfma_conj(r2[0], c, y0);
        y1 = cfma_conj(r2[1], c, y1);
        y2 = cfma_conj(r2[2], c, y2);
        w[3 * s] = coef * y0;
        w[3 * s + 1] = coef * y1;
        w[3 * s + 2] = coef * y2;
    }
}

}  // namespace wc

namespace wc {

// ---- compact forms for the double-FP32 operator ------------------------
// A double-FP32 site costs ~20 k instructions; written out per direction
// (as the FP32/FP16/FP64 kernels are) the code no longer fits the
// instruction cache (ncu: half of the fetches miss, 65 % of the stalls are
// "no instruction").  These forms run the eight hops and the clover rows as
// loops with a runtime index, so that one copy of the SU(3) product and of
// the clover row is in the code.

template <class R>
__device__ __forceinline__ void project_rt(int mu, int s, const cx<R> p[12], cx<R> h[6])
{
    switch (2 * mu + (s > 0)) {
    case 0: project<0, -1>(p, h); break;
    case 1: project<0, 1>(p, h); break;
    case 2: project<1, -1>(p, h); break;
    case 3: project<1, 1>(p, h); break;
    case 4: project<2, -1>(p, h); break;
    case 5: project<2, 1>(p, h); break;
    case 6: project<3, -1>(p, h); break;
    default: project<3, 1>(p, h);
    }
}

template <class R>
__device__ __forceinline__ void reconstruct_add_rt(int mu, int s, cx<R> acc[12], const cx<R> w[6])
{
    switch (2 * mu + (s > 0)) {
    case 0: reconstruct_add<0, -1>(acc, w); break;
    case 1: reconstruct_add<0, 1>(acc, w); break;
    case 2: reconstruct_add<1, -1>(acc, w); break;
    case 3: reconstruct_add<1, 1>(acc, w); break;
    case 4: reconstruct_add<2, -1>(acc, w); break;
    case 5: reconstruct_add<2, 1>(acc, w); break;
    case 6: reconstruct_add<3, -1>(acc, w); break;
    default: reconstruct_add<3, 1>(acc, w);
    }
}

// w = coef * W h with W = U (adj false) or U^+ (adj true), one spin per
// iteration of a runtime loop
template <class R>
__device__ __forceinline__ void su3_mul_rt(bool adj, const cx<R> u[6], const cx<R> r2[3], const cx<R> h[6], R coef,
                                           cx<R> w[6])
{
    cx<R> m[9];
    const cx<R> rows[9] = {u[0], u[1], u[2], u[3], u[4], u[5], r2[0], r2[1], r2[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m[3 * i + j] = adj ? conj(rows[3 * j + i]) : rows[3 * i + j];
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const cx<R> a = s ? h[3] : h[0], b = s ? h[4] : h[1], c = s ? h[5] : h[2];
        cx<R> y[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            y[i] = m[3 * i] * a;
            y[i] = cfma(m[3 * i + 1], b, y[i]);
            y[i] = cfma(m[3 * i + 2], c, y[i]);
            y[i] = coef * y[i];
        }
        if (s) {
            w[3] = y[0];
            w[4] = y[1];
            w[5] = y[2];
        } else {
            w[0] = y[0];
            w[1] = y[1];
            w[2] = y[2];
        }
    }
}

// Hops first..7 of site x (coordinates c; hop 2 mu is the forward, 2 mu + 1
// the backward hop in direction mu) added to acc: acc += k sum [W_fwd (1 +
// SF g_mu) in(x+mu) + W_bwd (1 - SF g_mu) in(x-mu)], the neighbour spinor
// read at sidx(y) of a field of Vin sites.
template <class P, int SF, class SiteIdx>
__device__ __forceinline__ void hops_rt(const Geom &g, const GaugeStore &U, const void *in, const float *in_nrm,
                                        int Vin, int x, const int c[4], typename P::real k,
                                        cx<typename P::real> acc[12], SiteIdx sidx, int first = 0)
{
    using R = typename P::real;
    unsigned wf = 0, wb = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (c[m] == g.L[m] - 1) wf |= 1u << m;
        if (c[m] == 0) wb |= 1u << m;
    }
#pragma unroll 1
    for (int hop = first; hop < 8; ++hop) {
        const int mu = hop >> 1;
        const bool fwd = (hop & 1) == 0;
        const int L = g.L[mu], st = g.stride[mu];
        const bool wrap = ((fwd ? wf : wb) >> mu) & 1u;
        const int y = wc_idx(fwd ? (wrap ? x - (L - 1) * st : x + st) : (wrap ? x + (L - 1) * st : x - st), g.V);
        cx<R> p[12], h[6], u[6], r2[3], w[6];
        const R scale = P::load_spinor_raw(in, in_nrm, Vin, sidx(y), p);
        const R coef = ((mu == 3 && wrap) ? k * R(g.tbc) : k) * scale;
        const int s = fwd ? SF : -SF;
        project_rt(mu, s, p, h);
        P::load_link(U, g.V, mu, fwd ? x : y, u, r2);
        su3_mul_rt(!fwd, u, r2, h, coef, w);
        reconstruct_add_rt(mu, s, acc, w);
    }
}

// y = A v for clover block b of the packed store (rows in a runtime loop;
// each row reads its six entries: diagonal, lower (i, j) and the conjugate
// of lower (j, i))
template <class P>
__device__ __forceinline__ void clover_block_rt(const CloverStore &C, int V, int x, int b,
                                                const cx<typename P::real> v[6], cx<typename P::real> y[6])
{
    using R = typename P::real;
#pragma unroll 1
    for (int i = 0; i < 6; ++i) {
        cx<R> acc = mkc(R(0.0f, 0.0f), R(0.0f, 0.0f));
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            cx<R> e;
            if (j == i) {
                e = cx<R>{P::clover_real(C, V, x, b, i), R(0.0f, 0.0f)};
            } else {
                const int hi = i > j ? i : j, lo = i > j ? j : i;
                const cx<R> l = P::clover_lower(C, V, x, b, hi * (hi - 1) / 2 + lo);
                e = j < i ? l : conj(l);
            }
            acc = cfma(e, v[j], acc);
        }
#pragma unroll
        for (int r = 0; r < 6; ++r)
            if (r == i) y[r] = acc;
    }
}

// ---- one site of the operator ------------------------------------------
// Shared by the whole-lattice operator kernels and the interior kernel of
// the domain-decomposed operator, so that both compute a site with the same
// arithmetic in the same order.

template <class P, int MU, int SF, int SB>
__device__ __forceinline__ void hop_dir(const Geom &g, const GaugeStore &U, const void *in, const float *in_nrm,
                                        int x, const int c[4], typename P::real k, cx<typename P::real> acc[12])
{
    using R = typename P::real;
    const int L = g.L[MU], st = g.stride[MU];
    {
        const bool wrap = c[MU] == L - 1;
        const int xf = wc_idx(wrap ? x - (L - 1) * st : x + st, g.V);
        cx<R> p[12], h[6], u[6], r2[3], w[6];
        const R scale = P::load_spinor_raw(in, in_nrm, g.V, xf, p);
        const R coef = ((MU == 3 && wrap) ? k * R(g.tbc) : k) * scale;
        project<MU, SF>(p, h);
        P::load_link(U, g.V, MU, x, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(acc, w);
    }
    {
        const bool wrap = c[MU] == 0;
        const int xb = wc_idx(wrap ? x + (L - 1) * st : x - st, g.V);
        cx<R> p[12], h[6], u[6], r2[3], w[6];
        const R scale = P::load_spinor_raw(in, in_nrm, g.V, xb, p);
        const R coef = ((MU == 3 && wrap) ? k * R(g.tbc) : k) * scale;
        project<MU, SB>(p, h);
        P::load_link(U, g.V, MU, xb, u, r2);
        su3_adj_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SB>(acc, w);
    }
}

// ---- FP16 storage: products and sums formed from the stored halves ------
// With FP16 storage the clover entries, the centre spinor and the
// neighbour spinors are binary16 values: fma.f32.f16 forms a product of
// two of them exactly (11 x 11 significand bits fit in FP32) and adds it in
// FP32 with one rounding -- the result of converting both to FP32 and using
// an FP32 fma, without the conversion instructions (the FP16 operator is
// bound by instruction issue).

__device__ __forceinline__ float fma_h(unsigned short a, unsigned short b, float c)
{
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
    return d;
}

__device__ __forceinline__ unsigned short lo16(unsigned w) { return (unsigned short)(w & 0xffffu); }
__device__ __forceinline__ unsigned short hi16(unsigned w) { return (unsigned short)(w >> 16); }

// y = B v for clover block b (FP16 store, site x) and the unscaled FP16
// centre spinor components v (half2 words (re, im), spins 2b, 2b + 1)
__device__ __forceinline__ void clover_block_h(const CloverStore &C, int V, int x, int b, const unsigned v[6],
                                               cx<float> y[6])
{
    unsigned short vr[6], vi[6], nvr[6], nvi[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        vr[i] = lo16(v[i]);
        vi[i] = hi16(v[i]);
        nvr[i] = vr[i] ^ 0x8000u;
        nvi[i] = vi[i] ^ 0x8000u;
    }
    const uint4 *p = C.c16 + x;
    auto entry = [&](int q) {   // half2 word q (0..17) of block b
        const int gq = 18 * b + q;
        const uint4 w = __ldg(p + (size_t)(gq >> 2) * V);
        return (gq & 3) == 0 ? w.x : ((gq & 3) == 1 ? w.y : ((gq & 3) == 2 ? w.z : w.w));
    };
#pragma unroll
    for (int q = 0; q < 3; ++q) {   // diagonal reals 2q, 2q + 1
        const unsigned d = entry(q);
        y[2 * q] = mkc(fma_h(lo16(d), vr[2 * q], 0.f), fma_h(lo16(d), vi[2 * q], 0.f));
        y[2 * q + 1] = mkc(fma_h(hi16(d), vr[2 * q + 1], 0.f), fma_h(hi16(d), vi[2 * q + 1], 0.f));
    }
    int k = 3;
#pragma unroll
    for (int a = 1; a < 6; ++a) {
#pragma unroll
        for (int c = 0; c < a; ++c) {
            const unsigned l = entry(k++);
            const unsigned short lr = lo16(l), li = hi16(l);
            // y[a] += l v[c]; y[c] += conj(l) v[a]
            y[a].re = fma_h(lr, vr[c], fma_h(li, nvi[c], y[a].re));
            y[a].im = fma_h(lr, vi[c], fma_h(li, vr[c], y[a].im));
            y[c].re = fma_h(lr, vr[a], fma_h(li, vi[a], y[c].re));
            y[c].im = fma_h(lr, vi[a], fma_h(li, nvr[a], y[c].im));
        }
    }
}

// a + S b for binary16 a, b, exactly rounded to FP32 (the FP32 sum of the
// two converted values); S = +-1
template <int S>
__device__ __forceinline__ float add_hh(unsigned short a, unsigned short b)
{
    const unsigned short one = 0x3c00u, s_one = S > 0 ? 0x3c00u : 0xbc00u;
    return fma_h(a, one, fma_h(b, s_one, 0.f));
}

// two-spinor of (1 + S gamma_MU) psi from the packed FP16 spinor words
// w[k] (component k = 3 spin + colour as half2 (re, im)), unscaled
template <int MU, int S>
__device__ __forceinline__ void project_h16(const unsigned w[12], cx<float> h[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const unsigned u0 = w[c], u1 = w[3 + c], d0 = w[6 + c], d1 = w[9 + c];
        if (MU == 0) {   // h0 = u0 + S i d1, h1 = u1 + S i d0
            h[c] = mkc(add_hh<-S>(lo16(u0), hi16(d1)), add_hh<S>(hi16(u0), lo16(d1)));
            h[3 + c] = mkc(add_hh<-S>(lo16(u1), hi16(d0)), add_hh<S>(hi16(u1), lo16(d0)));
        } else if (MU == 1) {   // h0 = u0 + S d1, h1 = u1 - S d0
            h[c] = mkc(add_hh<S>(lo16(u0), lo16(d1)), add_hh<S>(hi16(u0), hi16(d1)));
            h[3 + c] = mkc(add_hh<-S>(lo16(u1), lo16(d0)), add_hh<-S>(hi16(u1), hi16(d0)));
        } else if (MU == 2) {   // h0 = u0 + S i d0, h1 = u1 - S i d1
            h[c] = mkc(add_hh<-S>(lo16(u0), hi16(d0)), add_hh<S>(hi16(u0), lo16(d0)));
            h[3 + c] = mkc(add_hh<S>(lo16(u1), hi16(d1)), add_hh<-S>(hi16(u1), lo16(d1)));
        } else {   // h0 = u0 + S d0, h1 = u1 + S d1
            h[c] = mkc(add_hh<S>(lo16(u0), lo16(d0)), add_hh<S>(hi16(u0), hi16(d0)));
            h[3 + c] = mkc(add_hh<S>(lo16(u1), lo16(d1)), add_hh<S>(hi16(u1), hi16(d1)));
        }
    }
}

// acc += coef * (reconstruction of the two-spinor w), the coefficient
// folded into the accumulation (reconstruct_add of coef w without forming
// coef w)
template <int MU, int S>
__device__ __forceinline__ void reconstruct_fma(cx<float> acc[12], const cx<float> w[6], float coef)
{
    const float sc = S > 0 ? coef : -coef;   // S coef
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<float> w0 = w[c], w1 = w[3 + c];
        acc[c] = mkc(fmaf(coef, w0.re, acc[c].re), fmaf(coef, w0.im, acc[c].im));
        acc[3 + c] = mkc(fmaf(coef, w1.re, acc[3 + c].re), fmaf(coef, w1.im, acc[3 + c].im));
        if (MU == 0) {   // acc[6+c] -= S i w1, acc[9+c] -= S i w0
            acc[6 + c] = mkc(fmaf(sc, w1.im, acc[6 + c].re), fmaf(-sc, w1.re, acc[6 + c].im));
            acc[9 + c] = mkc(fmaf(sc, w0.im, acc[9 + c].re), fmaf(-sc, w0.re, acc[9 + c].im));
        } else if (MU == 1) {   // acc[6+c] -= S w1, acc[9+c] += S w0
            acc[6 + c] = mkc(fmaf(-sc, w1.re, acc[6 + c].re), fmaf(-sc, w1.im, acc[6 + c].im));
            acc[9 + c] = mkc(fmaf(sc, w0.re, acc[9 + c].re), fmaf(sc, w0.im, acc[9 + c].im));
        } else if (MU == 2) {   // acc[6+c] -= S i w0, acc[9+c] += S i w1
            acc[6 + c] = mkc(fmaf(sc, w0.im, acc[6 + c].re), fmaf(-sc, w0.re, acc[6 + c].im));
            acc[9 + c] = mkc(fmaf(-sc, w1.im, acc[9 + c].re), fmaf(sc, w1.re, acc[9 + c].im));
        } else {   // acc[6+c] += S w0, acc[9+c] += S w1
            acc[6 + c] = mkc(fmaf(sc, w0.re, acc[6 + c].re), fmaf(sc, w0.im, acc[6 + c].im));
            acc[9 + c] = mkc(fmaf(sc, w1.re, acc[9 + c].re), fmaf(sc, w1.im, acc[9 + c].im));
        }
    }
}

// the forward and backward hop of direction MU for FP16 storage (hop_dir
// with the projection formed from the stored halves and the coefficient
// folded into the accumulation)
template <int MU, int SF, int SB>
__device__ __forceinline__ void hop_dir_h16(const Geom &g, const GaugeStore &U, const void *in, const float *in_nrm,
                                            int x, const int c[4], float k, cx<float> acc[12])
{
    const int L = g.L[MU], st = g.stride[MU];
    const uint4 *ps = static_cast<const uint4 *>(in);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        const bool wrap = dir == 0 ? c[MU] == L - 1 : c[MU] == 0;
        const int y = wc_idx(dir == 0 ? (wrap ? x - (L - 1) * st : x + st) : (wrap ? x + (L - 1) * st : x - st), g.V);
        const uint4 s0 = __ldg(ps + y), s1 = __ldg(ps + (size_t)g.V + y), s2 = __ldg(ps + 2 * (size_t)g.V + y);
        const unsigned w[12] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w, s2.x, s2.y, s2.z, s2.w};
        const float coef = ((MU == 3 && wrap) ? k * (float)g.tbc : k) * __ldg(in_nrm + y);
        cx<float> h[6], u[6], r2[3], wv[6];
        if (dir == 0) {
            project_h16<MU, SF>(w, h);
            P16::load_link(U, g.V, MU, x, u, r2);
            su3_mul(u, r2, h, 1.0f, wv);
            reconstruct_fma<MU, SF>(acc, wv, coef);
        } else {
            project_h16<MU, SB>(w, h);
            P16::load_link(U, g.V, MU, y, u, r2);
            su3_adj_mul(u, r2, h, 1.0f, wv);
            reconstruct_fma<MU, SB>(acc, wv, coef);
        }
    }
}

// One site: out(x) = M in, M^+ in or H in (KIND 0, 1, 2) for the site of
// this thread in logical block blk.
template <class P, int KIND>
__device__ __forceinline__ void apply_site_at(const Geom &g, int x, const GaugeStore &U, const CloverStore &C,
                                              const void *in, const float *in_nrm, void *out, float *out_nrm,
                                              double kappa)
{
    using R = typename P::real;
    x = wc_idx(x, g.V);
    int c[4];
    if constexpr (std::is_same<P, P16>::value)
        site_coords_fast(g, x, c);
    else
        site_coords(g, x, c);
    cx<R> acc[12];
    if constexpr (std::is_same<P, PDF>::value) {
        // Six hops (directions y, z, t) in double-FP32 on the FP32 pipes, in
        // the compact form (the instruction cache); the clover term and the
        // two x hops in FP64 on the FP64 pipe, which the double-FP32 work of
        // the other warps leaves idle.
        constexpr int SF = KIND == 1 ? +1 : -1;
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = mkc(R(0.0f, 0.0f), R(0.0f, 0.0f));
        const R k = KIND == 2 ? R(1.0) : R(-kappa);
        hops_rt<P, SF>(g, U, in, in_nrm, g.V, x, c, k, acc, [](int y) { return y; }, 2);
        cx<double> ad[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) ad[q] = mkc(df_to_double(acc[q].re), df_to_double(acc[q].im));
        hop_dir<P64, 0, SF, -SF>(g, U, in, in_nrm, x, c, KIND == 2 ? 1.0 : -kappa, ad);
        if (KIND == 2) {
            P64::store_spinor(out, out_nrm, g.V, x, ad);
            return;
        }
        cx<double> pd[12];
        P64::load_spinor(in, nullptr, g.V, x, pd);
#pragma unroll 1
        for (int b = 0; b < 2; ++b) {
            double r[36];
            cx<double> v6[6], y6[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) v6[q] = b ? pd[6 + q] : pd[q];
            P64::load_clover(C, g.V, x, b, r);
            clover_block_mul(r, v6, y6);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                if (b) ad[6 + q] = ad[6 + q] + y6[q];
                else ad[q] = ad[q] + y6[q];
            }
        }
        P64::store_spinor(out, out_nrm, g.V, x, ad);
        return;
    }
    if (KIND == 2) {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = mkc(R(0), R(0));
    } else if constexpr (std::is_same<P, P16>::value) {
        // clover products from the stored halves, the centre scale applied
        // once to the result
        const uint4 *ps = static_cast<const uint4 *>(in);
        const uint4 s0 = __ldg(ps + x), s1 = __ldg(ps + (size_t)g.V + x), s2 = __ldg(ps + 2 * (size_t)g.V + x);
        const float sc = __ldg(in_nrm + x);
        const unsigned v0[6] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y};
        const unsigned v1[6] = {s1.z, s1.w, s2.x, s2.y, s2.z, s2.w};
        clover_block_h(C, g.V, x, 0, v0, acc);
        clover_block_h(C, g.V, x, 1, v1, acc + 6);
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = sc * acc[q];
    } else {
        cx<R> p[12];
        P::load_spinor(in, in_nrm, g.V, x, p);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            R r[36];
            P::load_clover(C, g.V, x, b, r);
            clover_block_mul(r, p + 6 * b, acc + 6 * b);
        }
    }
    const R k = KIND == 2 ? R(1) : R(-kappa);
    constexpr int SF = KIND == 1 ? +1 : -1;
    constexpr int SB = -SF;
    if constexpr (std::is_same<P, P16>::value) {
        hop_dir_h16<0, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
        hop_dir_h16<1, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
        hop_dir_h16<2, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
        hop_dir_h16<3, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
    } else {
        hop_dir<P, 0, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
        hop_dir<P, 1, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
        hop_dir<P, 2, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
        hop_dir<P, 3, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
    }
    P::store_spinor(out, out_nrm, g.V, x, acc);
}

}  // namespace wc
