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

#include "wc_internal.cuh"

namespace wc {

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
        const R s = R(S);
        if (MU == 0) {
            h[c] = u0 + s * times_i(d1);
            h[3 + c] = u1 + s * times_i(d0);
        } else if (MU == 1) {
            h[c] = u0 + s * d1;
            h[3 + c] = u1 - s * d0;
        } else if (MU == 2) {
            h[c] = u0 + s * times_i(d0);
            h[3 + c] = u1 - s * times_i(d1);
        } else {
            h[c] = u0 + s * d0;
            h[3 + c] = u1 + s * d1;
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
        const R s = R(S);
        acc[c] = acc[c] + w0;
        acc[3 + c] = acc[3 + c] + w1;
        if (MU == 0) {
            acc[6 + c] = acc[6 + c] - s * times_i(w1);
            acc[9 + c] = acc[9 + c] - s * times_i(w0);
        } else if (MU == 1) {
            acc[6 + c] = acc[6 + c] - s * w1;
            acc[9 + c] = acc[9 + c] + s * w0;
        } else if (MU == 2) {
            acc[6 + c] = acc[6 + c] - s * times_i(w0);
            acc[9 + c] = acc[9 + c] + s * times_i(w1);
        } else {
            acc[6 + c] = acc[6 + c] + s * w0;
            acc[9 + c] = acc[9 + c] + s * w1;
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
