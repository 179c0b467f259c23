// Wilson-Clover operator kernels: out = M in, M^+ in, H in; field casts.
//
// One thread per site, lexicographic site order (so the neighbour loads of a
// warp are contiguous in every direction and the 8-fold reuse of each input
// spinor is served by L1/L2).  Per direction the neighbour spinor is spin
// projected to a two-spinor before the SU(3) multiply, halving the matvec
// work (paper Sec. 2/3, the hopping multiplication "MULT"); links are read as
// two rows and the third rebuilt in registers (SU(3) reconstruction).  The
// clover term (two packed Hermitian 6x6 blocks) is applied to the centre
// spinor first and the hops are accumulated into that result with the
// coefficient -kappa, so out = (1 + T) in - kappa H in is written once.
//
#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

constexpr int kApplyBlock = 128;

template <class P, int MU, int SF, int SB>
__device__ __forceinline__ void hop_dir(const Geom &g, const GaugeStore &U, const void *in, const float *in_nrm,
                                        int x, const int c[4], typename P::real k, cx<typename P::real> acc[12])
{
    using R = typename P::real;
    const int L = g.L[MU], st = g.stride[MU];
    {
        const bool wrap = c[MU] == L - 1;
        const int xf = wrap ? x - (L - 1) * st : x + st;
        const R coef = (MU == 3 && wrap) ? k * R(g.tbc) : k;
        cx<R> p[12], h[6], u[6], r2[3], w[6];
        P::load_spinor(in, in_nrm, g.V, xf, p);
        project<MU, SF>(p, h);
        P::load_link(U, g.V, MU, x, u);
        reconstruct_row2(u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(acc, w);
    }
    {
        const bool wrap = c[MU] == 0;
        const int xb = wrap ? x + (L - 1) * st : x - st;
        const R coef = (MU == 3 && wrap) ? k * R(g.tbc) : k;
        cx<R> p[12], h[6], u[6], r2[3], w[6];
        P::load_spinor(in, in_nrm, g.V, xb, p);
        project<MU, SB>(p, h);
        P::load_link(U, g.V, MU, xb, u);
        reconstruct_row2(u, r2);
        su3_adj_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SB>(acc, w);
    }
}

// KIND 0: out = M in, 1: out = M^+ in, 2: out = H in
template <class P, int KIND>
__global__ void __launch_bounds__(kApplyBlock) k_apply(Geom g, GaugeStore U, CloverStore C, const void *in,
                                                       const float *in_nrm, void *out, float *out_nrm,
                                                       double kappa)
{
    using R = typename P::real;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    int c[4];
    site_coords(g, x, c);
    cx<R> acc[12];
    if (KIND == 2) {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = mkc(R(0), R(0));
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
    hop_dir<P, 0, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
    hop_dir<P, 1, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
    hop_dir<P, 2, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
    hop_dir<P, 3, SF, SB>(g, U, in, in_nrm, x, c, k, acc);
    P::store_spinor(out, out_nrm, g.V, x, acc);
}

template <class P>
cudaError_t launch_apply_p(wc_lattice lat, wc_field out, wc_field in, int kind, cudaStream_t stream)
{
    const int V = lat->g.V;
    dim3 grid((V + kApplyBlock - 1) / kApplyBlock), block(kApplyBlock);
    if (kind == 0)
        k_apply<P, 0><<<grid, block, 0, stream>>>(lat->g, lat->gauge, lat->clover, in->data, in->nrm,
                                                       out->data, out->nrm, lat->kappa);
    else if (kind == 1)
        k_apply<P, 1><<<grid, block, 0, stream>>>(lat->g, lat->gauge, lat->clover, in->data, in->nrm,
                                                       out->data, out->nrm, lat->kappa);
    else
        k_apply<P, 2><<<grid, block, 0, stream>>>(lat->g, lat->gauge, lat->clover, in->data, in->nrm,
                                                       out->data, out->nrm, lat->kappa);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// precision conversion / scaling: dst = scale * src
// ------------------------------------------------------------------------

template <class PS, class PD>
__global__ void k_copy(int V, const void *src, const float *src_nrm, void *dst, float *dst_nrm, double scale,
                       const double *dev_norm2, int invert)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    double sc = scale;
    if (dev_norm2) {
        const double n2 = *dev_norm2;
        const double n = sqrt(n2);
        sc *= invert ? (n > 0.0 ? 1.0 / n : 0.0) : n;
    }
    cx<typename PS::real> a[12];
    PS::load_spinor(src, src_nrm, V, x, a);
    cx<typename PD::real> b[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        // scale in the wider of the two precisions, then round once
        const double re = sc * (double)a[k].re, im = sc * (double)a[k].im;
        b[k] = mkc((typename PD::real)re, (typename PD::real)im);
    }
    PD::store_spinor(dst, dst_nrm, V, x, b);
}

template <class PS>
cudaError_t launch_copy_s(wc_lattice lat, wc_field dst, wc_field src, double scale, const double *dn, int inv,
                          cudaStream_t stream)
{
    const int V = lat->g.V;
    dim3 grid((V + 255) / 256), block(256);
    switch (dst->prec) {
    case WC_F64:
        k_copy<PS, P64><<<grid, block, 0, stream>>>(V, src->data, src->nrm, dst->data, dst->nrm, scale, dn, inv);
        break;
    case WC_F32:
        k_copy<PS, P32><<<grid, block, 0, stream>>>(V, src->data, src->nrm, dst->data, dst->nrm, scale, dn, inv);
        break;
    default:
        k_copy<PS, P16><<<grid, block, 0, stream>>>(V, src->data, src->nrm, dst->data, dst->nrm, scale, dn, inv);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply(wc_lattice lat, wc_field out, wc_field in, int kind, cudaStream_t stream)
{
    switch (in->prec) {
    case WC_F64: return launch_apply_p<P64>(lat, out, in, kind, stream);
    case WC_F32: return launch_apply_p<P32>(lat, out, in, kind, stream);
    default: return launch_apply_p<P16>(lat, out, in, kind, stream);
    }
}

cudaError_t launch_copy(wc_lattice lat, wc_field dst, wc_field src, double scale, const double *dev_scale,
                        int invert_scale, cudaStream_t stream)
{
    switch (src->prec) {
    case WC_F64: return launch_copy_s<P64>(lat, dst, src, scale, dev_scale, invert_scale, stream);
    case WC_F32: return launch_copy_s<P32>(lat, dst, src, scale, dev_scale, invert_scale, stream);
    default: return launch_copy_s<P16>(lat, dst, src, scale, dev_scale, invert_scale, stream);
    }
}

}  // namespace wc
