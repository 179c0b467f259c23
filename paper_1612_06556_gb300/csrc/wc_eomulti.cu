// Multi-right-hand-side even-odd (Schur complement) operator:
//   out_r = M^ in_r = A_ee in_r - kappa^2 H_eo A_oo^-1 H_oe in_r   (or M^+)
// for up to kMrhsMax half-lattice fields of one lattice, in two launches
// (odd-site pass, even-site pass) that serve every right-hand side.
//
// The right-hand sides of a propagator share the gauge field, A and A^-1.
// In one pass a site reads its 8 links (4 forward U_mu(x), 4 backward
// U_mu(x - mu)) and one clover-type block (A^-1 on the odd pass, A on the
// even pass): 672 B per site in FP32, 336 B in FP16 storage, against 96 /
// 52 B per spinor read or written.  A CTA covers kEoMSites consecutive
// sites of one parity for all n right-hand sides: it stages those shared
// words once in shared memory (coalesced along the sites), then thread
// (s, r) computes site s of right-hand side r from the staged links and
// block and the 8 neighbour spinors of field r (through L1/L2).  The third
// row of each link is rebuilt once per site after staging (into shared
// memory), not once per right-hand side.  The arithmetic per (site,
// right-hand side) is otherwise that of the single-field pass (spin
// projection, the block product, beta = -kappa^2 on the even pass).  Per-field device flags (the
// skip word of a lockstep batch's solver scalars) may skip fields.
#include <string>
#include <type_traits>
#include <vector>

#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

constexpr int kEoMSites = 32;

struct EoMultiArgs {
    int n;
    const void *hin[kMrhsMax];     // hop input (opposite parity)
    const float *hin_nrm[kMrhsMax];
    const void *vin[kMrhsMax];     // site input (even pass)
    const float *vin_nrm[kMrhsMax];
    void *out[kMrhsMax];
    float *out_nrm[kMrhsMax];
    const int *skip[kMrhsMax];     // nullable: *skip[r] != 0 skips right-hand side r
    // even pass only: partial sums of field r for the solver step that
    // follows, per CTA, written to part[(r * gridDim.x + blockIdx.x) * 4 + c]:
    // red 1: <dot[r], out> (c = 0, 1: real, imaginary part); red 2: <out, vin>,
    // |out|^2, |vin|^2.  FP32 fields only.
    int red;
    const void *dot[kMrhsMax];
    double *part;
};

// the staged words of one site: 4 forward and 4 backward links, the block
template <class P>
struct EoMStage;

template <>
struct EoMStage<P32> {
    using W = float4;
    static constexpr int kWords = 24 + 18;   // links [fwd/bwd][mu][3], block [18]
    static __device__ __forceinline__ W link_word(const GaugeStore &U, int V, int mu, int x, int j)
    {
        return __ldg(U.u32 + ((size_t)mu * 3 + j) * V + x);
    }
    static __device__ __forceinline__ W block_word(const CloverStore &C, int V, int pos, int q)
    {
        return __ldg(C.c32 + (size_t)q * V + pos);
    }
    static __device__ __forceinline__ void stage(const GaugeStore &U, const CloverStore &C, int V, int item, int x,
                                                 int xb_mu[4], int pos, W &out)
    {
        if (item < 12)
            out = link_word(U, V, item / 3, x, item % 3);
        else if (item < 24)
            out = link_word(U, V, (item - 12) / 3, xb_mu[(item - 12) / 3], (item - 12) % 3);
        else
            out = block_word(C, V, pos, item - 24);
    }
    // the two stored rows of link lam = 4 bwd + mu
    static __device__ __forceinline__ void rows(const W (*st)[kEoMSites], int s, int lam, cx<float> a[6])
    {
        const int base = (lam >= 4 ? 12 : 0) + 3 * (lam & 3);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float4 v = st[base + j][s];
            a[2 * j] = mkc(v.x, v.y);
            a[2 * j + 1] = mkc(v.z, v.w);
        }
    }
    static __device__ __forceinline__ void block(const W (*st)[kEoMSites], int s, int b, float r[36])
    {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float4 v = st[24 + 9 * b + q][s];
            r[4 * q] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        }
    }
};

template <>
struct EoMStage<P16> {
    using W = uint4;
    // links: [fwd/bwd][mu] as (uint4 row 0 + entry (1,0)) then the uint2
    // (entries (1,1), (1,2)) of two directions per word; block [9]
    static constexpr int kWords = 8 + 4 + 9;
    static __device__ __forceinline__ void stage(const GaugeStore &U, const CloverStore &C, int V, int item, int x,
                                                 int xb_mu[4], int pos, W &out)
    {
        if (item < 8) {
            const int mu = item & 3, y = item < 4 ? x : xb_mu[mu];
            out = __ldg(U.u16a + (size_t)mu * V + y);
        } else if (item < 12) {
            const int k = item - 8;   // words of (fwd mu 0,1), (fwd 2,3), (bwd 0,1), (bwd 2,3)
            const bool bwd = k >= 2;
            const int mu0 = 2 * (k & 1);
            const uint2 a = __ldg(U.u16b + (size_t)mu0 * V + (bwd ? xb_mu[mu0] : x));
            const uint2 b = __ldg(U.u16b + (size_t)(mu0 + 1) * V + (bwd ? xb_mu[mu0 + 1] : x));
            out = make_uint4(a.x, a.y, b.x, b.y);
        } else {
            out = __ldg(C.c16 + (size_t)(item - 12) * V + pos);
        }
    }
    static __device__ __forceinline__ void rows(const W (*st)[kEoMSites], int s, int lam, cx<float> a[6])
    {
        const int mu = lam & 3;
        const bool bwd = lam >= 4;
        const uint4 v = st[(bwd ? 4 : 0) + mu][s];
        const uint4 w = st[8 + (bwd ? 2 : 0) + (mu >> 1)][s];
        a[0] = h2c(v.x);
        a[1] = h2c(v.y);
        a[2] = h2c(v.z);
        a[3] = h2c(v.w);
        a[4] = h2c((mu & 1) ? w.z : w.x);
        a[5] = h2c((mu & 1) ? w.w : w.y);
    }
    static __device__ __forceinline__ void block(const W (*st)[kEoMSites], int s, int b, float r[36])
    {
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const int q = 18 * b + k;   // half2 index among the 36 of a site
            const uint4 v = st[12 + (q >> 2)][s];
            const unsigned w = (q & 3) == 0 ? v.x : (q & 3) == 1 ? v.y : (q & 3) == 2 ? v.z : v.w;
            const cx<float> f = h2c(w);
            r[2 * k] = f.re;
            r[2 * k + 1] = f.im;
        }
    }
};

// the two hops of direction MU of site x (full index, coordinates c) of the
// half field `in` (opposite parity), links from the stage
// link lam (mu, or 4 + mu for U_mu(x - mu)) of site s from the stage: the
// two stored rows and the third row rebuilt once per site at staging
template <class P>
__device__ __forceinline__ void eom_link(const typename EoMStage<P>::W (*st)[kEoMSites],
                                         const float2 (*r3)[3][kEoMSites], int s, int lam, cx<float> a[6],
                                         cx<float> c[3])
{
    EoMStage<P>::rows(st, s, lam, a);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float2 v = r3[lam][j][s];
        c[j] = mkc(v.x, v.y);
    }
}

template <class P, int MU, int SF, int SB>
__device__ __forceinline__ void eom_hops(const Geom &g, const typename EoMStage<P>::W (*st)[kEoMSites],
                                        const float2 (*r3)[3][kEoMSites], int s, const void *in,
                                        const float *in_nrm, int Vh, int x, const int c[4], cx<float> acc[12])
{
    const int L = g.L[MU], stride = g.stride[MU];
    {
        const bool wrap = c[MU] == L - 1;
        const int xf = wc_idx(wrap ? x - (L - 1) * stride : x + stride, g.V);
        cx<float> p[12], h[6], u[6], r2[3], w[6];
        const float scale = P::load_spinor_raw(in, in_nrm, Vh, xf >> 1, p);
        const float coef = ((MU == 3 && wrap) ? (float)g.tbc : 1.f) * scale;
        project<MU, SF>(p, h);
        eom_link<P>(st, r3, s, MU, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(acc, w);
    }
    {
        const bool wrap = c[MU] == 0;
        const int xb = wc_idx(wrap ? x + (L - 1) * stride : x - stride, g.V);
        cx<float> p[12], h[6], u[6], r2[3], w[6];
        const float scale = P::load_spinor_raw(in, in_nrm, Vh, xb >> 1, p);
        const float coef = ((MU == 3 && wrap) ? (float)g.tbc : 1.f) * scale;
        project<MU, SB>(p, h);
        eom_link<P>(st, r3, s, 4 + MU, u, r2);
        su3_adj_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SB>(acc, w);
    }
}

// full index and coordinates of half index i of parity p (all extents
// even): 2i is the full index of the site with x rounded down to even
__device__ __forceinline__ int eom_full_site(const Geom &g, int i, int p, int c[4])
{
    site_coords_fast(g, 2 * i, c);
    const int bit = (p + c[1] + c[2] + c[3]) & 1;
    c[0] += bit;
    return wc_idx(2 * i + bit, g.V);
}

// MODE 0 (odd pass): out_r = Blk H hin_r      (Blk = A^-1)
// MODE 1 (even pass): out_r = Blk vin_r + beta H hin_r   (Blk = A)
template <class P, int DAG, int MODE>
__global__ void __maxnreg__(80) k_eo_multi(Geom g, int p, GaugeStore U, CloverStore Blk,
                                                                   const __grid_constant__ EoMultiArgs a,
                                                                   double beta)
{
    using W = typename EoMStage<P>::W;
    constexpr int NW = EoMStage<P>::kWords;
    __shared__ W st[NW][kEoMSites];
    __shared__ float2 r3[8][3][kEoMSites];   // third rows of the 8 links
    const int Vh = g.V >> 1;
    const int i0 = blockIdx.x * kEoMSites;
    // blockDim is a multiple of kEoMSites: a thread stages and computes the
    // same site s
    const int s = threadIdx.x % kEoMSites, r = threadIdx.x / kEoMSites, i = i0 + s;
    int c[4] = {0, 0, 0, 0}, x = 0;
    if (i < Vh) {
        x = eom_full_site(g, i, p, c);
        int xb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
            xb[mu] = wc_idx(c[mu] == 0 ? x + (g.L[mu] - 1) * g.stride[mu] : x - g.stride[mu], g.V);
        const int pos = wc_idx(p * Vh + i, g.V);
        for (int item = r; item < NW; item += blockDim.x / kEoMSites)
            EoMStage<P>::stage(U, Blk, g.V, item, x, xb, pos, st[item][s]);
    }
    __syncthreads();
    // the third row of every staged link, once per site
    for (int q = threadIdx.x; q < 8 * kEoMSites; q += blockDim.x) {
        const int ss = q % kEoMSites, lam = q / kEoMSites;
        if (i0 + ss >= Vh) continue;
        cx<float> u[6], c3[3];
        EoMStage<P>::rows(st, ss, lam, u);
        reconstruct_row2(u, c3);
#pragma unroll
        for (int j = 0; j < 3; ++j) r3[lam][j][ss] = make_float2(c3[j].re, c3[j].im);
    }
    __syncthreads();
    if (r >= a.n) return;
    if (a.skip[r] && *a.skip[r]) return;   // the whole warp: one field per warp
    float red[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < Vh) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    cx<float> h[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) h[k] = mkc(0.f, 0.f);
    eom_hops<P, 0, SF, SB>(g, st, r3, s, a.hin[r], a.hin_nrm[r], Vh, x, c, h);
    eom_hops<P, 1, SF, SB>(g, st, r3, s, a.hin[r], a.hin_nrm[r], Vh, x, c, h);
    eom_hops<P, 2, SF, SB>(g, st, r3, s, a.hin[r], a.hin_nrm[r], Vh, x, c, h);
    eom_hops<P, 3, SF, SB>(g, st, r3, s, a.hin[r], a.hin_nrm[r], Vh, x, c, h);
    cx<float> v[12], o[12];
    const float bt = (float)beta;
    if (MODE == 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = h[k];
    } else {
        P::load_spinor(a.vin[r], a.vin_nrm[r], Vh, i, v);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        float blk[36];
        EoMStage<P>::block(st, s, b, blk);
        clover_block_mul(blk, v + 6 * b, o + 6 * b);
    }
    if (MODE == 1)
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = o[k] + bt * h[k];
    P::store_spinor(a.out[r], a.out_nrm[r], Vh, i, o);
    if (MODE == 1 && a.red == 1) {
        cx<float> d[12];
        P32::load_spinor(a.dot[r], nullptr, Vh, i, d);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            red[0] = fmaf(d[k].re, o[k].re, fmaf(d[k].im, o[k].im, red[0]));
            red[1] = fmaf(d[k].re, o[k].im, fmaf(-d[k].im, o[k].re, red[1]));
        }
    } else if (MODE == 1 && a.red == 2) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            red[0] = fmaf(o[k].re, v[k].re, fmaf(o[k].im, v[k].im, red[0]));
            red[1] = fmaf(o[k].re, v[k].im, fmaf(-o[k].im, v[k].re, red[1]));
            red[2] = fmaf(o[k].re, o[k].re, fmaf(o[k].im, o[k].im, red[2]));
            red[3] = fmaf(v[k].re, v[k].re, fmaf(v[k].im, v[k].im, red[3]));
        }
    }
    }   // i < Vh
    if (MODE == 1 && a.red != 0) {
        // the warp holds the 32 sites of this CTA for field r
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) red[c] += __shfl_xor_sync(0xffffffffu, red[c], o2);
        if (s == 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) a.part[((size_t)r * gridDim.x + blockIdx.x) * 4 + c] = (double)red[c];
    }
}

template <class P, int DAG>
cudaError_t launch_eom(const wc_lattice_s *full, int n, wc_field const *outs, wc_field const *ins,
                       wc_field const *tmps, const int *const *skip, int red, wc_field const *dots, double *part,
                       cudaStream_t stream)
{
    const int Vh = full->g.V >> 1;
    const dim3 grid((Vh + kEoMSites - 1) / kEoMSites), block(kEoMSites * n);
    EoMultiArgs a{};
    a.n = n;
    for (int r = 0; r < n; ++r) {
        a.skip[r] = skip ? skip[r] : nullptr;
        a.hin[r] = ins[r]->data;
        a.hin_nrm[r] = ins[r]->nrm;
        a.out[r] = tmps[r]->data;
        a.out_nrm[r] = tmps[r]->nrm;
    }
    // odd sites: tmp = A_oo^-1 H_oe in
    k_eo_multi<P, DAG, 0><<<grid, block, 0, stream>>>(full->g, 1, full->gauge, full->cinv, a, 0.0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // even sites: out = A_ee in - kappa^2 H_eo tmp
    for (int r = 0; r < n; ++r) {
        a.hin[r] = tmps[r]->data;
        a.hin_nrm[r] = tmps[r]->nrm;
        a.vin[r] = ins[r]->data;
        a.vin_nrm[r] = ins[r]->nrm;
        a.out[r] = outs[r]->data;
        a.out_nrm[r] = outs[r]->nrm;
    }
    a.red = red;
    a.part = part;
    for (int r = 0; r < n && red == 1; ++r) a.dot[r] = dots[r]->data;
    k_eo_multi<P, DAG, 1><<<grid, block, 0, stream>>>(full->g, 0, full->gauge, full->ceo, a,
                                                      -full->kappa * full->kappa);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_schur_multi(wc_lattice half, int n, wc_field const *outs, wc_field const *ins,
                               wc_field const *tmps, int dagger, const int *const *skip, cudaStream_t stream,
                               int red, wc_field const *dots, double *part)
{
    if (n < 1 || n > kMrhsMax || !half->schur_parent) return cudaErrorInvalidValue;
    const wc_lattice_s *full = half->schur_parent;
    const wc_prec pr = ins[0]->prec;
    if (red != 0 && (pr != WC_F32 || !part || (red == 1 && !dots))) return cudaErrorInvalidValue;
    if (pr == WC_F32)
        return dagger ? launch_eom<P32, 1>(full, n, outs, ins, tmps, skip, red, dots, part, stream)
                      : launch_eom<P32, 0>(full, n, outs, ins, tmps, skip, red, dots, part, stream);
    if (pr == WC_F16)
        return dagger ? launch_eom<P16, 1>(full, n, outs, ins, tmps, skip, 0, nullptr, nullptr, stream)
                      : launch_eom<P16, 0>(full, n, outs, ins, tmps, skip, 0, nullptr, nullptr, stream);
    return cudaErrorInvalidValue;
}

int schur_multi_blocks(wc_lattice half) { return (half->g.V + kEoMSites - 1) / kEoMSites; }

}  // namespace wc

using namespace wc;

// outs[r] = M^ ins[r] (even sites; odd sites of outs set to zero) for FP32
// or FP16 full-lattice fields of one lattice
extern "C" wc_status wc_apply_schur_multi(wc_lattice lat, int n, wc_field *outs, wc_field *ins, int dagger)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (n < 1 || n > kMrhsMax || !outs || !ins)
        return set_error(lat, WC_ERR_ARG, "n must be in 1.." + std::to_string(kMrhsMax) + ", outs/ins non-NULL");
    for (int r = 0; r < n; ++r) {
        if (!outs[r] || !ins[r] || outs[r]->lat != lat || ins[r]->lat != lat)
            return set_error(lat, WC_ERR_ARG, "fields must belong to the lattice");
        if (ins[r]->prec != ins[0]->prec || outs[r]->prec != ins[0]->prec || ins[0]->prec == WC_F64)
            return set_error(lat, WC_ERR_ARG, "the multi-RHS Schur operator takes FP32 or FP16 fields of one precision");
        for (int q = 0; q < n; ++q)
            if (outs[r] == ins[q] || (q < r && outs[r] == outs[q]))
                return set_error(lat, WC_ERR_ARG, "out fields must be distinct from each other and from the inputs");
    }
    wc_status st = require_operator(lat);
    if (st != WC_OK) return st;
    wc_lattice h = nullptr;
    st = half_lattice(lat, &h);
    if (st != WC_OK) return st;
    const wc_prec pr = ins[0]->prec;
    std::vector<wc_field> e(n, nullptr), r(n, nullptr), t(n, nullptr);
    for (int k = 0; k < n && st == WC_OK; ++k) {
        st = wc_field_create(h, pr, &e[k]);
        if (st == WC_OK) st = wc_field_create(h, pr, &r[k]);
        if (st == WC_OK) st = wc_field_create(h, pr, &t[k]);
    }
    for (int k = 0; k < n && st == WC_OK; ++k)
        st = check_cuda(lat, launch_split(lat, ins[k], e[k], nullptr, lat->stream), "split");
    if (st == WC_OK)
        st = check_cuda(lat, launch_schur_multi(h, n, r.data(), e.data(), t.data(), dagger ? 1 : 0, nullptr, lat->stream),
                        "schur_multi");
    for (int k = 0; k < n && st == WC_OK; ++k)
        st = check_cuda(lat, launch_merge(lat, r[k], nullptr, outs[k], lat->stream), "merge");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync");
    for (int k = 0; k < n; ++k) {
        wc_field_destroy(e[k]);
        wc_field_destroy(r[k]);
        wc_field_destroy(t[k]);
    }
    return st;
}
