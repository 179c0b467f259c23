// Even-odd (Schur complement) preconditioning of M.  Sec. 2: both the FP64
// outer solver and the FP32 inner solver of CCS-QCD act on the even-odd
// site preconditioned matrix; the elimination below is the standard one.
//
// Ordering the sites by parity, M = [[A_ee, -k H_eo], [-k H_oe, A_oo]], so
//   b^_e = b_e + k H_eo A_oo^-1 b_o
//   M^ x_e = b^_e,   M^ = A_ee - k^2 H_eo A_oo^-1 H_oe   (even sites only)
//   x_o = A_oo^-1 (b_o + k H_oe x_e)
// and M^+ = gamma5 M^ gamma5 (gamma5 commutes with A and anticommutes with
// each hop).  The solvers run unchanged on half-volume fields of a
// "half lattice" (same gauge field and clover term, V/2 sites); its operator
// is M^.
//
// Half-volume layout: a field of parity p stores site (x,y,z,t) at index
// i = (x + Lx (y + Ly (z + Lz t))) >> 1; all extents are even (so that
// every hop, also across the boundary, flips the parity), hence every x-row
// holds Lx/2 sites of each parity and i is unique within a parity.
#include <math.h>

#include <new>

#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

// ------------------------------------------------------------------------
// clover inverse: A^-1 as two packed Hermitian 6x6 blocks (FP64 arithmetic)
// ------------------------------------------------------------------------

__device__ void unpack_block(const double r[36], cx<double> m[6][6])
{
    for (int i = 0; i < 6; ++i) m[i][i] = mkc(r[i], 0.0);
    int k = 6;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j) {
            m[i][j] = mkc(r[k], r[k + 1]);
            m[j][i] = conj(m[i][j]);
            k += 2;
        }
}

__device__ void pack_block(cx<double> m[6][6], double r[36])
{
    // Hermitian by construction; symmetrise the rounding
    for (int i = 0; i < 6; ++i) r[i] = m[i][i].re;
    int k = 6;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j) {
            const cx<double> a = m[i][j], b = conj(m[j][i]);
            r[k++] = 0.5 * (a.re + b.re);
            r[k++] = 0.5 * (a.im + b.im);
        }
}

// Gauss-Jordan inverse with partial pivoting (6x6 complex, in place).
// Returns false if a pivot is below 1e-12 of the block's largest entry
// (numerically singular: the inverse would carry no significant digit).
__device__ bool invert6(cx<double> a[6][6])
{
    double amax = 0.0;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) amax = fmax(amax, fabs(a[i][j].re) + fabs(a[i][j].im));
    const double tiny2 = (1e-12 * amax) * (1e-12 * amax);
    cx<double> inv[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) inv[i][j] = mkc(i == j ? 1.0 : 0.0, 0.0);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = a[c][c].re * a[c][c].re + a[c][c].im * a[c][c].im;
        for (int r = c + 1; r < 6; ++r) {
            const double v = a[r][c].re * a[r][c].re + a[r][c].im * a[r][c].im;
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > tiny2) || !(best > 0.0)) return false;
        if (piv != c)
            for (int j = 0; j < 6; ++j) {
                cx<double> t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
                t = inv[c][j];
                inv[c][j] = inv[piv][j];
                inv[piv][j] = t;
            }
        const cx<double> p = a[c][c];
        const double d = p.re * p.re + p.im * p.im;
        const cx<double> pinv = mkc(p.re / d, -p.im / d);
        for (int j = 0; j < 6; ++j) {
            a[c][j] = pinv * a[c][j];
            inv[c][j] = pinv * inv[c][j];
        }
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            const cx<double> f = a[r][c];
            for (int j = 0; j < 6; ++j) {
                a[r][j] = a[r][j] - f * a[c][j];
                inv[r][j] = inv[r][j] - f * inv[c][j];
            }
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) a[i][j] = inv[i][j];
    return true;
}

// one packed block (36 reals) at position pos of a clover store, in all
// three precisions
__device__ void store_block(const CloverStore &S, int V, int pos, int b, const double r[36])
{
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const double2 v = make_double2(r[2 * q], r[2 * q + 1]);
        S.c64[((size_t)b * 18 + q) * V + pos] = v;
        S.cdf[((size_t)b * 18 + q) * V + pos] = df_pack(v);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q)
        S.c32[((size_t)b * 9 + q) * V + pos] =
            make_float4((float)r[4 * q], (float)r[4 * q + 1], (float)r[4 * q + 2], (float)r[4 * q + 3]);
    unsigned *c16 = reinterpret_cast<unsigned *>(S.c16);
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const int gq = 18 * b + q;
        c16[((size_t)(gq >> 2) * V + pos) * 4 + (gq & 3)] = c2h((float)r[2 * q], (float)r[2 * q + 1]);
    }
}

// Parity-ordered copies for the even-odd kernels: within every component
// plane, position parity(x) * V/2 + (x >> 1), so that the threads of one
// parity read contiguous memory (full-volume order would fetch every other
// site's entries with them).  Ce: A = 1 + T; Ci: A^-1.
__global__ void k_clover_invert(Geom g, CloverStore C, CloverStore Ce, CloverStore Ci, int *bad)
{
    const int V = g.V;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    int c[4];
    site_coords(g, x, c);
    const int pos = ((c[0] + c[1] + c[2] + c[3]) & 1) * (V >> 1) + (x >> 1);
    for (int b = 0; b < 2; ++b) {
        double r[36];
        P64::load_clover(C, V, x, b, r);
        store_block(Ce, V, pos, b, r);
        cx<double> m[6][6];
        unpack_block(r, m);
        if (!invert6(m)) atomicExch(bad, 1);
        pack_block(m, r);
        store_block(Ci, V, pos, b, r);
    }
}

// ------------------------------------------------------------------------
// parity stencil
// ------------------------------------------------------------------------

// full site of half index i of parity p
__device__ __forceinline__ int full_site(const Geom &g, int i, int p, int c[4])
{
    const int hx = g.L[0] >> 1;
    const int xh = i % hx;
    int rest = i / hx;
    c[1] = rest % g.L[1];
    rest /= g.L[1];
    c[2] = rest % g.L[2];
    c[3] = rest / g.L[2];
    c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
    return wc_idx(c[0] + g.stride[1] * c[1] + g.stride[2] * c[2] + g.stride[3] * c[3], g.V);
}

// hops of the opposite-parity half field `in` into site x (full index x,
// coordinates c), accumulated into acc with coefficient k (boundary phase
// included); links from the full-volume store
template <class P, int MU, int SF, int SB>
__device__ __forceinline__ void eo_hop_dir(const Geom &g, const GaugeStore &U, const void *in, const float *in_nrm,
                                           int Vh, int x, const int c[4], typename P::real k,
                                           cx<typename P::real> acc[12])
{
    using R = typename P::real;
    const int L = g.L[MU], st = g.stride[MU];
    {
        const bool wrap = c[MU] == L - 1;
        const int xf = wc_idx(wrap ? x - (L - 1) * st : x + st, g.V);
        cx<R> p[12], h[6], u[6], r2[3], w[6];
        const R scale = P::load_spinor_raw(in, in_nrm, Vh, xf >> 1, p);
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
        const R scale = P::load_spinor_raw(in, in_nrm, Vh, xb >> 1, p);
        const R coef = ((MU == 3 && wrap) ? k * R(g.tbc) : k) * scale;
        project<MU, SB>(p, h);
        P::load_link(U, g.V, MU, xb, u, r2);
        su3_adj_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SB>(acc, w);
    }
}

// y = A v at position pos of a parity-ordered clover store (A or A^-1)
template <class P>
__device__ __forceinline__ void clover_eo(const CloverStore &S, int V, int pos, const cx<typename P::real> v[12],
                                          cx<typename P::real> y[12])
{
    if constexpr (std::is_same<P, PDF>::value) {   // compact form (instruction cache)
        clover_block_rt<P>(S, V, pos, 0, v, y);
        clover_block_rt<P>(S, V, pos, 1, v + 6, y + 6);
    } else {
        using R = typename P::real;
        R r0[36], r1[36];
        P::load_clover(S, V, pos, 0, r0);
        P::load_clover(S, V, pos, 1, r1);
        clover_block_mul(r0, v, y);
        clover_block_mul(r1, v + 6, y + 6);
    }
}

// For the sites of parity p (half index i):
//   HOP: h = sum of hops of `hin` (opposite parity)
//   C, Ci: clover and inverse in parity order (k_clover_invert)
//   MODE 0: out = Cinv h
//        1: out = C vin + beta h
//        2: out = vin + beta h
//        3: out = Cinv (vin + beta h)
//        4: out = Cinv vin
//        5: out = Cinv w and out2 = w - C out, w = vin + beta h (with
//           vin = b_o, h = H_oe x_e, beta = k: the reconstructed x_o and
//           the odd-site residual b_o - (A_oo x_o - k H_oe x_e) of the
//           x_o as stored, in one pass; FP64 fields only)
// The site-local part of k_eo after the hops h: everything but the hops,
// in the arithmetic of P.
template <class P, int MODE>
__device__ __forceinline__ void eo_tail(const Geom &g, int p, const CloverStore &C, const CloverStore &Ci,
                                        const void *vin, const float *vin_nrm, void *out, float *out_nrm,
                                        void *out2, double beta, int Vh, int i, const cx<typename P::real> h[12])
{
    using R = typename P::real;
    cx<R> v[12], o[12];
    const R bt = R(beta);
    if (MODE == 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = h[k];
    } else {
        P::load_spinor(vin, vin_nrm, Vh, i, v);
        if (MODE == 1) {
            clover_eo<P>(C, g.V, wc_idx(p * Vh + i, g.V), v, o);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = o[k] + bt * h[k];
            P::store_spinor(out, out_nrm, Vh, i, o);
            return;
        }
        if (MODE == 2 || MODE == 3 || MODE == 5)
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = v[k] + bt * h[k];
        if (MODE == 2) {
            P::store_spinor(out, out_nrm, Vh, i, v);
            return;
        }
    }
    clover_eo<P>(Ci, g.V, wc_idx(p * Vh + i, g.V), v, o);
    P::store_spinor(out, out_nrm, Vh, i, o);
    if constexpr (MODE == 5) {
        // the residual of x_o as the caller receives it (the stored value)
        cx<R> y[12];
        P::as_stored(o);
        clover_eo<P>(C, g.V, wc_idx(p * Vh + i, g.V), o, y);
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = v[k] - y[k];
        P::store_spinor(out2, nullptr, Vh, i, y);
    }
}

template <class P, int DAG, int MODE>
__global__ void __launch_bounds__(128, P::kEoMinBlocks) k_eo(Geom g, int p, GaugeStore U, CloverStore C, CloverStore Ci,
                                            const void *hin, const float *hin_nrm, const void *vin,
                                            const float *vin_nrm, void *out, float *out_nrm, void *out2,
                                            double beta)
{
    using R = typename P::real;
    const int Vh = g.V >> 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vh) return;
    int c[4];
    const int x = full_site(g, i, p, c);
    if constexpr (std::is_same<P, PDF>::value) {
        // compact form (instruction cache): hops and clover rows in runtime
        // loops.  Measured at 24^3x32 (even-odd FP64-class solve, 40 such
        // passes): the site-local A / A^-1 products in FP64 on the FP64 pipe
        // 2 % slower, with the two x hops in FP64 too 8 % slower, and a
        // 168- or 255-register cap (12 or 8 warps per SM, no spills) 2 % and
        // 23 % slower than this form at 128 registers and 16 warps.
        cx<R> h[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) h[k] = mkc(R(0.0f, 0.0f), R(0.0f, 0.0f));
        if (MODE != 4)
            hops_rt<P, DAG ? +1 : -1>(g, U, hin, hin_nrm, Vh, x, c, R(1.0f, 0.0f), h, [](int y) { return y >> 1; });
        eo_tail<P, MODE>(g, p, C, Ci, vin, vin_nrm, out, out_nrm, out2, beta, Vh, i, h);
    } else {
        cx<R> h[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) h[k] = mkc(R(0), R(0));
        if (MODE != 4) {
            constexpr int SF = DAG ? +1 : -1;
            constexpr int SB = -SF;
            const R one = R(1);
            eo_hop_dir<P, 0, SF, SB>(g, U, hin, hin_nrm, Vh, x, c, one, h);
            eo_hop_dir<P, 1, SF, SB>(g, U, hin, hin_nrm, Vh, x, c, one, h);
            eo_hop_dir<P, 2, SF, SB>(g, U, hin, hin_nrm, Vh, x, c, one, h);
            eo_hop_dir<P, 3, SF, SB>(g, U, hin, hin_nrm, Vh, x, c, one, h);
        }
        eo_tail<P, MODE>(g, p, C, Ci, vin, vin_nrm, out, out_nrm, out2, beta, Vh, i, h);
    }
}

// full field <-> the two half fields (parity 0 = even, 1 = odd)
template <class P>
__global__ void k_split(Geom g, const void *full, const float *full_nrm, void *ev, float *ev_nrm, void *od,
                        float *od_nrm)
{
    const int Vh = g.V >> 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vh) return;
    int c[4];
    cx<typename P::real> s[12];
    P::load_spinor(full, full_nrm, g.V, full_site(g, i, 0, c), s);
    P::store_spinor(ev, ev_nrm, Vh, i, s);
    if (!od) return;   // odd half not wanted
    P::load_spinor(full, full_nrm, g.V, full_site(g, i, 1, c), s);
    P::store_spinor(od, od_nrm, Vh, i, s);
}

template <class P>
__global__ void k_merge(Geom g, const void *ev, const float *ev_nrm, const void *od, const float *od_nrm,
                        void *full, float *full_nrm)
{
    const int Vh = g.V >> 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vh) return;
    int c[4];
    cx<typename P::real> s[12];
    P::load_spinor(ev, ev_nrm, Vh, i, s);
    P::store_spinor(full, full_nrm, g.V, full_site(g, i, 0, c), s);
    if (od) {
        P::load_spinor(od, od_nrm, Vh, i, s);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = mkc(typename P::real(0), typename P::real(0));
    }
    P::store_spinor(full, full_nrm, g.V, full_site(g, i, 1, c), s);
}

template <class P, int DAG>
cudaError_t launch_eo_p(const wc_lattice_s *full, int parity, int mode, const wc_field_s *hin, const wc_field_s *vin,
                        wc_field_s *out, double beta, cudaStream_t stream, wc_field_s *out2)
{
    const int Vh = full->g.V >> 1;
    // CTAs of 128 sites; on small lattices (fewer than two such CTAs per SM)
    // CTAs of 32, so that the sites spread over more SMs
    const int threads = Vh < 2 * 128 * sm_count() ? 32 : 128;
    dim3 grid((Vh + threads - 1) / threads), block(threads);
    const void *hd = hin ? hin->data : nullptr;
    const float *hn = hin ? hin->nrm : nullptr;
    const void *vd = vin ? vin->data : nullptr;
    const float *vn = vin ? vin->nrm : nullptr;
    void *o2 = out2 ? out2->data : nullptr;
#define WC_EO(M)                                                                                                \
    k_eo<P, DAG, M><<<grid, block, 0, stream>>>(full->g, parity, full->gauge, full->ceo, full->cinv, hd, hn,    \
                                                vd, vn, out->data, out->nrm, o2, beta)
    switch (mode) {
    case 0: WC_EO(0); break;
    case 1: WC_EO(1); break;
    case 2: WC_EO(2); break;
    case 3: WC_EO(3); break;
    case 4: WC_EO(4); break;
    default:
        if constexpr (std::is_same<P, P64>::value || std::is_same<P, PDF>::value) {
            if (!out2 || out2->prec != WC_F64) return cudaErrorInvalidValue;
            WC_EO(5);
        } else {
            return cudaErrorInvalidValue;
        }
    }
#undef WC_EO
    return cudaGetLastError();
}

}  // namespace

// one parity-stencil step on half fields of the full lattice `full`
cudaError_t launch_eo(const wc_lattice_s *full, int parity, int mode, int dagger, const wc_field_s *hin,
                      const wc_field_s *vin, wc_field_s *out, double beta, cudaStream_t stream, wc_field_s *out2)
{
    const wc_prec pr = out->prec;
    if (pr == WC_F64 && full->fp64_arith == WC_ARITH_DF32)
        return dagger ? launch_eo_p<PDF, 1>(full, parity, mode, hin, vin, out, beta, stream, out2)
                      : launch_eo_p<PDF, 0>(full, parity, mode, hin, vin, out, beta, stream, out2);
    if (pr == WC_F64)
        return dagger ? launch_eo_p<P64, 1>(full, parity, mode, hin, vin, out, beta, stream, out2)
                      : launch_eo_p<P64, 0>(full, parity, mode, hin, vin, out, beta, stream, out2);
    if (pr == WC_F32)
        return dagger ? launch_eo_p<P32, 1>(full, parity, mode, hin, vin, out, beta, stream, out2)
                      : launch_eo_p<P32, 0>(full, parity, mode, hin, vin, out, beta, stream, out2);
    return dagger ? launch_eo_p<P16, 1>(full, parity, mode, hin, vin, out, beta, stream, out2)
                  : launch_eo_p<P16, 0>(full, parity, mode, hin, vin, out, beta, stream, out2);
}

// od may be NULL: only the even half is written
cudaError_t launch_split(const wc_lattice_s *full, const wc_field_s *f, wc_field_s *ev, wc_field_s *od,
                         cudaStream_t stream)
{
    const int Vh = full->g.V >> 1;
    dim3 grid((Vh + 255) / 256), block(256);
    void *od_d = od ? od->data : nullptr;
    float *od_n = od ? od->nrm : nullptr;
    if (f->prec == WC_F64)
        k_split<P64><<<grid, block, 0, stream>>>(full->g, f->data, f->nrm, ev->data, ev->nrm, od_d, od_n);
    else if (f->prec == WC_F32)
        k_split<P32><<<grid, block, 0, stream>>>(full->g, f->data, f->nrm, ev->data, ev->nrm, od_d, od_n);
    else
        k_split<P16><<<grid, block, 0, stream>>>(full->g, f->data, f->nrm, ev->data, ev->nrm, od_d, od_n);
    return cudaGetLastError();
}

// od may be NULL: the odd sites of f are set to zero
cudaError_t launch_merge(const wc_lattice_s *full, const wc_field_s *ev, const wc_field_s *od, wc_field_s *f,
                         cudaStream_t stream)
{
    const int Vh = full->g.V >> 1;
    dim3 grid((Vh + 255) / 256), block(256);
    const void *od_d = od ? od->data : nullptr;
    const float *od_n = od ? od->nrm : nullptr;
    if (f->prec == WC_F64)
        k_merge<P64><<<grid, block, 0, stream>>>(full->g, ev->data, ev->nrm, od_d, od_n, f->data, f->nrm);
    else if (f->prec == WC_F32)
        k_merge<P32><<<grid, block, 0, stream>>>(full->g, ev->data, ev->nrm, od_d, od_n, f->data, f->nrm);
    else
        k_merge<P16><<<grid, block, 0, stream>>>(full->g, ev->data, ev->nrm, od_d, od_n, f->data, f->nrm);
    return cudaGetLastError();
}

// out = M^ in (or M^+ in) on half fields of the half lattice `half`: t = A_oo^-1 H_oe in,
// out = A_ee in - k^2 H_eo t.  t: the half lattice's scratch of out's precision.
cudaError_t launch_schur(wc_lattice half, wc_field out, wc_field in, int dagger, cudaStream_t stream, wc_field tmp)
{
    const wc_lattice_s *full = half->schur_parent;
    wc_field_s *t = tmp ? tmp : half->schur_tmp[out->prec];
    cudaError_t e = launch_eo(full, 1, 0, dagger, in, nullptr, t, 0.0, stream);
    if (e == cudaSuccess) e = launch_eo(full, 0, 1, dagger, t, in, out, -full->kappa * full->kappa, stream);
    return e;
}

cudaError_t launch_apply(wc_lattice lat, wc_field out, wc_field in, int kind, SolverState &S)
{
    if (!lat->schur_parent) return launch_apply(lat, out, in, kind, S.stream);
    return launch_schur(lat, out, in, kind == 1, S.stream, S.work[kSchurSlot + out->prec]);
}

wc_status build_clover_inverse(wc_lattice lat)
{
    if (lat->cinv_loaded) return WC_OK;
    const int V = lat->g.V;
    wc_status st = WC_OK;
    for (CloverStore *c : {&lat->cinv, &lat->ceo}) {
        if (c->c64) continue;
        st = check_cuda(lat, cudaMalloc(&c->c64, sizeof(double2) * 36 * (size_t)V), "cudaMalloc(clover inverse)");
        if (st == WC_OK)
            st = check_cuda(lat, cudaMalloc(&c->cdf, sizeof(float4) * 36 * (size_t)V), "cudaMalloc(clover inverse)");
        if (st == WC_OK)
            st = check_cuda(lat, cudaMalloc(&c->c32, sizeof(float4) * 18 * (size_t)V), "cudaMalloc(clover inverse)");
        if (st == WC_OK)
            st = check_cuda(lat, cudaMalloc(&c->c16, sizeof(uint4) * 9 * (size_t)V), "cudaMalloc(clover inverse)");
        if (st != WC_OK) return st;
    }
    int *bad = nullptr;
    st = check_cuda(lat, cudaMalloc(&bad, sizeof(int)), "cudaMalloc");
    if (st != WC_OK) return st;
    st = check_cuda(lat, cudaMemsetAsync(bad, 0, sizeof(int), lat->stream), "memset");
    if (st == WC_OK) {
        k_clover_invert<<<(V + 63) / 64, 64, 0, lat->stream>>>(lat->g, lat->clover, lat->ceo, lat->cinv, bad);
        st = check_launch(lat, "clover_invert");
    }
    int h = 0;
    if (st == WC_OK) st = check_cuda(lat, cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, lat->stream),
                                     "copy");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync");
    cudaFree(bad);
    if (st != WC_OK) return st;
    if (h) return set_error(lat, WC_ERR_BREAKDOWN, "clover term is singular at some site");
    lat->cinv_loaded = true;
    return WC_OK;
}

// The half lattice of lat (created on first use): V/2 sites, operator M^.
wc_status half_lattice(wc_lattice lat, wc_lattice *out)
{
    // every hop must change the parity, also across the (anti)periodic
    // boundary: all four extents even
    for (int mu = 0; mu < 4; ++mu)
        if (lat->g.L[mu] % 2 != 0) return set_error(lat, WC_ERR_ARG, "even-odd needs even lattice extents");
    wc_status st = build_clover_inverse(lat);
    if (st != WC_OK) return st;
    if (!lat->half) {
        wc_lattice h = new (std::nothrow) wc_lattice_s();
        if (!h) return set_error(lat, WC_ERR_ARG, "out of host memory");
        h->g = lat->g;
        h->g.V = lat->g.V / 2;
        h->schur_parent = lat;
        h->gauge_loaded = h->clover_loaded = true;
        h->kappa = lat->kappa;
        h->csw = lat->csw;
        h->stream = lat->stream;
        st = state_init(lat, h->st);
        for (int pr = 0; pr < 3 && st == WC_OK; ++pr) st = wc_field_create(h, (wc_prec)pr, &h->schur_tmp[pr]);
        if (st != WC_OK) {
            for (auto &f : h->schur_tmp) wc_field_destroy(f);
            state_free(h->st);
            delete h;
            return st;
        }
        lat->half = h;
    }
    lat->half->stream = lat->stream;
    lat->half->kappa = lat->kappa;
    *out = lat->half;
    return WC_OK;
}

void free_batch_pool(wc_lattice lat)
{
    for (auto &s : lat->batch_states) state_free(s);
    lat->batch_states.clear();
    for (auto f : lat->batch_fields) wc_field_destroy(f);
    lat->batch_fields.clear();
}

void free_half(wc_lattice lat)
{
    if (!lat->half) return;
    free_batch_pool(lat->half);
    for (auto f : lat->batch_fields) wc_field_destroy(f);   // half-lattice fields
    lat->batch_fields.clear();
    for (auto &pr : lat->ras_half)
        for (auto &f : pr) {
            wc_field_destroy(f);
            f = nullptr;
        }
    for (auto &f : lat->half->schur_tmp) wc_field_destroy(f);
    state_free(lat->half->st);
    delete lat->half;
    lat->half = nullptr;
}

}  // namespace wc
