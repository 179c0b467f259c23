// Pseudofermion action S = phi^+ (M^+ M)^-1 phi and its force per link.
//
// With Y solving M^+ Y = phi and X solving M X = Y, S = |Y|^2 and, for a
// link variation U_mu(x) -> exp(eps L) U_mu(x) with L in su(3),
//   dS/deps = -2 Re <Y, (dM/deps) X> = Re tr(L G_mu(x)),
// and the force is the traceless anti-Hermitian projection
//   F = TA(G) = (G - G^+)/2 - tr(G - G^+)/6.
// TA is the orthogonal projection onto su(3) for <A, B> = Re tr(A^+ B), so G
// only matters through Re tr(L G) with L anti-Hermitian: G and G' give the
// same F whenever they differ by a Hermitian matrix or a multiple of 1.  In
// particular, for any complex c and matrix B, c B^+ and -conj(c) B give the
// same F.  The kernel uses this to move U_mu(x) to the far left of every
// term and forms F = TA(U H) from one 3x3 matrix H per link.
//
// Hopping part (the forward hop at x and the backward hop at x+mu use the
// link; p the time-boundary factor of the hop):
//   G_hop = 2 kappa p [ sum_s (U (1-g_mu) X(x+mu))_s Y_s(x)^+
//                       - sum_s ((1+g_mu) X(x))_s Y_s(x+mu)^+ U^+ ]
//   H_hop = 2 kappa p sum_s [ ((1-g_mu) X(x+mu))_s Y_s(x)^+
//                             + Y_s(x+mu) ((1+g_mu) X(x))_s^+ ].
//
// Clover part: T = i csw kappa sum_{a<b} sigma_ab (x) Fhat_ab, so
//   <Y, dT X> = sum_y sum_{a<b} (i csw kappa / 8)(tr(dQ Xi) - tr(dQ^+ Xi))
// with Xi_ab(y) the traceless part of sum_{s,t} sigma_ab[s][t] X_t(y) Y_s(y)^+.
// For the link (x, mu) and each plaquette containing it -- corners c0 = x,
// c1 = x+mu, c2 = x+mu+d nu, c3 = x+d nu (d = +-1), loop links U = L0, L1,
// L2, L3 in that order -- every clover leaf based at corner c_k contributes
// through W_k(Z) = L0 ... L_{k-1} Z L_k ... L3 (k = 1..4, corner c_{k mod 4}):
//   G += c sum_k [W_k(Xi(c_k)) + W_k(Xi(c_k)^+)^+],  c = -(i csw kappa / 4) sigma
// where sigma = +1 when the loop c0 c1 c2 c3 runs counter-clockwise in the
// (a, b) = (min(mu,nu), max(mu,nu)) plane (the leaves' orientation) and -1
// when the leaves run through the link backwards.  As c is imaginary, the
// second term gives the same F as c W_k(Xi^+), so only the Hermitian
// Xh = Xi + Xi^+ enters (k_xi stores it, 9 reals per plane and site), and
//   sum_k W_k(Xh_k) = U [ Xh(c1) T + L1 (S2 Xh(x) + (Xh(c2) L2 + L2 Xh(c3)) L3) ]
// with S2 = L2 L3 and T = L1 S2: eight 3x3 products per leaf pair (nu, d)
// instead of twenty-one for the four insertions taken one by one.

#include <math.h>

#include "wc_internal.cuh"
#include "wc_solver.cuh"
#include "wc_solver_kernels.cuh"

namespace wc {


namespace {

struct M3 {
    cx<double> m[3][3];
};

__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = a.m[i][0] * b.m[0][j];
            s = cfma(a.m[i][1], b.m[1][j], s);
            s = cfma(a.m[i][2], b.m[2][j], s);
            r.m[i][j] = s;
        }
    return r;
}

__device__ __forceinline__ M3 dag(const M3 &a)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

__device__ __forceinline__ M3 ident()
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = mkc(i == j ? 1.0 : 0.0, 0.0);
    return r;
}

__device__ __forceinline__ void add_scaled(M3 &acc, cx<double> s, const M3 &a)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) acc.m[i][j] = cfma(s, a.m[i][j], acc.m[i][j]);
}

__device__ M3 link(const GaugeStore &g, int V, int mu, int x)
{
    cx<double> u[6], r2[3];
    P64::load_link(g, V, mu, x, u, r2);
    M3 r;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        r.m[0][j] = u[j];
        r.m[1][j] = u[3 + j];
        r.m[2][j] = r2[j];
    }
    return r;
}

__device__ __forceinline__ int shift(const Geom &g, const int c[4], int mu, int dmu, int nu, int dnu)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + dmu + g.L[mu]) % g.L[mu];
    d[nu] = (d[nu] + dnu + g.L[nu]) % g.L[nu];
    return d[0] + g.stride[1] * d[1] + g.stride[2] * d[2] + g.stride[3] * d[3];
}

// plane index of (a, b), a < b: xy xz xt yz yt zt
__device__ __forceinline__ int plane_of(int a, int b)
{
    return a == 0 ? b - 1 : a == 1 ? b + 1 : 5;
}

// 2x2 block of sigma_ab on spin pair blk (chiral basis), as complex entries
// sigma_xy = -s3, sigma_xz = s2, sigma_yz = -s1 on both pairs;
// sigma_xt = eta s1, sigma_yt = eta s2, sigma_zt = eta s3, eta = -1, +1
__device__ __forceinline__ void sigma_block(int plane, int blk, cx<double> s[2][2])
{
    const double eta = blk == 0 ? -1.0 : 1.0;
    int pauli;
    double sg;
    switch (plane) {
    case 0: pauli = 3; sg = -1.0; break;   // xy
    case 1: pauli = 2; sg = 1.0; break;    // xz
    case 2: pauli = 1; sg = eta; break;    // xt
    case 3: pauli = 1; sg = -1.0; break;   // yz
    case 4: pauli = 2; sg = eta; break;    // yt
    default: pauli = 3; sg = eta; break;   // zt
    }
    const cx<double> z = mkc(0.0, 0.0);
    s[0][0] = s[0][1] = s[1][0] = s[1][1] = z;
    if (pauli == 1) {
        s[0][1] = mkc(sg, 0.0);
        s[1][0] = mkc(sg, 0.0);
    } else if (pauli == 2) {
        s[0][1] = mkc(0.0, -sg);
        s[1][0] = mkc(0.0, sg);
    } else {
        s[0][0] = mkc(sg, 0.0);
        s[1][1] = mkc(-sg, 0.0);
    }
}

// Hermitian 3x3 matrix: real diagonal d, upper entries o = (h01, h02, h12)
struct H3 {
    double d[3];
    cx<double> o[3];
};

// off-diagonal entry (i, k), i != k (constants once the callers are unrolled)
__device__ __forceinline__ cx<double> hoff(const H3 &h, int i, int k)
{
    const cx<double> v = h.o[i + k - 1];
    return i < k ? v : conj(v);
}

// acc + H B
__device__ __forceinline__ void fma_hm(const H3 &h, const M3 &b, M3 &acc)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = acc.m[i][j];
            s.re = fma(h.d[i], b.m[i][j].re, s.re);
            s.im = fma(h.d[i], b.m[i][j].im, s.im);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k != i) s = cfma(hoff(h, i, k), b.m[k][j], s);
            acc.m[i][j] = s;
        }
}

// acc + A H
__device__ __forceinline__ void fma_mh(const M3 &a, const H3 &h, M3 &acc)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = acc.m[i][j];
            s.re = fma(a.m[i][j].re, h.d[j], s.re);
            s.im = fma(a.m[i][j].im, h.d[j], s.im);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k != j) s = cfma(a.m[i][k], hoff(h, k, j), s);
            acc.m[i][j] = s;
        }
}

__device__ __forceinline__ M3 zero3()
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = mkc(0.0, 0.0);
    return r;
}

// Xh_ab(y) = Xi + Xi^+ for the six planes, Xi the traceless part of
// sum_{s,t} sigma_ab[s][t] X_t(y) Y_s(y)^+.  Layout [6][9][V] doubles:
// h00 h11 h22, re/im of h01, h02, h12.
__global__ void k_xi(Geom g, const double2 *X, const double2 *Y, double *xh)
{
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= g.V) return;
    const int V = g.V;
    cx<double> xs[12], ys[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 a = X[(size_t)k * V + y], b = Y[(size_t)k * V + y];
        xs[k] = mkc(a.x, a.y);
        ys[k] = mkc(b.x, b.y);
    }
#pragma unroll
    for (int pl = 0; pl < 6; ++pl) {
        M3 Z = zero3();
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
            cx<double> sg[2][2];
            sigma_block(pl, blk, sg);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const cx<double> w = sg[s][t];
                    if (w.re == 0.0 && w.im == 0.0) continue;
                    const int ss = 2 * blk + s, tt = 2 * blk + t;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            Z.m[i][j] = cfma(w, xs[3 * tt + i] * conj(ys[3 * ss + j]), Z.m[i][j]);
                }
        }
        const double tr = (2.0 / 3.0) * (Z.m[0][0].re + Z.m[1][1].re + Z.m[2][2].re);
        double *o = xh + (size_t)pl * 9 * V + y;
        o[0] = 2.0 * Z.m[0][0].re - tr;
        o[(size_t)V] = 2.0 * Z.m[1][1].re - tr;
        o[2 * (size_t)V] = 2.0 * Z.m[2][2].re - tr;
        const int ij[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const cx<double> v = Z.m[ij[k][0]][ij[k][1]] + conj(Z.m[ij[k][1]][ij[k][0]]);
            o[(size_t)(3 + 2 * k) * V] = v.re;
            o[(size_t)(4 + 2 * k) * V] = v.im;
        }
    }
}

__device__ __forceinline__ H3 load_xh(const double *xh, int V, int plane, int y)
{
    const double *p = xh + (size_t)plane * 9 * V + y;
    H3 h;
#pragma unroll
    for (int k = 0; k < 3; ++k) h.d[k] = __ldg(p + (size_t)k * V);
#pragma unroll
    for (int k = 0; k < 3; ++k) h.o[k] = mkc(__ldg(p + (size_t)(3 + 2 * k) * V), __ldg(p + (size_t)(4 + 2 * k) * V));
    return h;
}

// (1 + s gamma_mu) psi as a full spinor (chiral basis)
__device__ __forceinline__ void project_full(int mu, int s, const cx<double> p[12], cx<double> o[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<double> u0 = p[c], u1 = p[3 + c], d0 = p[6 + c], d1 = p[9 + c];
        const double sd = (double)s;
        cx<double> h0, h1, l0, l1;
        if (mu == 0) {
            h0 = u0 + sd * times_i(d1);
            h1 = u1 + sd * times_i(d0);
            l0 = (-sd) * times_i(h1);
            l1 = (-sd) * times_i(h0);
        } else if (mu == 1) {
            h0 = u0 + sd * d1;
            h1 = u1 - sd * d0;
            l0 = (-sd) * h1;
            l1 = sd * h0;
        } else if (mu == 2) {
            h0 = u0 + sd * times_i(d0);
            h1 = u1 - sd * times_i(d1);
            l0 = (-sd) * times_i(h0);
            l1 = sd * times_i(h1);
        } else {
            h0 = u0 + sd * d0;
            h1 = u1 + sd * d1;
            l0 = sd * h0;
            l1 = sd * h1;
        }
        o[c] = h0;
        o[3 + c] = h1;
        o[6 + c] = l0;
        o[9 + c] = l1;
    }
}

__device__ __forceinline__ void load_sp(const double2 *f, int V, int x, cx<double> s[12])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 v = __ldg(f + (size_t)k * V + x);
        s[k] = mkc(v.x, v.y);
    }
}

// acc + sum_s a_s b_s^+ (a, b spinors; 3x3 colour outer products summed over spin)
__device__ __forceinline__ void fma_outer(const cx<double> a[12], const cx<double> b[12], M3 &acc)
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc.m[p][q] = cfma(a[3 * s + p], conj(b[3 * s + q]), acc.m[p][q]);
}

// The four insertions of the leaf pair (nu, D) with U = L0 factored out:
// Xh(c1) T + L1 (S2 Xh(x) + (Xh(c2) L2 + L2 Xh(c3)) L3), S2 = L2 L3, T = L1 S2.
template <int D>
__device__ __forceinline__ M3 leaf_pair(const Geom &g, const GaugeStore &G, const double *xh, int x, const int c[4],
                                        int mu, int nu, int pl, int c1)
{
    const int V = g.V;
    const int c2 = shift(g, c, mu, 1, nu, D), c3 = shift(g, c, mu, 0, nu, D);
    const M3 L2 = dag(link(G, V, mu, c3));                          // c2 -> c3
    const M3 L3 = D == 1 ? dag(link(G, V, nu, x)) : link(G, V, nu, c3);   // c3 -> x
    const M3 S2 = mul(L2, L3);
    M3 K = zero3();
    fma_hm(load_xh(xh, V, pl, c2), L2, K);
    fma_mh(L2, load_xh(xh, V, pl, c3), K);
    K = mul(K, L3);
    fma_mh(S2, load_xh(xh, V, pl, x), K);
    const M3 L1 = D == 1 ? link(G, V, nu, c1) : dag(link(G, V, nu, c2));  // c1 -> c2
    M3 E = mul(L1, K);
    const M3 T = mul(L1, S2);
    fma_hm(load_xh(xh, V, pl, c1), T, E);
    return E;
}

// one thread per link (x, mu): F = TA(U H), canonical layout [V][4][3][3]
__global__ void __launch_bounds__(128) k_force(Geom g, GaugeStore G, const double2 *X, const double2 *Y,
                                               const double *xh, double kappa, double csw, double2 *F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    const int V = g.V;
    const int x = i % V, mu = i / V;
    int c[4];
    site_coords(g, x, c);
    M3 H = zero3();

    // clover part: H = -(i csw kappa / 4) sum_{nu, d} sigma E(nu, d)
    if (csw != 0.0) {
        M3 A = zero3();
        const int c1 = shift(g, c, mu, 1, mu, 0);
#pragma unroll 1
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            const int pl = plane_of(mu < nu ? mu : nu, mu < nu ? nu : mu);
            // d = +1 runs counter-clockwise in the (a, b) plane when mu < nu
            const double sp = mu < nu ? 1.0 : -1.0;
            const M3 Ep = leaf_pair<1>(g, G, xh, x, c, mu, nu, pl, c1);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) A.m[a][b] = A.m[a][b] + sp * Ep.m[a][b];
            const M3 Em = leaf_pair<-1>(g, G, xh, x, c, mu, nu, pl, c1);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) A.m[a][b] = A.m[a][b] - sp * Em.m[a][b];
        }
        const double beta = -csw * kappa / 4.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) H.m[a][b] = beta * times_i(A.m[a][b]);
    }

    // hopping part: H += 2 kappa p sum_s [((1-g) X(x+mu))_s Y_s(x)^+ + Y_s(x+mu) ((1+g) X(x))_s^+]
    {
        const bool wrap = c[mu] == g.L[mu] - 1;
        const int xf = wrap ? x - (g.L[mu] - 1) * g.stride[mu] : x + g.stride[mu];
        const double k2 = 2.0 * kappa * ((mu == 3 && wrap) ? (double)g.tbc : 1.0);
        M3 Z = zero3();
        cx<double> a[12], b[12];
        load_sp(X, V, xf, b);
        project_full(mu, -1, b, a);
        load_sp(Y, V, x, b);
        fma_outer(a, b, Z);
        load_sp(X, V, x, b);
        project_full(mu, +1, b, a);
        load_sp(Y, V, xf, b);
        fma_outer(b, a, Z);
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) H.m[p][q] = H.m[p][q] + k2 * Z.m[p][q];
    }

    // F = TA(U H) = (G - G^+)/2 - tr(G - G^+)/6
    const M3 Gm = mul(link(G, V, mu, x), H);
    M3 D;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) D.m[p][q] = Gm.m[p][q] - conj(Gm.m[q][p]);
    const cx<double> tr = (1.0 / 6.0) * (D.m[0][0] + D.m[1][1] + D.m[2][2]);
    double2 *out = F + ((size_t)x * 4 + mu) * 9;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            cx<double> f = 0.5 * D.m[p][q];
            if (p == q) f = f - tr;
            out[3 * p + q] = make_double2(f.re, f.im);
        }
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// F from X, Y (FP64 fields) into the canonical force layout at dst (device).
wc_status force_from_solutions(wc_lattice lat, wc_field X, wc_field Y, double2 *dst)
{
    const int V = lat->g.V;
    double *xh = nullptr;
    wc_status st = check_cuda(lat, cudaMalloc(&xh, sizeof(double) * 54 * (size_t)V), "cudaMalloc(xh)");
    if (st != WC_OK) return st;
    k_xi<<<(V + 127) / 128, 128, 0, lat->stream>>>(lat->g, static_cast<const double2 *>(X->data),
                                                   static_cast<const double2 *>(Y->data), xh);
    st = check_launch(lat, "xi");
    if (st == WC_OK) {
        k_force<<<(4 * V + 127) / 128, 128, 0, lat->stream>>>(lat->g, lat->gauge, static_cast<const double2 *>(X->data),
                                                           static_cast<const double2 *>(Y->data), xh, lat->kappa,
                                                           lat->csw, dst);
        st = check_launch(lat, "force");
    }
    cudaStreamSynchronize(lat->stream);
    cudaFree(xh);
    return st;
}

}  // namespace wc

using namespace wc;

namespace wc {
namespace {

// out = scale * F U per link (3x3 complex, canonical [4V][3][3] order)
__global__ void k_force_times_links(long long nlinks, const double2 *F, const double2 *U, double scale, double2 *out)
{
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= nlinks) return;
    const double2 *f = F + 9 * l, *u = U + 9 * l;
    cx<double> a[9], b[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        a[k] = mkc(f[k].x, f[k].y);
        b[k] = mkc(u[k].x, u[k].y);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> acc = a[3 * i] * b[j];
            acc = cfma(a[3 * i + 1], b[3 + j], acc);
            acc = cfma(a[3 * i + 2], b[6 + j], acc);
            out[9 * l + 3 * i + j] = make_double2(scale * acc.re, scale * acc.im);
        }
}

}  // namespace
}  // namespace wc

extern "C" {

wc_status wc_force_times_links(wc_lattice lat, const double *force, const double *U, double scale, double *out)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!force || !U || !out) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (!is_device_ptr(force) || !is_device_ptr(U) || !is_device_ptr(out))
        return set_error(lat, WC_ERR_ARG, "force, U and out must be device pointers");
    const long long n = 4LL * lat->g.V;
    k_force_times_links<<<(unsigned)((n + 255) / 256), 256, 0, lat->stream>>>(
        n, reinterpret_cast<const double2 *>(force), reinterpret_cast<const double2 *>(U), scale,
        reinterpret_cast<double2 *>(out));
    return check_cuda(lat, cudaGetLastError(), "force_times_links");
}

wc_status wc_action_force(wc_lattice lat, wc_field phi, double *S_out, double *force, const wc_solve_params *p)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!phi || !p || !S_out || !force) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (phi->lat != lat || phi->prec != WC_F64) return set_error(lat, WC_ERR_ARG, "phi must be an FP64 field of lat");
    wc_field X = nullptr, Y = nullptr;
    wc_status st = wc_field_create(lat, WC_F64, &Y);
    if (st == WC_OK) st = wc_field_create(lat, WC_F64, &X);
    if (st == WC_OK) st = check_solve_args(lat, Y, phi, p);
    wc_solve_info info{};
    if (st == WC_OK) st = bicgstab(lat, 1, Y, phi, *p, &info);   // M^+ Y = phi
    if (st == WC_OK) st = bicgstab(lat, 0, X, Y, *p, &info);     // M X = Y
    double S = 0.0;
    if (st == WC_OK) st = reduce_norm2(lat, Y, &S);
    if (st == WC_OK) {
        const int V = lat->g.V;
        const size_t bytes = sizeof(double2) * 36 * (size_t)V;
        if (is_device_ptr(force)) {
            st = force_from_solutions(lat, X, Y, reinterpret_cast<double2 *>(force));
        } else {
            double2 *tmp = nullptr;
            st = check_cuda(lat, cudaMalloc(&tmp, bytes), "cudaMalloc(force)");
            if (st == WC_OK) st = force_from_solutions(lat, X, Y, tmp);
            if (st == WC_OK) st = check_cuda(lat, cudaMemcpy(force, tmp, bytes, cudaMemcpyDeviceToHost), "copy force");
            cudaFree(tmp);
        }
    }
    if (st == WC_OK) *S_out = S;
    wc_field_destroy(X);
    wc_field_destroy(Y);
    return st;
}

}  // extern "C"
