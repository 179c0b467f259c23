// Pseudofermion action S = phi^+ (M^+ M)^-1 phi and its force per link.
//
// With Y solving M^+ Y = phi and X solving M X = Y, S = |Y|^2 and, for a
// link variation U_mu(x) -> exp(eps L) U_mu(x) with L in su(3),
//   dS/deps = -2 Re <Y, (dM/deps) X> = Re tr(L G_mu(x)),
// and the force is the traceless anti-Hermitian projection
//   F = TA(G) = (G - G^+)/2 - tr(G - G^+)/6.
//
// Hopping part (the forward hop at x and the backward hop at x+mu use the
// link):  G += 2 kappa p [ sum_s (U (1-g_mu) X(x+mu))_s Y_s(x)^+
//                          - sum_s ((1+g_mu) X(x))_s Y_s(x+mu)^+ U^+ ]
// (p the time-boundary factor of the hop; for M^+-free form see above).
//
// Clover part: T = i csw kappa sum_{a<b} sigma_ab (x) Fhat_ab, so
//   <Y, dT X> = sum_y sum_{a<b} (i csw kappa / 8)(tr(dQ Xi) - tr(dQ^+ Xi))
// with Xi_ab(y) the traceless part of sum_{s,t} sigma_ab[s][t] X_t(y) Y_s(y)^+
// (kernel k_xi).  For the link (x, mu) and each plaquette containing it --
// corners c0 = x, c1 = x+mu, c2 = x+mu+d nu, c3 = x+d nu (d = +-1), loop
// links L0 = U_mu(x), L1, L2, L3 in that order -- every clover leaf based at
// corner c_k contributes through W_k(Z) = L0 ... L_{k-1} Z L_k ... L3
// (k = 1..4, corner c_{k mod 4}):
//   G += -(i csw kappa / 4) sigma sum_k [W_k(Xi(c_k)) + W_k(Xi(c_k)^+)^+]
// where sigma = +1 when the loop c0 c1 c2 c3 runs counter-clockwise in the
// (a, b) = (min(mu,nu), max(mu,nu)) plane (the leaves' orientation) and -1
// when the leaves run through the link backwards.
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
__device__ void sigma_block(int plane, int blk, cx<double> s[2][2])
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

// Xi_ab(y) for the six planes, traceless part: xi[(plane*9 + 3i + j) * V + y]
__global__ void k_xi(Geom g, const double2 *X, const double2 *Y, double2 *xi)
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
    for (int pl = 0; pl < 6; ++pl) {
        M3 Z;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Z.m[i][j] = mkc(0.0, 0.0);
        for (int blk = 0; blk < 2; ++blk) {
            cx<double> sg[2][2];
            sigma_block(pl, blk, sg);
            for (int s = 0; s < 2; ++s)
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
        const cx<double> tr = (1.0 / 3.0) * (Z.m[0][0] + Z.m[1][1] + Z.m[2][2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) Z.m[i][i] = Z.m[i][i] - tr;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                xi[((size_t)pl * 9 + 3 * i + j) * V + y] = make_double2(Z.m[i][j].re, Z.m[i][j].im);
    }
}

__device__ M3 load_xi(const double2 *xi, int V, int plane, int y)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double2 v = xi[((size_t)plane * 9 + 3 * i + j) * V + y];
            r.m[i][j] = mkc(v.x, v.y);
        }
    return r;
}

// (1 + s gamma_mu) psi as a full spinor (chiral basis)
__device__ void project_full(int mu, int s, const cx<double> p[12], cx<double> o[12])
{
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

__device__ void load_sp(const double2 *f, int V, int x, cx<double> s[12])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 v = f[(size_t)k * V + x];
        s[k] = mkc(v.x, v.y);
    }
}

// one thread per link (x, mu): F = TA(G_hop + G_clover), canonical layout
__global__ void k_force(Geom g, GaugeStore G, const double2 *X, const double2 *Y, const double2 *xi,
                        double kappa, double csw, double2 *F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    const int V = g.V;
    const int x = i % V, mu = i / V;
    int c[4];
    site_coords(g, x, c);
    const M3 U = link(G, V, mu, x);
    M3 Gm;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Gm.m[a][b] = mkc(0.0, 0.0);

    // hopping part
    {
        const bool wrap = c[mu] == g.L[mu] - 1;
        const int xf = wrap ? x - (g.L[mu] - 1) * g.stride[mu] : x + g.stride[mu];
        const double ph = (mu == 3 && wrap) ? (double)g.tbc : 1.0;
        cx<double> xf_s[12], x_s[12], a[12], cpl[12], yx[12], yf[12];
        load_sp(X, V, xf, xf_s);
        load_sp(X, V, x, x_s);
        load_sp(Y, V, x, yx);
        load_sp(Y, V, xf, yf);
        project_full(mu, -1, xf_s, a);    // (1 - g) X(x+mu)
        project_full(mu, +1, x_s, cpl);   // (1 + g) X(x)
        M3 Z1, Z2;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Z1.m[p][q] = mkc(0.0, 0.0);
                Z2.m[p][q] = mkc(0.0, 0.0);
            }
        for (int s = 0; s < 4; ++s) {
            cx<double> ua[3];
            for (int p = 0; p < 3; ++p) {
                ua[p] = U.m[p][0] * a[3 * s];
                ua[p] = cfma(U.m[p][1], a[3 * s + 1], ua[p]);
                ua[p] = cfma(U.m[p][2], a[3 * s + 2], ua[p]);
            }
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    Z1.m[p][q] = Z1.m[p][q] + ua[p] * conj(yx[3 * s + q]);
                    Z2.m[p][q] = Z2.m[p][q] + cpl[3 * s + p] * conj(yf[3 * s + q]);
                }
        }
        Z2 = mul(Z2, dag(U));
        const cx<double> k2 = mkc(2.0 * kappa * ph, 0.0);
        add_scaled(Gm, k2, Z1);
        add_scaled(Gm, (-1.0) * k2, Z2);
    }

    // clover part
    if (csw != 0.0) {
        const cx<double> pref = mkc(0.0, -csw * kappa / 4.0);   // -(i csw kappa / 4)
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            const int a = mu < nu ? mu : nu, b = mu < nu ? nu : mu;
            const int pl = plane_of(a, b);
            for (int d = -1; d <= 1; d += 2) {
                const bool ccw = (d == 1) == (mu < nu);
                const double sigma = ccw ? 1.0 : -1.0;
                // corners and loop links
                const int c1 = shift(g, c, mu, 1, nu, 0);
                const int c2 = shift(g, c, mu, 1, nu, d);
                const int c3 = shift(g, c, mu, 0, nu, d);
                M3 L[4];
                L[0] = U;
                if (d == 1) {
                    L[1] = link(G, V, nu, c1);            // c1 -> c1 + nu
                    L[3] = dag(link(G, V, nu, x));        // c3 = x + nu -> x
                } else {
                    L[1] = dag(link(G, V, nu, c2));       // c1 -> c1 - nu
                    L[3] = link(G, V, nu, c3);            // c3 = x - nu -> x
                }
                L[2] = dag(link(G, V, mu, c3));           // c2 -> c3
                const int corner[4] = {x, c1, c2, c3};
                M3 pre = L[0];
                M3 suf[5];
                suf[4] = ident();
                suf[3] = L[3];
                suf[2] = mul(L[2], L[3]);
                suf[1] = mul(L[1], suf[2]);
                M3 acc;
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q) acc.m[p][q] = mkc(0.0, 0.0);
                for (int k = 1; k <= 4; ++k) {
                    // pre = L0 ... L_{k-1}, suf[k] = L_k ... L3
                    const M3 Xi = load_xi(xi, V, pl, corner[k & 3]);
                    const M3 w1 = mul(mul(pre, Xi), suf[k]);
                    const M3 w2 = dag(mul(mul(pre, dag(Xi)), suf[k]));
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int q = 0; q < 3; ++q) acc.m[p][q] = acc.m[p][q] + w1.m[p][q] + w2.m[p][q];
                    if (k < 4) pre = mul(pre, L[k]);
                }
                add_scaled(Gm, sigma * pref, acc);
            }
        }
    }

    // F = (G - G^+)/2 - tr(G - G^+)/6
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
    double2 *xi = nullptr;
    wc_status st = check_cuda(lat, cudaMalloc(&xi, sizeof(double2) * 54 * (size_t)V), "cudaMalloc(xi)");
    if (st != WC_OK) return st;
    k_xi<<<(V + 127) / 128, 128, 0, lat->stream>>>(lat->g, static_cast<const double2 *>(X->data),
                                                   static_cast<const double2 *>(Y->data), xi);
    st = check_launch(lat, "xi");
    if (st == WC_OK) {
        k_force<<<(4 * V + 63) / 64, 64, 0, lat->stream>>>(lat->g, lat->gauge, static_cast<const double2 *>(X->data),
                                                           static_cast<const double2 *>(Y->data), xi, lat->kappa,
                                                           lat->csw, dst);
        st = check_launch(lat, "force");
    }
    cudaStreamSynchronize(lat->stream);
    cudaFree(xi);
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
