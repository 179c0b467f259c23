/*
 * wc_oracle.c -- plain, slow FP64 CPU oracle for the Wilson-Clover operator.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg call it; the CUDA library never links, includes or calls
 * it, and it shares no code, header, table or constant with that library.
 *
 * Everything here is written out from the definitions of the operator, in
 * the canonical layout that the library's import/export calls also use:
 *   gauge   U[V][4][3][3]  complex (mu = x,y,z,t; row; column)
 *   spinor  psi[V][4][3]   complex (spin; colour)
 *   clover  T[V][12][12]   complex, index 3*spin + colour
 *   site    x + Lx*(y + Ly*(z + Lz*t))
 * Complex numbers cross the ABI as interleaved (re, im) doubles.
 *
 * The paper (Sec. 2) names the operator -- the even-odd/RAS preconditioned
 * Wilson-Clover matrix solved by (flexible) BiCGStab with a kappa parameter --
 * but prints none of its formulas.  The readings used here are:
 *   gamma matrices   chiral basis: gamma_k = [[0, i s_k], [-i s_k, 0]],
 *                    gamma_4 = [[0, 1], [1, 0]], s_k the Pauli matrices
 *   hopping term     (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                               + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu),
 *                    every hop across the time boundary times t_bc (+1/-1)
 *   clover term      T(x) = i csw kappa sum_{mu<nu} sigma_munu (x) Fhat_munu(x),
 *                    sigma_munu = (i/2)[gamma_mu, gamma_nu],
 *                    Fhat = (1/8)[(Q - Q^+) - (1/3) tr(Q - Q^+)],
 *                    Q = sum of the four counter-clockwise plaquette leaves
 *                    at x; plaquettes never take the fermion boundary phase
 *   operator         M = (1 + T) - kappa H
 *   RAS block solve  k minimal-residual steps of M restricted (Dirichlet) to
 *                    a block extended by delta sites per face, from zero;
 *                    only the block's core is written back.  Pinned to this
 *                    definition by dense brute force in the tests; against
 *                    the paper's own RAS variant: parity unpinned (the paper
 *                    gives no formula and its cited RAS paper is not at hand)
 *   force            S = phi^+ (M^+ M)^-1 phi, dS/deps = Re tr(Lambda G) for
 *                    U -> exp(eps Lambda) U; F = TA(G)
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Lattice geometry                                                     */
/* ------------------------------------------------------------------ */

static long vol_of(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int L[4], long s, int c[4])
{
    c[0] = (int)(s % L[0]); s /= L[0];
    c[1] = (int)(s % L[1]); s /= L[1];
    c[2] = (int)(s % L[2]); s /= L[2];
    c[3] = (int)s;
}

static long site_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* Site s + d*mu_hat (d = +1 or -1), periodic wrap.  *phase receives the
 * fermion boundary factor of this hop: t_bc when the hop crosses the time
 * boundary, else 1. */
static long neighbour(const int L[4], int tbc, long s, int mu, int d, double *phase)
{
    int c[4];
    coords_of(L, s, c);
    int n = c[mu] + d;
    double ph = 1.0;
    if (n >= L[mu]) { n -= L[mu]; if (mu == 3) ph = (double)tbc; }
    if (n < 0)      { n += L[mu]; if (mu == 3) ph = (double)tbc; }
    c[mu] = n;
    if (phase) *phase = ph;
    return site_of(L, c);
}

/* ------------------------------------------------------------------ */
/* Small complex matrices                                               */
/* ------------------------------------------------------------------ */

typedef struct { cplx m[3][3]; } su3;

static su3 m3_zero(void) { su3 r; memset(&r, 0, sizeof r); return r; }

static su3 m3_id(void)
{
    su3 r = m3_zero();
    r.m[0][0] = r.m[1][1] = r.m[2][2] = 1.0;
    return r;
}

static su3 m3_mul(su3 a, su3 b)
{
    su3 r = m3_zero();
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                r.m[i][j] += a.m[i][k] * b.m[k][j];
    return r;
}

static su3 m3_adj(su3 a)
{
    su3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            r.m[i][j] = conj(a.m[j][i]);
    return r;
}

static su3 m3_add(su3 a, su3 b)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            a.m[i][j] += b.m[i][j];
    return a;
}

static su3 m3_scale(cplx s, su3 a)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            a.m[i][j] *= s;
    return a;
}

static cplx m3_trace(su3 a) { return a.m[0][0] + a.m[1][1] + a.m[2][2]; }

static su3 link_at(const cplx *U, long s, int mu)
{
    su3 r;
    const cplx *p = U + (s * 4 + mu) * 9;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            r.m[i][j] = p[3 * i + j];
    return r;
}

/* ------------------------------------------------------------------ */
/* Dirac matrices (chiral basis)                                        */
/* ------------------------------------------------------------------ */

static void pauli(int k, cplx s[2][2])
{
    memset(s, 0, sizeof(cplx) * 4);
    if (k == 1) { s[0][1] = 1; s[1][0] = 1; }
    if (k == 2) { s[0][1] = -I; s[1][0] = I; }
    if (k == 3) { s[0][0] = 1; s[1][1] = -1; }
}

/* gamma for direction mu = 0,1,2,3 (x,y,z,t) */
static void gamma_mat(int mu, cplx g[4][4])
{
    memset(g, 0, sizeof(cplx) * 16);
    if (mu == 3) {
        g[0][2] = g[1][3] = g[2][0] = g[3][1] = 1;
        return;
    }
    cplx s[2][2];
    pauli(mu + 1, s);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            g[a][2 + b] = I * s[a][b];
            g[2 + a][b] = -I * s[a][b];
        }
}

static void m4_mul(cplx a[4][4], cplx b[4][4], cplx r[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 4; ++k) acc += a[i][k] * b[k][j];
            r[i][j] = acc;
        }
}

/* projector 1 + sign * gamma_mu */
static void projector(int mu, int sign, cplx P[4][4])
{
    cplx g[4][4];
    gamma_mat(mu, g);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            P[i][j] = (i == j ? 1.0 : 0.0) + sign * g[i][j];
}

/* sigma_munu = (i/2)(gamma_mu gamma_nu - gamma_nu gamma_mu) */
static void sigma_mat(int mu, int nu, cplx s[4][4])
{
    cplx gm[4][4], gn[4][4], a[4][4], b[4][4];
    gamma_mat(mu, gm);
    gamma_mat(nu, gn);
    m4_mul(gm, gn, a);
    m4_mul(gn, gm, b);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            s[i][j] = 0.5 * I * (a[i][j] - b[i][j]);
}

/* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 */
static void gamma5_mat(cplx g5[4][4])
{
    cplx g0[4][4], g1[4][4], g2[4][4], g3[4][4], a[4][4], b[4][4];
    gamma_mat(0, g0); gamma_mat(1, g1); gamma_mat(2, g2); gamma_mat(3, g3);
    m4_mul(g0, g1, a);
    m4_mul(a, g2, b);
    m4_mul(b, g3, g5);
}

/* out[s][a] += coef * sum_{s',b} P[s][s'] W[a][b] in[s'][b] */
static void spin_colour_add(cplx coef, cplx P[4][4], su3 W, const cplx *in, cplx *out)
{
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int t = 0; t < 4; ++t) {
                if (P[s][t] == 0) continue;
                cplx wv = 0;
                for (int b = 0; b < 3; ++b) wv += W.m[a][b] * in[3 * t + b];
                acc += P[s][t] * wv;
            }
            out[3 * s + a] += coef * acc;
        }
}

/* ------------------------------------------------------------------ */
/* Clover term                                                          */
/* ------------------------------------------------------------------ */

/* A path step is +(mu+1) (hop forward in mu: multiply by U_mu(y), move to
 * y+mu) or -(mu+1) (move to y-mu, multiply by U_mu(y-mu)^+). */
static void leaf_steps(int mu, int nu, int leaf, int st[4])
{
    int pm = mu + 1, pn = nu + 1;
    switch (leaf) {
    case 0: st[0] = pm;  st[1] = pn;  st[2] = -pm; st[3] = -pn; break;
    case 1: st[0] = pn;  st[1] = -pm; st[2] = -pn; st[3] = pm;  break;
    case 2: st[0] = -pm; st[1] = -pn; st[2] = pm;  st[3] = pn;  break;
    default: st[0] = -pn; st[1] = pm; st[2] = pn;  st[3] = -pm; break;
    }
}

/* The link factor of one step taken from site *y; advances *y.
 * *link_site / *link_mu identify the link, *dag whether it enters daggered. */
static su3 step_factor(const int L[4], const cplx *U, long *y, int step,
                       long *link_site, int *link_mu, int *dag)
{
    int mu = abs(step) - 1;
    if (step > 0) {
        *link_site = *y; *link_mu = mu; *dag = 0;
        su3 f = link_at(U, *y, mu);
        *y = neighbour(L, 1, *y, mu, +1, NULL);
        return f;
    }
    long yb = neighbour(L, 1, *y, mu, -1, NULL);
    *link_site = yb; *link_mu = mu; *dag = 1;
    *y = yb;
    return m3_adj(link_at(U, yb, mu));
}

static su3 clover_leaf_sum(const int L[4], const cplx *U, long x, int mu, int nu)
{
    su3 Q = m3_zero();
    for (int leaf = 0; leaf < 4; ++leaf) {
        int st[4];
        leaf_steps(mu, nu, leaf, st);
        long y = x, ls; int lm, dg;
        su3 P = m3_id();
        for (int j = 0; j < 4; ++j)
            P = m3_mul(P, step_factor(L, U, &y, st[j], &ls, &lm, &dg));
        Q = m3_add(Q, P);
    }
    return Q;
}

/* Fhat = (1/8)[(Q - Q^+) - (1/3) tr(Q - Q^+) 1] */
static su3 field_strength(const int L[4], const cplx *U, long x, int mu, int nu)
{
    su3 Q = clover_leaf_sum(L, U, x, mu, nu);
    su3 D = m3_add(Q, m3_scale(-1.0, m3_adj(Q)));
    cplx tr = m3_trace(D) / 3.0;
    for (int i = 0; i < 3; ++i) D.m[i][i] -= tr;
    return m3_scale(0.125, D);
}

static void clover_site(const int L[4], double csw, double kappa, const cplx *U,
                        long x, cplx T[144])
{
    memset(T, 0, sizeof(cplx) * 144);
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            su3 F = field_strength(L, U, x, mu, nu);
            cplx sg[4][4];
            sigma_mat(mu, nu, sg);
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            T[(3 * s + a) * 12 + 3 * t + b] +=
                                I * csw * kappa * sg[s][t] * F.m[a][b];
        }
}

/* ------------------------------------------------------------------ */
/* Operator                                                             */
/* ------------------------------------------------------------------ */

/* (H psi)(x), gather form */
static void hop_site(const int L[4], int tbc, const cplx *U, const cplx *psi, long x,
                     cplx out[12])
{
    memset(out, 0, sizeof(cplx) * 12);
    for (int mu = 0; mu < 4; ++mu) {
        cplx Pm[4][4], Pp[4][4];
        projector(mu, -1, Pm);
        projector(mu, +1, Pp);
        double pf, pb;
        long xf = neighbour(L, tbc, x, mu, +1, &pf);
        long xb = neighbour(L, tbc, x, mu, -1, &pb);
        spin_colour_add(pf, Pm, link_at(U, x, mu), psi + 12 * xf, out);
        spin_colour_add(pb, Pp, m3_adj(link_at(U, xb, mu)), psi + 12 * xb, out);
    }
}

/* (M psi)(x) = psi(x) + T(x) psi(x) - kappa (H psi)(x) */
static void apply_M_site(const int L[4], int tbc, double kappa, double csw,
                         const cplx *U, const cplx *T, const cplx *psi, long x,
                         cplx out[12])
{
    cplx h[12], Tl[144];
    const cplx *Tx = T ? T + 144 * x : Tl;
    if (!T) clover_site(L, csw, kappa, U, x, Tl);
    hop_site(L, tbc, U, psi, x, h);
    const cplx *in = psi + 12 * x;
    for (int i = 0; i < 12; ++i) {
        cplx acc = in[i];
        for (int j = 0; j < 12; ++j) acc += Tx[12 * i + j] * in[j];
        out[i] = acc - kappa * h[i];
    }
}

/* ------------------------------------------------------------------ */
/* Exported entry points                                               */
/* ------------------------------------------------------------------ */

long orc_volume(const int L[4]) { return vol_of(L); }

/* gamma_mu (mu = 0..3) or gamma_5 (mu = 4) as 16 complex, row-major */
void orc_gamma(int mu, double *out)
{
    cplx g[4][4];
    if (mu == 4) gamma5_mat(g); else gamma_mat(mu, g);
    memcpy(out, g, sizeof g);
}

/* Clover term T at every site: T[V][12][12]. */
void orc_clover_field(const int L[4], double csw, double kappa, const double *U,
                      double *T)
{
    long V = vol_of(L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        clover_site(L, csw, kappa, (const cplx *)U, x, (cplx *)T + 144 * x);
}

/* Sum of the clover leaves Q_munu(x) (3x3 complex), exported for tests. */
void orc_leaf_sum(const int L[4], const double *U, long x, int mu, int nu, double *Q)
{
    su3 q = clover_leaf_sum(L, (const cplx *)U, x, mu, nu);
    memcpy(Q, q.m, sizeof q.m);
}

/* out = H psi over all sites (nsites < 0) or at the listed sites only
 * (out then holds nsites spinors in list order). */
void orc_apply_hop(const int L[4], int tbc, const double *U, const double *psi,
                   double *out, long nsites, const long *sites)
{
    long n = nsites < 0 ? vol_of(L) : nsites;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        long x = nsites < 0 ? i : sites[i];
        hop_site(L, tbc, (const cplx *)U, (const cplx *)psi, x, (cplx *)out + 12 * i);
    }
}

/* out = M psi over all sites (nsites < 0) or at the listed sites.  T may be
 * NULL: the clover term is then rebuilt at each site from U and csw. */
void orc_apply_M(const int L[4], int tbc, double kappa, double csw, const double *U,
                 const double *T, const double *psi, double *out, long nsites,
                 const long *sites)
{
    long n = nsites < 0 ? vol_of(L) : nsites;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        long x = nsites < 0 ? i : sites[i];
        apply_M_site(L, tbc, kappa, csw, (const cplx *)U, (const cplx *)T,
                     (const cplx *)psi, x, (cplx *)out + 12 * i);
    }
}

/* out = M^+ psi, written independently of orc_apply_M: every block of M
 * (row x, column y) is conjugate-transposed explicitly and scattered into
 * row y.  Serial (the scatter would race under threads). */
void orc_apply_Mdag(const int L[4], int tbc, double kappa, const double *U_,
                    const double *T_, const double *psi_, double *out_)
{
    const cplx *U = (const cplx *)U_, *T = (const cplx *)T_, *psi = (const cplx *)psi_;
    cplx *out = (cplx *)out_;
    long V = vol_of(L);
    memset(out, 0, sizeof(cplx) * 12 * V);
    for (long x = 0; x < V; ++x) {
        /* diagonal block 1 + T(x): adjoint is 1 + T(x)^+ */
        const cplx *in = psi + 12 * x;
        for (int i = 0; i < 12; ++i) {
            cplx acc = in[i];
            for (int j = 0; j < 12; ++j) acc += conj(T[144 * x + 12 * j + i]) * in[j];
            out[12 * x + i] += acc;
        }
    }
    for (long x = 0; x < V; ++x) {
        for (int mu = 0; mu < 4; ++mu) {
            for (int d = -1; d <= 1; d += 2) {
                /* block of -kappa*H at (row x, column y = x + d mu) */
                double ph;
                long y = neighbour(L, tbc, x, mu, d, &ph);
                cplx P[4][4], Pa[4][4];
                projector(mu, d > 0 ? -1 : +1, P);
                su3 W = d > 0 ? link_at(U, x, mu) : m3_adj(link_at(U, y, mu));
                for (int i = 0; i < 4; ++i)
                    for (int j = 0; j < 4; ++j) Pa[i][j] = conj(P[j][i]);
                /* adjoint block (row y, column x) acts on psi(x) */
                spin_colour_add(-kappa * ph, Pa, m3_adj(W), psi + 12 * x, out + 12 * y);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Overlapped RAS with minimal-residual block solves                    */
/* ------------------------------------------------------------------ */

/* z = sum_i Rtilde_i^T MR_k(A_i, R_i^delta v).  Blocks b[mu] tile the
 * lattice from the origin; each is extended by delta sites per face
 * (periodic).  A_i is M on the extended block with hops leaving it dropped.
 * Returns 0, or -1 when the block shape does not fit the lattice. */
int orc_ras(const int L[4], int tbc, double kappa, const double *U_, const double *T_,
            const int b[4], int delta, int k, const double *v_, double *z_)
{
    const cplx *U = (const cplx *)U_, *T = (const cplx *)T_, *v = (const cplx *)v_;
    cplx *z = (cplx *)z_;
    int nb[4], e[4];
    for (int mu = 0; mu < 4; ++mu) {
        if (b[mu] <= 0 || L[mu] % b[mu] != 0 || L[mu] <= b[mu] + 2 * delta || delta < 0)
            return -1;
        nb[mu] = L[mu] / b[mu];
        e[mu] = b[mu] + 2 * delta;
    }
    long ne = (long)e[0] * e[1] * e[2] * e[3];
    long nblocks = (long)nb[0] * nb[1] * nb[2] * nb[3];

#pragma omp parallel
    {
        cplx *r = malloc(sizeof(cplx) * 12 * ne);
        cplx *q = malloc(sizeof(cplx) * 12 * ne);
        cplx *xs = malloc(sizeof(cplx) * 12 * ne);
        long *gsite = malloc(sizeof(long) * ne);
        int *gt = malloc(sizeof(int) * ne);
#pragma omp for schedule(dynamic)
        for (long ib = 0; ib < nblocks; ++ib) {
            int bc[4];
            coords_of(nb, ib, bc);
            /* global site of every local (extended) site */
            for (long l = 0; l < ne; ++l) {
                int lc[4], g[4];
                coords_of(e, l, lc);
                for (int mu = 0; mu < 4; ++mu)
                    g[mu] = ((bc[mu] * b[mu] - delta + lc[mu]) % L[mu] + L[mu]) % L[mu];
                gsite[l] = site_of(L, g);
                gt[l] = g[3];
            }
            for (long l = 0; l < ne; ++l)
                for (int i = 0; i < 12; ++i) {
                    r[12 * l + i] = v[12 * gsite[l] + i];
                    xs[12 * l + i] = 0;
                }
            for (int it = 0; it < k; ++it) {
                /* q = A_i r */
                for (long l = 0; l < ne; ++l) {
                    long gx = gsite[l];
                    cplx *ql = q + 12 * l;
                    const cplx *rl = r + 12 * l;
                    for (int i = 0; i < 12; ++i) {
                        cplx acc = rl[i];
                        for (int j = 0; j < 12; ++j) acc += T[144 * gx + 12 * i + j] * rl[j];
                        ql[i] = acc;
                    }
                    cplx h[12];
                    memset(h, 0, sizeof h);
                    int lc[4];
                    coords_of(e, l, lc);
                    for (int mu = 0; mu < 4; ++mu) {
                        cplx Pm[4][4], Pp[4][4];
                        projector(mu, -1, Pm);
                        projector(mu, +1, Pp);
                        if (lc[mu] + 1 < e[mu]) {
                            int c2[4] = {lc[0], lc[1], lc[2], lc[3]};
                            c2[mu] += 1;
                            long lf = site_of(e, c2);
                            double ph = (mu == 3 && gt[l] == L[3] - 1) ? (double)tbc : 1.0;
                            spin_colour_add(ph, Pm, link_at(U, gx, mu), r + 12 * lf, h);
                        }
                        if (lc[mu] - 1 >= 0) {
                            int c2[4] = {lc[0], lc[1], lc[2], lc[3]};
                            c2[mu] -= 1;
                            long lb = site_of(e, c2);
                            double ph = (mu == 3 && gt[l] == 0) ? (double)tbc : 1.0;
                            spin_colour_add(ph, Pp, m3_adj(link_at(U, gsite[lb], mu)),
                                            r + 12 * lb, h);
                        }
                    }
                    for (int i = 0; i < 12; ++i) ql[i] -= kappa * h[i];
                }
                /* alpha = <q, r> / <q, q> */
                cplx qr = 0;
                double qq = 0;
                for (long i = 0; i < 12 * ne; ++i) {
                    qr += conj(q[i]) * r[i];
                    qq += creal(conj(q[i]) * q[i]);
                }
                cplx alpha = qq > 0 ? qr / qq : 0;
                for (long i = 0; i < 12 * ne; ++i) {
                    xs[i] += alpha * r[i];
                    r[i] -= alpha * q[i];
                }
            }
            /* restricted prolongation: write the core only */
            for (long l = 0; l < ne; ++l) {
                int lc[4], core = 1;
                coords_of(e, l, lc);
                for (int mu = 0; mu < 4; ++mu)
                    if (lc[mu] < delta || lc[mu] >= delta + b[mu]) core = 0;
                if (core)
                    for (int i = 0; i < 12; ++i) z[12 * gsite[l] + i] = xs[12 * l + i];
            }
        }
        free(r); free(q); free(xs); free(gsite); free(gt);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Pseudofermion force                                                  */
/* ------------------------------------------------------------------ */

/* For S = phi^+ (M^+M)^-1 phi with X = (M^+M)^-1 phi and Y = M X:
 *   dS = -2 Re <Y, dM X>.
 * For U_mu(x) -> exp(eps Lambda) U_mu(x) this accumulates G with
 * dS/deps = Re tr(Lambda G) and returns F = TA(G) per link
 * (F[V][4][3][3]).  With hop_only != 0 the clover part is skipped. */
void orc_force(const int L[4], int tbc, double kappa, double csw, const double *U_,
               const double *X_, const double *Y_, double *F_, int hop_only)
{
    const cplx *U = (const cplx *)U_, *X = (const cplx *)X_, *Y = (const cplx *)Y_;
    long V = vol_of(L);
    su3 *G = calloc((size_t)V * 4, sizeof(su3));

    /* hopping part: the forward hop at x and the backward hop at x+mu */
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            double ph;
            long xf = neighbour(L, tbc, x, mu, +1, &ph);
            su3 Ux = link_at(U, x, mu);
            cplx Pm[4][4], Pp[4][4];
            projector(mu, -1, Pm);
            projector(mu, +1, Pp);
            cplx a[12], c[12];
            memset(a, 0, sizeof a);
            memset(c, 0, sizeof c);
            su3 one = m3_id();
            spin_colour_add(1.0, Pm, Ux, X + 12 * xf, a);   /* U (1-g) X(x+mu) */
            spin_colour_add(1.0, Pp, one, X + 12 * x, c);   /* (1+g) X(x) */
            su3 Z1 = m3_zero(), Z2 = m3_zero();
            for (int s = 0; s < 4; ++s)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        Z1.m[i][j] += a[3 * s + i] * conj(Y[12 * x + 3 * s + j]);
                        Z2.m[i][j] += c[3 * s + i] * conj(Y[12 * xf + 3 * s + j]);
                    }
            Z2 = m3_mul(Z2, m3_adj(Ux));
            G[4 * x + mu] = m3_add(G[4 * x + mu],
                                   m3_scale(2.0 * kappa * ph, m3_add(Z1, m3_scale(-1.0, Z2))));
        }

    if (!hop_only) {
        /* clover part: every leaf of every plaquette clover that holds the link */
        const cplx c = I * csw * kappa / 8.0;
        for (long y = 0; y < V; ++y)
            for (int mu = 0; mu < 4; ++mu)
                for (int nu = mu + 1; nu < 4; ++nu) {
                    cplx sg[4][4];
                    sigma_mat(mu, nu, sg);
                    /* Xi = sum_{s,t} sigma[s][t] X_t(y) Y_s(y)^+, traceless part */
                    su3 Xi = m3_zero();
                    for (int s = 0; s < 4; ++s)
                        for (int t = 0; t < 4; ++t)
                            for (int i = 0; i < 3; ++i)
                                for (int j = 0; j < 3; ++j)
                                    Xi.m[i][j] += sg[s][t] * X[12 * y + 3 * t + i] *
                                                  conj(Y[12 * y + 3 * s + j]);
                    cplx tr = m3_trace(Xi) / 3.0;
                    for (int i = 0; i < 3; ++i) Xi.m[i][i] -= tr;
                    for (int leaf = 0; leaf < 4; ++leaf) {
                        int st[4];
                        leaf_steps(mu, nu, leaf, st);
                        su3 fac[4];
                        long ls[4]; int lm[4], dg[4];
                        long w = y;
                        for (int j = 0; j < 4; ++j)
                            fac[j] = step_factor(L, U, &w, st[j], &ls[j], &lm[j], &dg[j]);
                        for (int j = 0; j < 4; ++j) {
                            su3 A = m3_id(), B = m3_id();
                            for (int m = 0; m < j; ++m) A = m3_mul(A, fac[m]);
                            for (int m = j + 1; m < 4; ++m) B = m3_mul(B, fac[m]);
                            su3 Ul = link_at(U, ls[j], lm[j]);
                            su3 W;
                            if (!dg[j]) {
                                /* leaf = A U B: W = U B Xi A + A^+ Xi B^+ U^+, G -= 2cW */
                                W = m3_add(m3_mul(m3_mul(m3_mul(Ul, B), Xi), A),
                                           m3_mul(m3_mul(m3_mul(m3_adj(A), Xi), m3_adj(B)),
                                                  m3_adj(Ul)));
                                W = m3_scale(-2.0 * c, W);
                            } else {
                                /* leaf = A U^+ B: W = B Xi A U^+ + U A^+ Xi B^+, G += 2cW */
                                W = m3_add(m3_mul(m3_mul(m3_mul(B, Xi), A), m3_adj(Ul)),
                                           m3_mul(m3_mul(m3_mul(Ul, m3_adj(A)), Xi),
                                                  m3_adj(B)));
                                W = m3_scale(2.0 * c, W);
                            }
                            G[4 * ls[j] + lm[j]] = m3_add(G[4 * ls[j] + lm[j]], W);
                        }
                    }
                }
    }

    /* F = TA(G) = (G - G^+)/2 - (1/6) tr(G - G^+) 1 */
    cplx *F = (cplx *)F_;
    for (long l = 0; l < 4 * V; ++l) {
        su3 D = m3_add(G[l], m3_scale(-1.0, m3_adj(G[l])));
        cplx tr = m3_trace(D) / 6.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                F[9 * l + 3 * i + j] = 0.5 * D.m[i][j] - (i == j ? tr : 0.0);
    }
    free(G);
}
