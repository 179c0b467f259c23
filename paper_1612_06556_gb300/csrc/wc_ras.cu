// Overlapped Restricted Additive Schwarz preconditioner with minimal-residual
// block solves solved inside CTAs (Sec. 2: the paper's single-precision
// solver is preconditioned by even-odd site ordering and by overlapped RAS).
//
//   z = sum_i Rtilde_i^T MR_k(A_i, R_i^delta v)
//
// Block i: core b[0]xb[1]xb[2]xb[3] sites tiled from the origin, extended by
// delta sites on every face (periodic) to e[mu] = b[mu] + 2 delta.  A_i is M
// restricted to the extended block: hops whose target lies outside it are
// dropped (Dirichlet cut); the time-boundary factor still applies to hops
// inside the block that cross t = Lt-1 -> 0.  MR_k: x = 0, r = v on the
// block, then k times q = A_i r, alpha = <q, r>/<q, q>, x += alpha r,
// r -= alpha q (alpha = 0 when q = 0).  Only the core of x is written.
//
// Two GB300 mappings:
//
// k_ras_cluster (FP32 storage, whenever the block fits): one extended block
// per cluster of two CTAs on two SMs, split in half along t, one site per
// thread.  Each CTA stages its half of the block once per application in
// shared memory -- the residual r and the links U_mu(x) of its sites (12
// reals each) -- so the k MR sweeps read links from shared memory instead
// of re-fetching them from L2 every sweep.  A site's backward link
// U_mu(x - mu) is the link of a site inside the extended block whenever the
// hop is kept, so the block's own links are all that is needed.  Hops that
// cross the split (forward in t from the last slice of CTA 0, backward in t
// from the first slice of CTA 1) read the neighbour's r and link from the
// other CTA's shared memory (distributed shared memory).  alpha is summed
// from per-warp FP32 partials of both CTAs in one fixed order, so both CTAs
// get the same alpha; two cluster barriers per MR step (after the partial
// sums, after the r update).  The clover term (72 reals per site) does not
// fit beside r and the links and is read from global memory.
//
// k_ras (FP16 storage, and block shapes the cluster kernel does not take:
// odd extended t extent, more than 1344 sites): one CTA per block, two
// sites per thread, r and the core of x in shared memory, links and clover
// from global memory every sweep.  On FP16 storage it measured faster than
// the cluster kernel with the block's FP16 links and clover staged in
// shared memory (1.03 against 1.08 ms at 24^3x32): both are bound by
// instruction issue, not by the L2 reads the staging removes.
//
// Arithmetic is FP32 on FP32 and FP16 storage; <q, r> and <q, q> are summed
// in FP32 (GB300's FP64 pipe runs at 1/64 of the FP32 rate, and alpha only
// steers a preconditioner).
#include <cooperative_groups.h>

#include <algorithm>

#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

constexpr int kRasSPT = 2;         // sites per thread
constexpr int kRasMaxThreads = 672;

struct RasGeom {
    int e[4];       // extended extents
    int es[4];      // local strides 1, e0, e0 e1, e0 e1 e2
    int b[4];       // core extents
    int nb[4];      // blocks per direction
    int ne;         // sites of an extended block
    int ncore;      // sites of a core
    int delta;
    int k;          // MR iterations
};

// alpha = <q, r> / <q, q> from per-thread FP32 partials: lanes are summed
// by warp shuffles, the warp sums are published in shared memory and every
// warp then adds them in the same fixed order, so all threads get the same
// alpha after a single barrier.  FP32 throughout: the FP64 pipe of GB300
// runs at 1/64 of the FP32 rate, and alpha only steers a preconditioner.
__device__ __forceinline__ cx<float> block_alpha(const float v[3], float *sm /*[32*3]*/)
{
    float w[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w[i] += __shfl_xor_sync(0xffffffffu, w[i], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 3; ++i) sm[wid * 3 + i] = w[i];
    __syncthreads();
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        t[i] = lane < nw ? sm[lane * 3 + i] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[i] += __shfl_xor_sync(0xffffffffu, t[i], o);
    }
    return t[2] > 0.f ? mkc(t[0] / t[2], t[1] / t[2]) : mkc(0.f, 0.f);
}

// Spinors in shared memory are float4 planes [6][n] paired by colour:
// plane 2c holds spins 0 and 1 of colour c, plane 2c+1 spins 2 and 3
// (component k = 3 spin + colour).  A spin projection of colour c is then
// two 16-byte accesses, a clover block (spins 0,1 or 2,3) three, and a
// warp's access to one plane is contiguous (conflict-free).
__device__ __forceinline__ void sm_load(const float4 *a, int n, int i, cx<float> s[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 v = a[(2 * c) * n + i], w = a[(2 * c + 1) * n + i];
        s[c] = mkc(v.x, v.y);
        s[3 + c] = mkc(v.z, v.w);
        s[6 + c] = mkc(w.x, w.y);
        s[9 + c] = mkc(w.z, w.w);
    }
}

__device__ __forceinline__ void sm_store(float4 *a, int n, int i, const cx<float> s[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[(2 * c) * n + i] = make_float4(s[c].re, s[c].im, s[3 + c].re, s[3 + c].im);
        a[(2 * c + 1) * n + i] = make_float4(s[6 + c].re, s[6 + c].im, s[9 + c].re, s[9 + c].im);
    }
}

// spins 2b, 2b+1 (clover block b) of site i: v[3 s_local + c]
__device__ __forceinline__ void sm_load_block(const float4 *a, int n, int i, int b, cx<float> v[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 t = a[(2 * c + b) * n + i];
        v[c] = mkc(t.x, t.y);
        v[3 + c] = mkc(t.z, t.w);
    }
}

template <int MU, int S>
__device__ __forceinline__ void project_sm(const float4 *a, int n, int i, cx<float> h[6])
{
    project_from<MU, S, float>(
        [&](int c, cx<float> &u0, cx<float> &u1, cx<float> &d0, cx<float> &d1) {
            const float4 v = a[(2 * c) * n + i], w = a[(2 * c + 1) * n + i];
            u0 = mkc(v.x, v.y);
            u1 = mkc(v.z, v.w);
            d0 = mkc(w.x, w.y);
            d1 = mkc(w.z, w.w);
        },
        h);
}

// q += -kappa * (forward and backward hop in direction MU), both dropped
// when their target leaves the extended block.  SF = -1 for M (forward
// projector 1 - gamma), +1 for M^+ = gamma5 M gamma5.
template <class P, int MU, int SF>
__device__ __forceinline__ void ras_hops(const Geom &g, const RasGeom &rg, const GaugeStore &U, const float4 *r,
                                         int l, int site, unsigned lpack, unsigned wbits, float mk, cx<float> q[12])
{
    const int lm = (lpack >> (8 * MU)) & 255u;
    const int stl = rg.es[MU];
    if (lm + 1 < rg.e[MU]) {
        const float coef = (MU == 3 && (wbits & (16u << 3))) ? mk * (float)g.tbc : mk;
        cx<float> h[6], u[6], r2[3], w[6];
        project_sm<MU, SF>(r, rg.ne, wc_idx(l + stl, rg.ne), h);
        P::load_link(U, g.V, MU, site, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(q, w);
    }
    if (lm >= 1) {
        const int sb = wc_idx((wbits & (1u << MU)) ? site + (g.L[MU] - 1) * g.stride[MU] : site - g.stride[MU], g.V);
        const float coef = (MU == 3 && (wbits & (1u << 3))) ? mk * (float)g.tbc : mk;
        cx<float> h[6], u[6], r2[3], w[6];
        project_sm<MU, -SF>(r, rg.ne, wc_idx(l - stl, rg.ne), h);
        P::load_link(U, g.V, MU, sb, u, r2);
        su3_adj_mul(u, r2, h, coef, w);
        reconstruct_add<MU, -SF>(q, w);
    }
}

template <class P, int SF>
__global__ void __launch_bounds__(kRasMaxThreads, 1)
    k_ras(Geom g, RasGeom rg, GaugeStore U, CloverStore C, const void *vin, const float *vin_nrm, void *zout,
          float *zout_nrm, float kappa)
{
    extern __shared__ float4 smem_raw[];
    float4 *r = smem_raw;                                            // [6][ne]
    float4 *qs = r + 6 * rg.ne;                                      // [6][blockDim.x]
    float4 *xc = qs + 6 * blockDim.x;                                // [6][ncore]
    __shared__ float red[32 * 3];
    if (kChecked) {   // every slot read before it is written shows up as NaN
        const float nan = __int_as_float(0x7fc00000);
        for (int q = threadIdx.x; q < 6 * (rg.ne + (int)blockDim.x + rg.ncore); q += blockDim.x)
            r[q] = make_float4(nan, nan, nan, nan);
        __syncthreads();
    }

    // block origin
    int bc[4];
    {
        int ib = blockIdx.x;
        bc[0] = ib % rg.nb[0];
        ib /= rg.nb[0];
        bc[1] = ib % rg.nb[1];
        ib /= rg.nb[1];
        bc[2] = ib % rg.nb[2];
        bc[3] = ib / rg.nb[2];
    }
    const int V = g.V;

    // per-thread sites: global site, packed local coordinates (8 bits per
    // direction), boundary bits (bit mu: global coordinate 0, bit 4+mu:
    // global coordinate L-1) and core index (-1 outside the core)
    int gs[kRasSPT], core[kRasSPT];
    unsigned lpack[kRasSPT], wbits[kRasSPT];
#pragma unroll
    for (int j = 0; j < kRasSPT; ++j) {
        const int l = threadIdx.x + j * blockDim.x;
        gs[j] = -1;
        core[j] = -1;
        lpack[j] = 0u;
        wbits[j] = 0u;
        if (l < rg.ne) {
            int t = l, site = 0, ci = 0, cs = 1;
            bool in_core = true;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int lm = t % rg.e[m];
                t /= rg.e[m];
                lpack[j] |= (unsigned)lm << (8 * m);
                int gm = bc[m] * rg.b[m] - rg.delta + lm;
                gm = gm < 0 ? gm + g.L[m] : (gm >= g.L[m] ? gm - g.L[m] : gm);
                site += gm * g.stride[m];
                if (gm == 0) wbits[j] |= 1u << m;
                if (gm == g.L[m] - 1) wbits[j] |= 16u << m;
                const int cm = lm - rg.delta;
                if (cm < 0 || cm >= rg.b[m]) in_core = false;
                ci += cm * cs;
                cs *= rg.b[m];
            }
            gs[j] = wc_idx(site, g.V);
            if (in_core) core[j] = wc_idx(ci, rg.ncore);
            // r = R v, x = 0
            cx<float> sp[12];
            P::load_spinor(vin, vin_nrm, V, site, sp);
            sm_store(r, rg.ne, l, sp);
            if (in_core)
#pragma unroll
                for (int j = 0; j < 6; ++j) xc[j * rg.ncore + ci] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();

    const float mk = -kappa;
    const int nt = blockDim.x;
    for (int it = 0; it < rg.k; ++it) {
        cx<float> q[12];   // q of this thread's last valid site
        float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < kRasSPT; ++j) {
            const int l = threadIdx.x + j * nt;
            if (gs[j] < 0) continue;
            if (j > 0 && gs[0] >= 0) sm_store(qs, nt, threadIdx.x, q);   // park the first site's q
            // q = A r_l - kappa (hops inside the extended block)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                cx<float> rl[6];
                sm_load_block(r, rg.ne, l, b, rl);
                float cl[36];
                P::load_clover(C, V, gs[j], b, cl);
                clover_block_mul(cl, rl, q + 6 * b);
            }
            // one direction at a time (not unrolled): bounds the registers
            // the scheduler spends on loads in flight
#pragma unroll 1
            for (int mu = 0; mu < 4; ++mu) {
                switch (mu) {
                case 0: ras_hops<P, 0, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q); break;
                case 1: ras_hops<P, 1, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q); break;
                case 2: ras_hops<P, 2, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q); break;
                default: ras_hops<P, 3, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q); break;
                }
            }
            cx<float> rl[12];
            sm_load(r, rg.ne, l, rl);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[0] = fmaf(q[k].re, rl[k].re, fmaf(q[k].im, rl[k].im, acc[0]));    // Re <q, r>
                acc[1] = fmaf(q[k].re, rl[k].im, fmaf(-q[k].im, rl[k].re, acc[1]));   // Im <q, r>
                acc[2] = fmaf(q[k].re, q[k].re, fmaf(q[k].im, q[k].im, acc[2]));
            }
        }
        // contains __syncthreads: every read of r is done after it
        const cx<float> alpha = block_alpha(acc, red);
        // x += alpha r, r -= alpha q on this thread's sites
#pragma unroll
        for (int j = 0; j < kRasSPT; ++j) {
            const int l = threadIdx.x + j * nt;
            if (gs[j] < 0) continue;
            const bool last = (j == kRasSPT - 1) || gs[kRasSPT - 1] < 0;
            cx<float> rk[12], qk[12];
            sm_load(r, rg.ne, l, rk);
            if (last) {
#pragma unroll
                for (int k = 0; k < 12; ++k) qk[k] = q[k];
            } else {
                sm_load(qs, nt, threadIdx.x, qk);
            }
            if (core[j] >= 0) {
                cx<float> xk[12];
                sm_load(xc, rg.ncore, core[j], xk);
#pragma unroll
                for (int k = 0; k < 12; ++k) xk[k] = cfma(alpha, rk[k], xk[k]);
                sm_store(xc, rg.ncore, core[j], xk);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) rk[k] = rk[k] - alpha * qk[k];
            sm_store(r, rg.ne, l, rk);
        }
        __syncthreads();
    }

    // restricted prolongation: the core of x
#pragma unroll
    for (int j = 0; j < kRasSPT; ++j) {
        if (core[j] < 0) continue;
        cx<float> sp[12];
        sm_load(xc, rg.ncore, core[j], sp);
        P::store_spinor(zout, zout_nrm, V, gs[j], sp);
    }
}


// ------------------------------------------------------------------------
// cluster kernel: one extended block per pair of CTAs
// ------------------------------------------------------------------------

constexpr int kRasCSmemMax = 226 * 1024;   // dynamic; the static 384 bytes fit beside it

// Shared-memory images of links and clover of the sites of one CTA: the
// same plane-major formats as global memory, with planes of np sites.
template <class P>
struct RasLinks;

template <>
struct RasLinks<P32> {
    static constexpr int kBytes = 4 * 3 * 16;   // per site: float4 [4 mu][3]
    static __device__ __forceinline__ void stage(void *sm, int np, int i, const GaugeStore &U, int V, int site)
    {
        float4 *d = static_cast<float4 *>(sm);
#pragma unroll
        for (int p = 0; p < 12; ++p) d[p * np + i] = __ldg(U.u32 + (size_t)p * V + site);
    }
    static __device__ __forceinline__ void load(const void *sm, int np, int mu, int i, cx<float> a[6], cx<float> c[3])
    {
        const float4 *s = static_cast<const float4 *>(sm) + mu * 3 * np + i;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float4 v = s[j * np];
            a[2 * j] = mkc(v.x, v.y);
            a[2 * j + 1] = mkc(v.z, v.w);
        }
        reconstruct_row2(a, c);
    }
};

// y = s y + B v for one packed Hermitian 6x6 clover block whose 18 complex
// pairs are produced one at a time by fetch(p) (p = 0..2: the diagonal
// reals 2p, 2p+1; p = 3..17: lower entry p - 3 in row order), consumed as
// they arrive so that the 36 reals are never live together
// (accumulating form: y = s y + B v)
template <class Fetch>
__device__ __forceinline__ void clover_block_stream(Fetch fetch, const cx<float> v[6], cx<float> y[6], float s)
{
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const float2 d = fetch(p);
        y[2 * p] = mkc(fmaf(d.x, v[2 * p].re, s * y[2 * p].re), fmaf(d.x, v[2 * p].im, s * y[2 * p].im));
        y[2 * p + 1] =
            mkc(fmaf(d.y, v[2 * p + 1].re, s * y[2 * p + 1].re), fmaf(d.y, v[2 * p + 1].im, s * y[2 * p + 1].im));
    }
    int k = 3;
#pragma unroll
    for (int a = 1; a < 6; ++a) {
#pragma unroll
        for (int b = 0; b < a; ++b) {
            const float2 e = fetch(k++);
            const cx<float> l = mkc(e.x, e.y);
            y[a] = cfma(l, v[b], y[a]);        // lower entry (a, b)
            y[b] = cfma_conj(l, v[a], y[b]);   // its mirror (b, a) = conj(l)
        }
    }
}

// FP32 clover block b of global site x
__device__ __forceinline__ void clover32_mul(const CloverStore &C, int V, int x, int b, const cx<float> v[6],
                                             cx<float> y[6], float s)
{
    const float4 *p0 = C.c32 + (size_t)b * 9 * V + x;
    clover_block_stream(
        [&](int p) {
            const float4 c = __ldg(p0 + (size_t)(p >> 1) * V);
            return (p & 1) ? make_float2(c.z, c.w) : make_float2(c.x, c.y);
        },
        v, y, s);
}

// q[c], q[3+c], q[6+c], q[9+c] += the spin reconstruction of the two-spinor
// components (w0, w1) of colour c (the per-colour form of reconstruct_add)
template <int MU, int S>
__device__ __forceinline__ void reconstruct_add_colour(cx<float> q[12], int c, cx<float> w0, cx<float> w1)
{
    q[c] = q[c] + w0;
    q[3 + c] = q[3 + c] + w1;
    if (MU == 0) {
        q[6 + c] = q[6 + c] - sgn<S>(times_i(w1));
        q[9 + c] = q[9 + c] - sgn<S>(times_i(w0));
    } else if (MU == 1) {
        q[6 + c] = q[6 + c] - sgn<S>(w1);
        q[9 + c] = q[9 + c] + sgn<S>(w0);
    } else if (MU == 2) {
        q[6 + c] = q[6 + c] - sgn<S>(times_i(w0));
        q[9 + c] = q[9 + c] + sgn<S>(times_i(w1));
    } else {
        q[6 + c] = q[6 + c] + sgn<S>(w0);
        q[9 + c] = q[9 + c] + sgn<S>(w1);
    }
}

// Geometry of one CTA's half of an extended block.
struct RasHalf {
    int n;          // sites of this CTA: ne / 2
    int np;         // plane length in shared memory (n rounded up to even)
    int h;          // extended t slices per CTA: e[3] / 2
    int ncmax;      // core sites of the CTA with more of them (x planes)
};

// One hop of the block operator: q += coef * (1 + S gamma_MU) W r(nbr),
// W = U (forward) or U^+ (backward); r and the link come from the shared
// memory images rs / ls (this CTA's or another CTA's) at index ri / li;
// coef multiplies the hop only when SCALED (the -kappa of the hopping term
// is applied once per site, after all hops).
// The product is formed one colour row of W at a time and reconstructed
// into q at once.
template <class P, int MU, int S, bool FWD, bool SCALED = false>
__device__ __forceinline__ void ras_hop_c(const float4 *rs, const void *ls, int np, int ri, int li, float coef,
                                          cx<float> q[12])
{
    cx<float> h[6], u[6], r2[3];
    project_sm<MU, S>(rs, np, ri, h);
    RasLinks<P>::load(ls, np, MU, li, u, r2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<float> m0, m1, m2;   // row c of W
        if (FWD) {
            m0 = c < 2 ? u[3 * c] : r2[0];
            m1 = c < 2 ? u[3 * c + 1] : r2[1];
            m2 = c < 2 ? u[3 * c + 2] : r2[2];
        } else {
            m0 = conj(u[c]);
            m1 = conj(u[3 + c]);
            m2 = conj(r2[c]);
        }
        cx<float> w0 = m0 * h[0], w1 = m0 * h[3];
        w0 = cfma(m1, h[1], w0);
        w1 = cfma(m1, h[4], w1);
        w0 = cfma(m2, h[2], w0);
        w1 = cfma(m2, h[5], w1);
        if (SCALED) {
            w0 = coef * w0;
            w1 = coef * w1;
        }
        reconstruct_add_colour<MU, S>(q, c, w0, w1);
    }
}

// One site per thread, one CTA per SM: 21 warps; the SM's register file
// then caps a thread at 80 registers.
constexpr int kRasCThreads = 672;
constexpr int kRasNC = 2;   // CTAs per block (t halves)

template <class P, int SF>
__global__ void __cluster_dims__(kRasNC, 1, 1) __launch_bounds__(kRasCThreads, 1)
    k_ras_cluster(Geom g, RasGeom rg, RasHalf hg, GaugeStore U, CloverStore C, const void *vin,
                  const float *vin_nrm, void *zout, float *zout_nrm, float kappa)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();   // t slices [rank h, (rank + 1) h) of the block
    const int np = hg.np;

    extern __shared__ float4 smem_raw[];
    float4 *r = smem_raw;                                                  // [6][np]
    void *lk = r + 6 * np;                                                 // links
    float4 *xc = reinterpret_cast<float4 *>(static_cast<char *>(lk) + (size_t)RasLinks<P>::kBytes * np);   // [6][ncmax]
    __shared__ float red[32 * 3];
    if (kChecked) {   // every slot read before it is written shows up as NaN
        const float nan = __int_as_float(0x7fc00000);
        const int nf4 = 6 * np + RasLinks<P>::kBytes / 16 * np + 6 * hg.ncmax;
        for (int q = threadIdx.x; q < nf4; q += blockDim.x) r[q] = make_float4(nan, nan, nan, nan);
        __syncthreads();
    }

    // the neighbouring CTAs' images (distributed shared memory)
    constexpr int NC = kRasNC;
    const int rup = rank + 1 < NC ? rank + 1 : rank, rdn = rank > 0 ? rank - 1 : rank;
    const float4 *r_up = cluster.map_shared_rank(r, rup);
    const float4 *r_dn = cluster.map_shared_rank(r, rdn);
    const void *lk_dn = cluster.map_shared_rank(static_cast<char *>(lk), rdn);

    int bc[4];
    {
        int ib = blockIdx.x / NC;
        bc[0] = ib % rg.nb[0];
        ib /= rg.nb[0];
        bc[1] = ib % rg.nb[1];
        ib /= rg.nb[1];
        bc[2] = ib % rg.nb[2];
        bc[3] = ib / rg.nb[2];
    }
    const int V = g.V;
    const int i = threadIdx.x;   // site of this CTA: local index l = i + rank h es[3]
    const bool active = i < hg.n;
    int lc[4] = {0, 0, 0, 0}, site = 0, core = -1;
    unsigned wbits = 0u;     // bit mu: global coordinate 0; bit 4+mu: L-1
    unsigned hopmask = 0u;   // bit 2 mu: forward hop kept, bit 2 mu + 1: backward hop kept
    if (active) {
        int t = i;
        lc[0] = t % rg.e[0];
        t /= rg.e[0];
        lc[1] = t % rg.e[1];
        t /= rg.e[1];
        lc[2] = t % rg.e[2];
        lc[3] = t / rg.e[2] + rank * hg.h;
        bool in_core = true;
        int ci = 0, cs = 1;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int gm = bc[m] * rg.b[m] - rg.delta + lc[m];
            gm = gm < 0 ? gm + g.L[m] : (gm >= g.L[m] ? gm - g.L[m] : gm);
            site += gm * g.stride[m];
            if (gm == 0) wbits |= 1u << m;
            if (gm == g.L[m] - 1) wbits |= 16u << m;
            const int cm = lc[m] - rg.delta;
            if (cm < 0 || cm >= rg.b[m]) in_core = false;
            if (lc[m] + 1 < rg.e[m]) hopmask |= 1u << (2 * m);
            if (lc[m] >= 1) hopmask |= 2u << (2 * m);
            if (m < 3) {
                ci += cm * cs;
                cs *= rg.b[m];
            }
        }
        // core t slices of this CTA start at max(delta, rank h)
        const int t0 = max(rg.delta, rank * hg.h);
        if (in_core) core = wc_idx(ci + (lc[3] - t0) * cs, hg.ncmax);
        site = wc_idx(site, V);
        cx<float> sp[12];
        P::load_spinor(vin, vin_nrm, V, site, sp);
        sm_store(r, np, i, sp);
        RasLinks<P>::stage(lk, np, i, U, V, site);
        if (core >= 0)
#pragma unroll
            for (int j = 0; j < 6; ++j) xc[j * hg.ncmax + core] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    cluster.sync();

    const float mk = -kappa;
    // time-boundary factor of the t hops (the -kappa comes after all hops)
    const float ph_t_fwd = (wbits & (16u << 3)) ? (float)g.tbc : 1.f;
    const float ph_t_bwd = (wbits & (1u << 3)) ? (float)g.tbc : 1.f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int es1 = rg.es[1], es2 = rg.es[2], st3 = rg.es[3];
    const int lt = lc[3] - rank * hg.h;   // t slice within this CTA
    for (int it = 0; it < rg.k; ++it) {
        cx<float> q[12];
        float acc[3] = {0.f, 0.f, 0.f};
        if (active) {
#pragma unroll
            for (int k = 0; k < 12; ++k) q[k] = mkc(0.f, 0.f);
            // sum of the kept hops, unscaled; x, y, z hops one at a time
            // (runtime loop): bounds the registers the scheduler spends on
            // loads in flight
#pragma unroll 1
            for (int hop = 0; hop < 6; ++hop) {
                if (!((hopmask >> hop) & 1u)) continue;
                const int mu = hop >> 1;
                const int st = mu == 0 ? 1 : (mu == 1 ? es1 : es2);
                if (hop & 1) {
                    const int j = wc_idx(i - st, hg.n);
                    switch (mu) {
                    case 0: ras_hop_c<P, 0, -SF, false>(r, lk, np, j, j, 1.f, q); break;
                    case 1: ras_hop_c<P, 1, -SF, false>(r, lk, np, j, j, 1.f, q); break;
                    default: ras_hop_c<P, 2, -SF, false>(r, lk, np, j, j, 1.f, q); break;
                    }
                } else {
                    const int j = wc_idx(i + st, hg.n);
                    switch (mu) {
                    case 0: ras_hop_c<P, 0, SF, true>(r, lk, np, j, i, 1.f, q); break;
                    case 1: ras_hop_c<P, 1, SF, true>(r, lk, np, j, i, 1.f, q); break;
                    default: ras_hop_c<P, 2, SF, true>(r, lk, np, j, i, 1.f, q); break;
                    }
                }
            }
            if (hopmask & 64u) {
                if (lt + 1 < hg.h)
                    ras_hop_c<P, 3, SF, true, true>(r, lk, np, wc_idx(i + st3, hg.n), i, ph_t_fwd, q);
                else   // last slice: neighbour in the next CTA's first slice
                    ras_hop_c<P, 3, SF, true, true>(r_up, lk, np, wc_idx(i - lt * st3, hg.n), i, ph_t_fwd, q);
            }
            if (hopmask & 128u) {
                if (lt >= 1) {
                    const int j = wc_idx(i - st3, hg.n);
                    ras_hop_c<P, 3, -SF, false, true>(r, lk, np, j, j, ph_t_bwd, q);
                } else {   // first slice: neighbour (and its link) in the previous CTA's last slice
                    const int j = wc_idx(i + (hg.h - 1) * st3, hg.n);
                    ras_hop_c<P, 3, -SF, false, true>(r_dn, lk_dn, np, j, j, ph_t_bwd, q);
                }
            }
            // q = A_b r - kappa (hops) per clover block
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                cx<float> rl[6];
                sm_load_block(r, np, i, b, rl);
                clover32_mul(C, V, site, b, rl, q + 6 * b, mk);
            }
            // <q, r> and <q, q>, one plane of r at a time
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const float4 v = r[j * np + i];
                const int k0 = (j >> 1) + ((j & 1) ? 6 : 0), k1 = k0 + 3;
                const cx<float> ra = mkc(v.x, v.y), rb = mkc(v.z, v.w);
                acc[0] = fmaf(q[k0].re, ra.re, fmaf(q[k0].im, ra.im, acc[0]));    // Re <q, r>
                acc[1] = fmaf(q[k0].re, ra.im, fmaf(-q[k0].im, ra.re, acc[1]));   // Im <q, r>
                acc[2] = fmaf(q[k0].re, q[k0].re, fmaf(q[k0].im, q[k0].im, acc[2]));
                acc[0] = fmaf(q[k1].re, rb.re, fmaf(q[k1].im, rb.im, acc[0]));
                acc[1] = fmaf(q[k1].re, rb.im, fmaf(-q[k1].im, rb.re, acc[1]));
                acc[2] = fmaf(q[k1].re, q[k1].re, fmaf(q[k1].im, q[k1].im, acc[2]));
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < 3; ++j) red[wid * 3 + j] = acc[j];
        // every q is computed (all reads of r of this sweep, in every CTA,
        // are done) and every warp partial is published
        cluster.sync();
        float t[3] = {0.f, 0.f, 0.f};
        if (lane < nw) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {   // rank order: the same sum in every CTA
                const float *rc = cluster.map_shared_rank(red, c);
#pragma unroll
                for (int j = 0; j < 3; ++j) t[j] += rc[lane * 3 + j];
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t[j] += __shfl_xor_sync(0xffffffffu, t[j], o);
        const cx<float> alpha = t[2] > 0.f ? mkc(t[0] / t[2], t[1] / t[2]) : mkc(0.f, 0.f);
        const bool last = it + 1 == rg.k;
        if (active) {
            // x += alpha r (core), r -= alpha q, one plane at a time
            if (core >= 0 && last) {
                cx<float> xk[12];
                sm_load(xc, hg.ncmax, core, xk);
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const float4 v = r[j * np + i];
                    const int k0 = (j >> 1) + ((j & 1) ? 6 : 0), k1 = k0 + 3;
                    xk[k0] = cfma(alpha, mkc(v.x, v.y), xk[k0]);
                    xk[k1] = cfma(alpha, mkc(v.z, v.w), xk[k1]);
                }
                P::store_spinor(zout, zout_nrm, V, site, xk);
            }
            if (!last) {
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const float4 v = r[j * np + i];
                    const int k0 = (j >> 1) + ((j & 1) ? 6 : 0), k1 = k0 + 3;
                    cx<float> ra = mkc(v.x, v.y), rb = mkc(v.z, v.w);
                    if (core >= 0) {
                        const float4 xv = xc[j * hg.ncmax + core];
                        const cx<float> xa = cfma(alpha, ra, mkc(xv.x, xv.y));
                        const cx<float> xb = cfma(alpha, rb, mkc(xv.z, xv.w));
                        xc[j * hg.ncmax + core] = make_float4(xa.re, xa.im, xb.re, xb.im);
                    }
                    ra = ra - alpha * q[k0];
                    rb = rb - alpha * q[k1];
                    r[j * np + i] = make_float4(ra.re, ra.im, rb.re, rb.im);
                }
            }
        }
        // r is updated before the next sweep reads it; on the last sweep the
        // barrier keeps every CTA (and its shared memory) alive until the
        // others have read the partial sums
        cluster.sync();
    }
    if (rg.k == 0 && core >= 0) {
        cx<float> z[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = mkc(0.f, 0.f);
        P::store_spinor(zout, zout_nrm, V, site, z);
    }
}

// ------------------------------------------------------------------------
// RAS on block Schur complements (even-odd solves): MR on
// M^_B = A_ee - kappa^2 H^B_eo A_oo^-1 H^B_oe, the even-site Schur
// complement of the Dirichlet-cut block operator M_B
// ------------------------------------------------------------------------

constexpr int kRasEoMaxThreads = 768;

// One CTA per extended block; thread j owns the j-th even and the j-th odd
// site of the block.  The local x extent e[0] is even, so along every local
// x row the two parities alternate and local site l of either parity has
// compact index l >> 1 in its parity's arrays: thread j = (row, k) owns the
// sites 2k + p_row (even) and 2k + 1 - p_row (odd) of its row, p_row the
// global parity of the row's first site.  Shared memory: r (even), t
// (odd intermediate) and x (even), float4 planes [6][nh].  One MR step:
// odd pass t = A_oo^-1 H^B r, barrier, even pass q = A_ee r - kappa^2 H^B t
// and the partial sums, alpha (barrier inside), x += alpha r,
// r -= alpha q, barrier.  Links, A and A^-1 are read from global memory.

// acc += coef * (the hops of direction MU into local site l whose source,
// of the opposite parity, lies inside the extended block); src: compact
// planes of that parity
template <class P, int MU, int SF>
__device__ __forceinline__ void ras_eo_hops(const Geom &g, const RasGeom &rg, const GaugeStore &U,
                                            const float4 *src, int nh, int l, int site, unsigned lpack,
                                            unsigned wbits, float coef, cx<float> acc[12])
{
    const int lm = (lpack >> (8 * MU)) & 255u;
    const int stl = rg.es[MU];
    if (lm + 1 < rg.e[MU]) {
        const float c = (MU == 3 && (wbits & (16u << 3))) ? coef * (float)g.tbc : coef;
        cx<float> h[6], u[6], r2[3], w[6];
        project_sm<MU, SF>(src, nh, wc_idx((l + stl) >> 1, nh), h);
        P::load_link(U, g.V, MU, site, u, r2);
        su3_mul(u, r2, h, c, w);
        reconstruct_add<MU, SF>(acc, w);
    }
    if (lm >= 1) {
        const int sb = wc_idx((wbits & (1u << MU)) ? site + (g.L[MU] - 1) * g.stride[MU] : site - g.stride[MU], g.V);
        const float c = (MU == 3 && (wbits & (1u << 3))) ? coef * (float)g.tbc : coef;
        cx<float> h[6], u[6], r2[3], w[6];
        project_sm<MU, -SF>(src, nh, wc_idx((l - stl) >> 1, nh), h);
        P::load_link(U, g.V, MU, sb, u, r2);
        su3_adj_mul(u, r2, h, c, w);
        reconstruct_add<MU, -SF>(acc, w);
    }
}

template <class P, int SF>
__device__ __forceinline__ void ras_eo_all_hops(const Geom &g, const RasGeom &rg, const GaugeStore &U,
                                                const float4 *src, int nh, int l, int site, unsigned lpack,
                                                unsigned wbits, cx<float> acc[12])
{
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        switch (mu) {
        case 0: ras_eo_hops<P, 0, SF>(g, rg, U, src, nh, l, site, lpack, wbits, 1.f, acc); break;
        case 1: ras_eo_hops<P, 1, SF>(g, rg, U, src, nh, l, site, lpack, wbits, 1.f, acc); break;
        case 2: ras_eo_hops<P, 2, SF>(g, rg, U, src, nh, l, site, lpack, wbits, 1.f, acc); break;
        default: ras_eo_hops<P, 3, SF>(g, rg, U, src, nh, l, site, lpack, wbits, 1.f, acc); break;
        }
    }
}

// local site l = row * e0 + lx of block bc: global site, packed local
// coordinates, boundary bits (bit mu: global coordinate 0, bit 4+mu: L-1),
// core flag
__device__ __forceinline__ int ras_eo_site(const Geom &g, const RasGeom &rg, const int bc[4], int l,
                                           unsigned &lpack, unsigned &wbits, bool &in_core)
{
    int t = l, site = 0;
    lpack = 0u;
    wbits = 0u;
    in_core = true;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int lm = t % rg.e[m];
        t /= rg.e[m];
        lpack |= (unsigned)lm << (8 * m);
        int gm = bc[m] * rg.b[m] - rg.delta + lm;
        gm = gm < 0 ? gm + g.L[m] : (gm >= g.L[m] ? gm - g.L[m] : gm);
        site += gm * g.stride[m];
        if (gm == 0) wbits |= 1u << m;
        if (gm == g.L[m] - 1) wbits |= 16u << m;
        if (lm < rg.delta || lm >= rg.delta + rg.b[m]) in_core = false;
    }
    return wc_idx(site, g.V);
}

// vin, zout: half-lattice (even-site) fields, index full_site >> 1; A: the
// parity-ordered A (position x >> 1 for even x), Ai: A^-1 (position
// V/2 + (x >> 1) for odd x)
template <class P, int SF>
__global__ void __launch_bounds__(kRasEoMaxThreads, 1)
    k_ras_schur(Geom g, RasGeom rg, GaugeStore U, CloverStore A, CloverStore Ai, const void *vin,
                const float *vin_nrm, void *zout, float *zout_nrm, float kappa)
{
    extern __shared__ float4 smem_raw[];
    const int nh = rg.ne >> 1;
    float4 *r = smem_raw;          // [6][nh] even
    float4 *t = r + 6 * nh;        // [6][nh] odd
    float4 *x = t + 6 * nh;        // [6][nh] even
    __shared__ float red[32 * 3];
    if (kChecked) {   // every slot read before it is written shows up as NaN
        const float nan = __int_as_float(0x7fc00000);
        for (int q = threadIdx.x; q < 18 * nh; q += blockDim.x) r[q] = make_float4(nan, nan, nan, nan);
        __syncthreads();
    }
    int bc[4];
    {
        int ib = blockIdx.x;
        bc[0] = ib % rg.nb[0];
        ib /= rg.nb[0];
        bc[1] = ib % rg.nb[1];
        ib /= rg.nb[1];
        bc[2] = ib % rg.nb[2];
        bc[3] = ib / rg.nb[2];
    }
    const int V = g.V, Vh = V >> 1;
    const int j = threadIdx.x;
    const bool own = j < nh;
    int le = 0, lo = 0, ge = 0, go = 0;
    unsigned lpe = 0u, wbe = 0u, lpo = 0u, wbo = 0u;
    bool core = false;
    if (own) {
        const int h0 = rg.e[0] >> 1, row = j / h0, k = j - row * h0;
        const int ly = row % rg.e[1], lz = (row / rg.e[1]) % rg.e[2], lt = row / (rg.e[1] * rg.e[2]);
        int par = ly + lz + lt;
#pragma unroll
        for (int m = 0; m < 4; ++m) par += bc[m] * rg.b[m] - rg.delta;
        const int prow = par & 1;
        le = row * rg.e[0] + 2 * k + prow;
        lo = row * rg.e[0] + 2 * k + 1 - prow;
        bool dummy;
        ge = ras_eo_site(g, rg, bc, le, lpe, wbe, core);
        go = ras_eo_site(g, rg, bc, lo, lpo, wbo, dummy);
        cx<float> sp[12];
        P::load_spinor(vin, vin_nrm, Vh, ge >> 1, sp);
        sm_store(r, nh, j, sp);
#pragma unroll
        for (int c = 0; c < 6; ++c) x[c * nh + j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float beta = -kappa * kappa;
    for (int it = 0; it < rg.k; ++it) {
        // odd pass: t = A_oo^-1 H^B r
        if (own) {
            cx<float> h[12], o[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) h[c] = mkc(0.f, 0.f);
            ras_eo_all_hops<P, SF>(g, rg, U, r, nh, lo, go, lpo, wbo, h);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                float cl[36];
                P::load_clover(Ai, V, wc_idx(Vh + (go >> 1), V), b, cl);
                clover_block_mul(cl, h + 6 * b, o + 6 * b);
            }
            sm_store(t, nh, j, o);
        }
        __syncthreads();
        // even pass: q = A_ee r - kappa^2 H^B t
        cx<float> q[12];
        float acc[3] = {0.f, 0.f, 0.f};
        if (own) {
            cx<float> h[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) h[c] = mkc(0.f, 0.f);
            ras_eo_all_hops<P, SF>(g, rg, U, t, nh, le, ge, lpe, wbe, h);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                cx<float> rl[6];
                sm_load_block(r, nh, j, b, rl);
                float cl[36];
                P::load_clover(A, V, wc_idx(ge >> 1, V), b, cl);
                clover_block_mul(cl, rl, q + 6 * b);
            }
            cx<float> rl[12];
            sm_load(r, nh, j, rl);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                q[c] = q[c] + beta * h[c];
                acc[0] = fmaf(q[c].re, rl[c].re, fmaf(q[c].im, rl[c].im, acc[0]));    // Re <q, r>
                acc[1] = fmaf(q[c].re, rl[c].im, fmaf(-q[c].im, rl[c].re, acc[1]));   // Im <q, r>
                acc[2] = fmaf(q[c].re, q[c].re, fmaf(q[c].im, q[c].im, acc[2]));
            }
        }
        // contains __syncthreads: every read of r and t is done after it
        const cx<float> alpha = block_alpha(acc, red);
        if (own) {
            cx<float> rk[12], xk[12];
            sm_load(r, nh, j, rk);
            sm_load(x, nh, j, xk);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                xk[c] = cfma(alpha, rk[c], xk[c]);
                rk[c] = rk[c] - alpha * q[c];
            }
            sm_store(x, nh, j, xk);
            sm_store(r, nh, j, rk);
        }
        __syncthreads();
    }
    // restricted prolongation: the even sites of the core
    if (own && core) {
        cx<float> sp[12];
        sm_load(x, nh, j, sp);
        P::store_spinor(zout, zout_nrm, Vh, ge >> 1, sp);
    }
}

}  // namespace

int ras_threads(const wc_ras_params &p);

size_t ras_smem_bytes(const wc_ras_params &p)
{
    size_t ne = 1, nc = 1;
    for (int m = 0; m < 4; ++m) {
        ne *= (size_t)(p.block[m] + 2 * p.overlap);
        nc *= (size_t)p.block[m];
    }
    return (ne + (size_t)ras_threads(p) + nc) * 6 * sizeof(float4);
}

int ras_threads(const wc_ras_params &p)
{
    int ne = 1;
    for (int m = 0; m < 4; ++m) ne *= p.block[m] + 2 * p.overlap;
    const int t = (ne + kRasSPT - 1) / kRasSPT;
    return (t + 31) / 32 * 32;
}

// Launch plan of the cluster kernel for a block shape (FP32 storage; on
// FP16 storage the one-CTA kernel measured faster): the extended t extent
// must split into two equal halves of at most kRasCThreads sites, and the
// images must fit in shared memory.
struct RasClusterPlan {
    RasHalf hg;
    int threads;
    size_t smem;
};

bool ras_cluster_plan(const wc_ras_params &p, wc_prec prec, RasClusterPlan *out)
{
    if (prec != WC_F32) return false;
    constexpr int nc = kRasNC;
    int e[4], ne = 1, ncore = 1;
    for (int m = 0; m < 4; ++m) {
        e[m] = p.block[m] + 2 * p.overlap;
        ne *= e[m];
        ncore *= p.block[m];
    }
    if (e[3] % nc != 0 || ne / nc > kRasCThreads) return false;
    RasClusterPlan c;
    c.hg.n = ne / nc;
    c.hg.np = (c.hg.n + 1) & ~1;
    c.hg.h = e[3] / nc;
    // core sites of the CTA with the most core t slices
    int most = 0;
    for (int rk = 0; rk < nc; ++rk) {
        const int lo = std::max(p.overlap, rk * c.hg.h), hi = std::min(p.overlap + p.block[3], (rk + 1) * c.hg.h);
        most = std::max(most, hi - lo);
    }
    c.hg.ncmax = ncore / p.block[3] * most;
    c.threads = (c.hg.n + 31) / 32 * 32;
    c.smem = (size_t)c.hg.np * (6 * sizeof(float4) + RasLinks<P32>::kBytes) + (size_t)c.hg.ncmax * 6 * sizeof(float4);
    if (c.smem > (size_t)kRasCSmemMax) return false;
    *out = c;
    return true;
}

bool ras_fits(const wc_ras_params &p)
{
    // the one-CTA kernel serves FP16 storage (and FP32 when the cluster
    // kernel does not take the shape)
    return ras_threads(p) <= kRasMaxThreads && ras_smem_bytes(p) <= 226 * 1024;
}

// The shared-memory opt-in is set once per device and kernel (outside any
// stream capture that later launches it), to the largest size allowed.
template <class K>
cudaError_t smem_optin(K kernel, unsigned long long &done_mask, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && (done_mask >> dev) & 1ull) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev < 64) done_mask |= 1ull << dev;
    return e;
}

template <class P, int SF>
cudaError_t ras_smem_optin()
{
    static unsigned long long done = 0;
    return smem_optin(k_ras<P, SF>, done, 226 * 1024);
}

template <class P, int SF>
cudaError_t ras_cluster_optin()
{
    static unsigned long long done = 0;
    return smem_optin(k_ras_cluster<P, SF>, done, kRasCSmemMax);
}

template <class P, int SF>
cudaError_t launch_ras_k(wc_lattice lat, const RasGeom &rg, int nblocks, int threads, size_t smem, wc_field out,
                         wc_field in, cudaStream_t stream)
{
    cudaError_t e = ras_smem_optin<P, SF>();
    if (e != cudaSuccess) return e;
    k_ras<P, SF><<<nblocks, threads, smem, stream>>>(lat->g, rg, lat->gauge, lat->clover, in->data, in->nrm,
                                                     out->data, out->nrm, (float)lat->kappa);
    return cudaGetLastError();
}

template <class P, int SF>
cudaError_t launch_ras_c(wc_lattice lat, const RasGeom &rg, int nblocks, const RasClusterPlan &c, wc_field out,
                         wc_field in, cudaStream_t stream)
{
    cudaError_t e = ras_cluster_optin<P, SF>();
    if (e != cudaSuccess) return e;
    k_ras_cluster<P, SF><<<kRasNC * nblocks, c.threads, c.smem, stream>>>(
        lat->g, rg, c.hg, lat->gauge, lat->clover, in->data, in->nrm, out->data, out->nrm, (float)lat->kappa);
    return cudaGetLastError();
}

// Block-Schur RAS: one CTA per block, e[0] even, at most 2 x 768 sites
int ras_schur_threads(const wc_ras_params &p)
{
    int ne = 1;
    for (int m = 0; m < 4; ++m) ne *= p.block[m] + 2 * p.overlap;
    return (ne / 2 + 31) / 32 * 32;
}

bool ras_schur_fits(const wc_ras_params &p)
{
    if ((p.block[0] + 2 * p.overlap) % 2 != 0) return false;
    int ne = 1;
    for (int m = 0; m < 4; ++m) ne *= p.block[m] + 2 * p.overlap;
    return ras_schur_threads(p) <= kRasEoMaxThreads && (size_t)(ne / 2) * 18 * sizeof(float4) <= 226 * 1024;
}

template <class P, int SF>
cudaError_t ras_schur_optin()
{
    static unsigned long long done = 0;
    return smem_optin(k_ras_schur<P, SF>, done, 226 * 1024);
}

cudaError_t launch_ras_schur(const wc_lattice_s *full, wc_field out, wc_field in, const wc_ras_params &p, int dagger,
                             cudaStream_t stream)
{
    if (!ras_schur_fits(p) || !full->cinv_loaded) return cudaErrorInvalidValue;
    RasGeom rg;
    rg.ne = 1;
    rg.ncore = 1;
    int nblocks = 1;
    for (int m = 0; m < 4; ++m) {
        rg.b[m] = p.block[m];
        rg.e[m] = p.block[m] + 2 * p.overlap;
        rg.nb[m] = full->g.L[m] / p.block[m];
        rg.es[m] = m == 0 ? 1 : rg.es[m - 1] * rg.e[m - 1];
        rg.ne *= rg.e[m];
        rg.ncore *= rg.b[m];
        nblocks *= rg.nb[m];
    }
    rg.delta = p.overlap;
    rg.k = p.mr_iters;
    const size_t smem = (size_t)(rg.ne / 2) * 18 * sizeof(float4);
    const int threads = ras_schur_threads(p);
    const float kappa = (float)full->kappa;
    cudaError_t e = cudaSuccess;
#define WC_RAS_SCHUR(PP, SS)                                                                                   \
    e = ras_schur_optin<PP, SS>();                                                                             \
    if (e == cudaSuccess)                                                                                      \
        k_ras_schur<PP, SS><<<nblocks, threads, smem, stream>>>(full->g, rg, full->gauge, full->ceo, full->cinv, \
                                                                in->data, in->nrm, out->data, out->nrm, kappa)
    if (in->prec == WC_F16) {
        if (dagger) { WC_RAS_SCHUR(P16, +1); } else { WC_RAS_SCHUR(P16, -1); }
    } else {
        if (dagger) { WC_RAS_SCHUR(P32, +1); } else { WC_RAS_SCHUR(P32, -1); }
    }
#undef WC_RAS_SCHUR
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t ras_prepare()
{
    cudaError_t e = ras_smem_optin<P32, -1>();
    if (e == cudaSuccess) e = ras_smem_optin<P32, +1>();
    if (e == cudaSuccess) e = ras_smem_optin<P16, -1>();
    if (e == cudaSuccess) e = ras_smem_optin<P16, +1>();
    if (e == cudaSuccess) e = ras_cluster_optin<P32, -1>();
    if (e == cudaSuccess) e = ras_cluster_optin<P32, +1>();
    if (e == cudaSuccess) e = ras_schur_optin<P32, -1>();
    if (e == cudaSuccess) e = ras_schur_optin<P32, +1>();
    if (e == cudaSuccess) e = ras_schur_optin<P16, -1>();
    if (e == cudaSuccess) e = ras_schur_optin<P16, +1>();
    return e;
}

cudaError_t launch_ras(wc_lattice lat, wc_field out, wc_field in, const wc_ras_params &p, int dagger,
                       cudaStream_t stream)
{
    RasGeom rg;
    rg.ne = 1;
    rg.ncore = 1;
    int nblocks = 1;
    for (int m = 0; m < 4; ++m) {
        rg.b[m] = p.block[m];
        rg.e[m] = p.block[m] + 2 * p.overlap;
        rg.nb[m] = lat->g.L[m] / p.block[m];
        rg.es[m] = m == 0 ? 1 : rg.es[m - 1] * rg.e[m - 1];
        rg.ne *= rg.e[m];
        rg.ncore *= rg.b[m];
        nblocks *= rg.nb[m];
    }
    rg.delta = p.overlap;
    rg.k = p.mr_iters;
    const bool f16 = in->prec == WC_F16;
    RasClusterPlan c;
    if (ras_cluster_plan(p, in->prec, &c))
        return dagger ? launch_ras_c<P32, +1>(lat, rg, nblocks, c, out, in, stream)
                      : launch_ras_c<P32, -1>(lat, rg, nblocks, c, out, in, stream);
    const size_t smem = ras_smem_bytes(p);
    const int threads = ras_threads(p);
    if (f16)
        return dagger ? launch_ras_k<P16, +1>(lat, rg, nblocks, threads, smem, out, in, stream)
                      : launch_ras_k<P16, -1>(lat, rg, nblocks, threads, smem, out, in, stream);
    return dagger ? launch_ras_k<P32, +1>(lat, rg, nblocks, threads, smem, out, in, stream)
                  : launch_ras_k<P32, -1>(lat, rg, nblocks, threads, smem, out, in, stream);
}

}  // namespace wc
