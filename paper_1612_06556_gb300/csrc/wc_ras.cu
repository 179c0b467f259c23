// Overlapped Restricted Additive Schwarz preconditioner with minimal-residual
// block solves, one CTA per block (Sec. 2: the paper's single-precision
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
// GB300 mapping: the extended block's residual r lives in shared memory
// (FP32, component-major [12][ne] so a warp's accesses are contiguous), as
// does the core of x.  Each thread owns two sites; the q of its first site
// is parked in shared memory and the q of its second stays in registers
// across the block-wide reduction of <q, r> and <q, q> (4^4 blocks with
// overlap 1: 1296 sites, 672 threads, 211 KB of shared memory, one CTA per
// SM).  <q, r> and <q, q> are summed in FP32 (GB300's FP64 pipe runs at
// 1/64 of the FP32 rate) with one barrier per MR step for the reduction and
// one before the next sweep reads the updated r.  Links and clover are read from
// global memory (L2-resident across the k sweeps of a block).  Arithmetic is
// FP32 for FP32 and FP16 storage.
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
        project_sm<MU, SF>(r, rg.ne, l + stl, h);
        P::load_link(U, g.V, MU, site, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(q, w);
    }
    if (lm >= 1) {
        const int sb = (wbits & (1u << MU)) ? site + (g.L[MU] - 1) * g.stride[MU] : site - g.stride[MU];
        const float coef = (MU == 3 && (wbits & (1u << 3))) ? mk * (float)g.tbc : mk;
        cx<float> h[6], u[6], r2[3], w[6];
        project_sm<MU, -SF>(r, rg.ne, l - stl, h);
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
            gs[j] = site;
            if (in_core) core[j] = ci;
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

bool ras_fits(const wc_ras_params &p)
{
    return ras_threads(p) <= kRasMaxThreads && ras_smem_bytes(p) <= 226 * 1024;
}

// The shared-memory opt-in is set once per device and kernel (outside any
// stream capture that later launches it), to the largest size allowed.
template <class P, int SF>
cudaError_t ras_smem_optin()
{
    static unsigned long long done_mask = 0;   // bit d: device d
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && (done_mask >> dev) & 1ull) return cudaSuccess;
    e = cudaFuncSetAttribute(k_ras<P, SF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
    if (e == cudaSuccess && dev < 64) done_mask |= 1ull << dev;
    return e;
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

cudaError_t ras_prepare()
{
    cudaError_t e = ras_smem_optin<P32, -1>();
    if (e == cudaSuccess) e = ras_smem_optin<P32, +1>();
    if (e == cudaSuccess) e = ras_smem_optin<P16, -1>();
    if (e == cudaSuccess) e = ras_smem_optin<P16, +1>();
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
    const size_t smem = ras_smem_bytes(p);
    const int threads = ras_threads(p);
    if (in->prec == WC_F16)
        return dagger ? launch_ras_k<P16, +1>(lat, rg, nblocks, threads, smem, out, in, stream)
                      : launch_ras_k<P16, -1>(lat, rg, nblocks, threads, smem, out, in, stream);
    return dagger ? launch_ras_k<P32, +1>(lat, rg, nblocks, threads, smem, out, in, stream)
                  : launch_ras_k<P32, -1>(lat, rg, nblocks, threads, smem, out, in, stream);
}

}  // namespace wc
