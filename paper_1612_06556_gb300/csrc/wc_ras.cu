// Overlapped Restricted Additive Schwarz preconditioner with minimal-residual
// block solves, one CTA per block (paper Sec. 2: the single-precision solver
// is "further preconditioned with the even-odd site and the overlapped RAS
// preconditioning").
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

// q += -kappa * (forward and backward hop in direction MU), both dropped
// when their target leaves the extended block.  SF = -1 for M (forward
// projector 1 - gamma), +1 for M^+ = gamma5 M gamma5.
template <class P, int MU, int SF>
__device__ __forceinline__ void ras_hops(const Geom &g, const RasGeom &rg, const GaugeStore &U, const float2 *r,
                                         int l, int site, unsigned lpack, unsigned wbits, float mk, cx<float> q[12])
{
    const int lm = (lpack >> (8 * MU)) & 255u;
    const int stl = rg.es[MU];
    if (lm + 1 < rg.e[MU]) {
        const int lf = l + stl;
        const float coef = (MU == 3 && (wbits & (16u << 3))) ? mk * (float)g.tbc : mk;
        cx<float> h[6], u[6], r2[3], w[6];
        project_from<MU, SF, float>([&](int k) {
            const float2 v = r[k * rg.ne + lf];
            return mkc(v.x, v.y);
        }, h);
        P::load_link(U, g.V, MU, site, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(q, w);
    }
    if (lm >= 1) {
        const int lb = l - stl;
        const int sb = (wbits & (1u << MU)) ? site + (g.L[MU] - 1) * g.stride[MU] : site - g.stride[MU];
        const float coef = (MU == 3 && (wbits & (1u << 3))) ? mk * (float)g.tbc : mk;
        cx<float> h[6], u[6], r2[3], w[6];
        project_from<MU, -SF, float>([&](int k) {
            const float2 v = r[k * rg.ne + lb];
            return mkc(v.x, v.y);
        }, h);
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
    float2 *r = reinterpret_cast<float2 *>(smem_raw);               // [12][ne]
    float2 *qs = r + 12 * rg.ne;                                     // [12][blockDim.x]
    float2 *xc = qs + 12 * blockDim.x;                               // [12][ncore]
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
#pragma unroll
            for (int k = 0; k < 12; ++k) r[k * rg.ne + l] = make_float2(sp[k].re, sp[k].im);
            if (in_core)
#pragma unroll
                for (int k = 0; k < 12; ++k) xc[k * rg.ncore + ci] = make_float2(0.f, 0.f);
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
            if (j > 0 && gs[0] >= 0) {
                // park the first site's q in shared memory
#pragma unroll
                for (int k = 0; k < 12; ++k) qs[k * nt + threadIdx.x] = make_float2(q[k].re, q[k].im);
            }
            // q = A r_l - kappa (hops inside the extended block)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                cx<float> rl[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float2 v = r[(6 * b + k) * rg.ne + l];
                    rl[k] = mkc(v.x, v.y);
                }
                float cl[36];
                P::load_clover(C, V, gs[j], b, cl);
                clover_block_mul(cl, rl, q + 6 * b);
            }
            ras_hops<P, 0, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q);
            ras_hops<P, 1, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q);
            ras_hops<P, 2, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q);
            ras_hops<P, 3, SF>(g, rg, U, r, l, gs[j], lpack[j], wbits[j], mk, q);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float2 v = r[k * rg.ne + l];
                acc[0] = fmaf(q[k].re, v.x, fmaf(q[k].im, v.y, acc[0]));    // Re <q, r>
                acc[1] = fmaf(q[k].re, v.y, fmaf(-q[k].im, v.x, acc[1]));   // Im <q, r>
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
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float2 v = r[k * rg.ne + l];
                const cx<float> rk = mkc(v.x, v.y);
                cx<float> qk;
                if (last) {
                    qk = q[k];
                } else {
                    const float2 w = qs[k * nt + threadIdx.x];
                    qk = mkc(w.x, w.y);
                }
                if (core[j] >= 0) {
                    float2 *xp = xc + k * rg.ncore + core[j];
                    const cx<float> xn = cfma(alpha, rk, mkc(xp->x, xp->y));
                    *xp = make_float2(xn.re, xn.im);
                }
                const cx<float> rn = rk - alpha * qk;
                r[k * rg.ne + l] = make_float2(rn.re, rn.im);
            }
        }
        __syncthreads();
    }

    // restricted prolongation: the core of x
#pragma unroll
    for (int j = 0; j < kRasSPT; ++j) {
        if (core[j] < 0) continue;
        cx<float> s[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float2 v = xc[k * rg.ncore + core[j]];
            s[k] = mkc(v.x, v.y);
        }
        P::store_spinor(zout, zout_nrm, V, gs[j], s);
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
    return (ne + (size_t)ras_threads(p) + nc) * 12 * sizeof(float2);
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
