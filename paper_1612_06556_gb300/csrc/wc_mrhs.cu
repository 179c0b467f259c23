// Multi-right-hand-side Wilson-Clover operator: out_r = M in_r (or M^+ in_r)
// for up to kMrhsMax fields of one lattice in one launch.
//
// The right-hand sides of a propagator share the gauge field and the clover
// term, which are 480 of the 672 bytes per site of a single FP32 apply.  A
// CTA covers kMrhsSites consecutive sites for all n right-hand sides: it
// first stages, once, the 4 forward links of its sites, the 4 backward links
// U_mu(x - mu) of their neighbours and their clover blocks in shared memory
// (42 float4 per site, coalesced along the sites), then thread (s, r)
// computes site s of right-hand side r, reading links and clover from
// shared memory and the 9 spinors of field r from global memory (neighbours
// through L1/L2); the third row of each link is rebuilt once per site
// after staging.  Compulsory bytes per site and right-hand side:
// 2 x 96 (spinor in, out) + 480 / n, i.e. 232 B at n = 12 against 672 B for
// separate applies.  The arithmetic per (site, right-hand side) is that of
// the single-field operator (spin projection, two-row links with the third
// row rebuilt, clover first, then -kappa times the hops).
#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

constexpr int kMrhsSites = 32;
constexpr int kStageF4 = 42;   // float4 per site: 12 forward link, 12 backward link, 18 clover

struct MrhsArgs {
    int n;
    const float4 *in[kMrhsMax];
    float4 *out[kMrhsMax];
};

// the two stored rows of staged link lam (mu, or 4 + mu for U_mu(x - mu))
__device__ __forceinline__ void rows_from_stage(const float4 (*st)[kMrhsSites], int lam, int s, cx<float> a[6])
{
    const int base = 3 * lam;   // words 0-11 forward, 12-23 backward links
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float4 v = st[base + j][s];
        a[2 * j] = mkc(v.x, v.y);
        a[2 * j + 1] = mkc(v.z, v.w);
    }
}

// link lam of site s: stored rows and the third row rebuilt at staging
__device__ __forceinline__ void link_from_stage(const float4 (*st)[kMrhsSites], const float2 (*r3)[3][kMrhsSites],
                                                int lam, int s, cx<float> a[6], cx<float> c[3])
{
    rows_from_stage(st, lam, s, a);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float2 v = r3[lam][j][s];
        c[j] = mkc(v.x, v.y);
    }
}

template <int MU, int SF>
__device__ __forceinline__ void hop_mrhs(const Geom &g, const float4 (*st)[kMrhsSites],
                                         const float2 (*r3)[3][kMrhsSites], int s, const float4 *in, int x,
                                         const int c[4], float k, cx<float> acc[12])
{
    const int L = g.L[MU], stl = g.stride[MU];
    {
        const bool wrap = c[MU] == L - 1;
        const int xf = wc_idx(wrap ? x - (L - 1) * stl : x + stl, g.V);
        cx<float> p[12], h[6], u[6], r2[3], w[6];
        P32::load_spinor(in, nullptr, g.V, xf, p);
        const float coef = (MU == 3 && wrap) ? k * (float)g.tbc : k;
        project<MU, SF>(p, h);
        link_from_stage(st, r3, MU, s, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(acc, w);
    }
    {
        const bool wrap = c[MU] == 0;
        const int xb = wc_idx(wrap ? x + (L - 1) * stl : x - stl, g.V);
        cx<float> p[12], h[6], u[6], r2[3], w[6];
        P32::load_spinor(in, nullptr, g.V, xb, p);
        const float coef = (MU == 3 && wrap) ? k * (float)g.tbc : k;
        project<MU, -SF>(p, h);
        link_from_stage(st, r3, 4 + MU, s, u, r2);
        su3_adj_mul(u, r2, h, coef, w);
        reconstruct_add<MU, -SF>(acc, w);
    }
}

// KIND 0: M, 1: M^+.  blockDim = kMrhsSites * n.  active (nullable): 0 skips
// right-hand side r (its out is left untouched).  80 registers: two CTAs of
// 12 right-hand sides (24 warps) per SM.
template <int KIND>
__global__ void __maxnreg__(80)
    k_apply_mrhs(Geom g, GaugeStore U, CloverStore C, const __grid_constant__ MrhsArgs a, const int *active,
                 double kappa)
{
    __shared__ float4 st[kStageF4][kMrhsSites];
    __shared__ float2 r3[8][3][kMrhsSites];   // third rows of the 8 links
    const int x0 = blockIdx.x * kMrhsSites;
    // blockDim is a multiple of kMrhsSites: a thread stages and computes the
    // same site s
    const int s = threadIdx.x % kMrhsSites, r = threadIdx.x / kMrhsSites, x = x0 + s;
    int c[4] = {0, 0, 0, 0};
    if (x < g.V) {
        site_coords_fast(g, x, c);
        for (int item = r; item < kStageF4; item += blockDim.x / kMrhsSites) {
            float4 v;
            if (item < 12) {                               // U_mu(x), plane item of [4][3][V]
                v = __ldg(U.u32 + (size_t)item * g.V + x);
            } else if (item < 24) {                        // U_mu(x - mu)
                const int mu = (item - 12) / 3, j = (item - 12) % 3;
                const int xb = wc_idx(c[mu] == 0 ? x + (g.L[mu] - 1) * g.stride[mu] : x - g.stride[mu], g.V);
                v = __ldg(U.u32 + ((size_t)mu * 3 + j) * g.V + xb);
            } else {                                       // clover plane item - 24 of [18][V]
                v = __ldg(C.c32 + (size_t)(item - 24) * g.V + x);
            }
            st[item][s] = v;
        }
    }
    __syncthreads();
    // the third row of every staged link, once per site
    for (int q = threadIdx.x; q < 8 * kMrhsSites; q += blockDim.x) {
        const int ss = q % kMrhsSites, lam = q / kMrhsSites;
        if (x0 + ss >= g.V) continue;
        cx<float> u[6], c3[3];
        rows_from_stage(st, lam, ss, u);
        reconstruct_row2(u, c3);
#pragma unroll
        for (int j = 0; j < 3; ++j) r3[lam][j][ss] = make_float2(c3[j].re, c3[j].im);
    }
    __syncthreads();
    if (r >= a.n || x >= g.V || (active && !active[r])) return;
    const float4 *in = a.in[r];
    cx<float> acc[12];
    {
        cx<float> p[12];
        P32::load_spinor(in, nullptr, g.V, x, p);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float cl[36];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float4 v = st[24 + 9 * b + q][s];
                cl[4 * q] = v.x;
                cl[4 * q + 1] = v.y;
                cl[4 * q + 2] = v.z;
                cl[4 * q + 3] = v.w;
            }
            clover_block_mul(cl, p + 6 * b, acc + 6 * b);
        }
    }
    const float k = (float)(-kappa);
    constexpr int SF = KIND == 1 ? +1 : -1;
    hop_mrhs<0, SF>(g, st, r3, s, in, x, c, k, acc);
    hop_mrhs<1, SF>(g, st, r3, s, in, x, c, k, acc);
    hop_mrhs<2, SF>(g, st, r3, s, in, x, c, k, acc);
    hop_mrhs<3, SF>(g, st, r3, s, in, x, c, k, acc);
    P32::store_spinor(a.out[r], nullptr, g.V, x, acc);
}

}  // namespace

cudaError_t launch_apply_multi(wc_lattice lat, int n, const wc_field *outs, const wc_field *ins, int kind,
                               const int *active, cudaStream_t stream)
{
    if (n < 1 || n > kMrhsMax) return cudaErrorInvalidValue;
    MrhsArgs a{};
    a.n = n;
    for (int r = 0; r < n; ++r) {
        a.in[r] = static_cast<const float4 *>(ins[r]->data);
        a.out[r] = static_cast<float4 *>(outs[r]->data);
    }
    const Geom &g = lat->g;
    const dim3 grid((g.V + kMrhsSites - 1) / kMrhsSites), block(kMrhsSites * n);
    if (kind == 1)
        k_apply_mrhs<1><<<grid, block, 0, stream>>>(g, lat->gauge, lat->clover, a, active, lat->kappa);
    else
        k_apply_mrhs<0><<<grid, block, 0, stream>>>(g, lat->gauge, lat->clover, a, active, lat->kappa);
    return cudaGetLastError();
}

}  // namespace wc
