// Fused BLAS-1 with FP64 accumulation: inner products, norms, axpy, and the
// per-iteration vector updates of BiCGStab, each one pass over its fields.
//
// Reductions are deterministic: every block reduces its grid-stride share
// (warp shuffles, then one warp over the block's warps), writes one partial,
// and the last block to finish (completion ticket) adds the partials in
// block order and runs the scalar update of the solver in one thread.  The
// ticket resets itself, so no memset is needed between launches.
#include <math.h>

#include <algorithm>

#include "wc_internal.cuh"
#include "wc_solver_kernels.cuh"

namespace wc {

namespace {

constexpr int kRedBlock = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// Last block of a grid reduction: every thread adds the partials of blocks
// t, t + blockDim, ... (independent loads, unrolled), then the block sums
// the thread totals by warp shuffles and one warp over the warp totals --
// a fixed order, so the result is the same on every run.  (One warp
// walking all partials serialises ~gridDim/32 L2 round trips per value,
// 15-20 us per reduction kernel at 8 blocks per SM.)  sm: >= 32 * N
// doubles of shared scratch.  Resets the ticket.
template <int N>
__device__ __forceinline__ void final_sum(const ReduceScratch &rs, double *out, double *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = 0.0;
#pragma unroll 4
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < N; ++i) t[i] += __ldcg(rs.partials + (size_t)b * 8 + i);
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = warp_sum(t[i]);
    __syncthreads();   // sm may still be read by the first stage
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) sm[wid * N + i] = t[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double u = lane < nw ? sm[lane * N + i] : 0.0;
            u = warp_sum(u);
            if (lane == 0) out[i] = u;
        }
        if (lane == 0) *rs.ticket = 0u;
    }
    __syncthreads();   // out[] is read by thread 0 after return
}

// Reduce v[0..N) over the grid.  Returns true in thread 0 of the last block,
// after out[0..N) holds the grid totals (summed in a fixed order).
template <int N>
__device__ __forceinline__ bool grid_reduce(double (&v)[N], const ReduceScratch &rs, double *out)
{
    __shared__ double sm[32][N];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) sm[wid][i] = v[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = lane < nw ? sm[lane][i] : 0.0;
            s = warp_sum(s);
            if (lane == 0) rs.partials[(size_t)blockIdx.x * 8 + i] = s;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(rs.ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    final_sum<N>(rs, out, &sm[0][0]);
    return threadIdx.x == 0;
}

int reduce_grid(const ReduceScratch &rs, long long n)
{
    long long b = (n + kRedBlock - 1) / kRedBlock;
    if (b > rs.max_blocks) b = rs.max_blocks;
    if (b < 1) b = 1;
    return (int)b;
}

namespace {

// ------------------------------------------------------------------------
// generic (any precision, per site) dot / norm / axpy for the C ABI
// ------------------------------------------------------------------------

template <class PA, class PB>
__global__ void __launch_bounds__(kRedBlock) k_dot(int V, const void *a, const float *an, const void *b,
                                                   const float *bn, ReduceScratch rs)
{
    double v[2] = {0.0, 0.0};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<typename PA::real> sa[12];
        cx<typename PB::real> sb[12];
        PA::load_spinor(a, an, V, x, sa);
        PB::load_spinor(b, bn, V, x, sb);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double ar = sa[k].re, ai = sa[k].im, br = sb[k].re, bi = sb[k].im;
            v[0] += ar * br + ai * bi;
            v[1] += ar * bi - ai * br;
        }
    }
    grid_reduce<2>(v, rs, rs.result);
}

template <class P>
__global__ void __launch_bounds__(kRedBlock) k_axpy_norm(int V, double ar, double ai, const void *x_,
                                                         const float *xn, void *y_, float *yn, ReduceScratch rs)
{
    double v[1] = {0.0};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        using R = typename P::real;
        cx<R> sx[12], sy[12];
        P::load_spinor(x_, xn, V, x, sx);
        P::load_spinor(y_, yn, V, x, sy);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double re = (double)sy[k].re + ar * sx[k].re - ai * sx[k].im;
            const double im = (double)sy[k].im + ar * sx[k].im + ai * sx[k].re;
            sy[k] = mkc((R)re, (R)im);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) v[0] += (double)sy[k].re * sy[k].re + (double)sy[k].im * sy[k].im;
        P::store_spinor(y_, yn, V, x, sy);
    }
    grid_reduce<1>(v, rs, rs.result);
}

template <class PA>
cudaError_t launch_dot_a(wc_lattice lat, wc_field a, wc_field b)
{
    const int V = lat->g.V;
    const int grid = reduce_grid(lat->st.red, V);
    switch (b->prec) {
    case WC_F64:
        k_dot<PA, P64><<<grid, kRedBlock, 0, lat->stream>>>(V, a->data, a->nrm, b->data, b->nrm, lat->st.red);
        break;
    case WC_F32:
        k_dot<PA, P32><<<grid, kRedBlock, 0, lat->stream>>>(V, a->data, a->nrm, b->data, b->nrm, lat->st.red);
        break;
    default:
        k_dot<PA, P16><<<grid, kRedBlock, 0, lat->stream>>>(V, a->data, a->nrm, b->data, b->nrm, lat->st.red);
    }
    return cudaGetLastError();
}

wc_status fetch_result(wc_lattice lat, int n, double *out)
{
    wc_status st = check_cuda(lat,
                              cudaMemcpyAsync(lat->st.red.host_result, lat->st.red.result, sizeof(double) * n,
                                              cudaMemcpyDeviceToHost, lat->stream),
                              "cudaMemcpyAsync(reduce)");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync(reduce)");
    if (st == WC_OK)
        for (int i = 0; i < n; ++i) out[i] = lat->st.red.host_result[i];
    return st;
}

}  // namespace

wc_status reduce_dot(wc_lattice lat, wc_field a, wc_field b, double out[2])
{
    cudaError_t e;
    switch (a->prec) {
    case WC_F64: e = launch_dot_a<P64>(lat, a, b); break;
    case WC_F32: e = launch_dot_a<P32>(lat, a, b); break;
    default: e = launch_dot_a<P16>(lat, a, b);
    }
    wc_status st = check_cuda(lat, e, "dot");
    if (st != WC_OK) return st;
    return fetch_result(lat, 2, out);
}

wc_status reduce_norm2(wc_lattice lat, wc_field a, double *out)
{
    double d[2];
    wc_status st = reduce_dot(lat, a, a, d);
    if (st == WC_OK) *out = d[0];
    return st;
}

wc_status axpy_norm(wc_lattice lat, const double a[2], wc_field x, wc_field y, double *norm2)
{
    const int V = lat->g.V;
    const int grid = reduce_grid(lat->st.red, V);
    switch (y->prec) {
    case WC_F64:
        k_axpy_norm<P64><<<grid, kRedBlock, 0, lat->stream>>>(V, a[0], a[1], x->data, x->nrm, y->data, y->nrm,
                                                              lat->st.red);
        break;
    case WC_F32:
        k_axpy_norm<P32><<<grid, kRedBlock, 0, lat->stream>>>(V, a[0], a[1], x->data, x->nrm, y->data, y->nrm,
                                                              lat->st.red);
        break;
    default:
        k_axpy_norm<P16><<<grid, kRedBlock, 0, lat->stream>>>(V, a[0], a[1], x->data, x->nrm, y->data, y->nrm,
                                                              lat->st.red);
    }
    wc_status st = check_launch(lat, "axpy_norm");
    if (st != WC_OK) return st;
    double n2 = 0.0;
    st = fetch_result(lat, 1, &n2);
    if (st == WC_OK && norm2) *norm2 = n2;
    return st;
}

// ------------------------------------------------------------------------
// BiCGStab vector updates on FP64 fields (flat arrays of n = 12 V complex)
// ------------------------------------------------------------------------

namespace {

__device__ __forceinline__ cx<double> ld(const double2 *p, long long i)
{
    const double2 v = p[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void st(double2 *p, long long i, cx<double> a) { p[i] = make_double2(a.re, a.im); }
__device__ __forceinline__ cx<double> c_of(double2 a) { return {a.x, a.y}; }
__device__ __forceinline__ double2 d2_of(cx<double> a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ bool finite2(cx<double> a) { return isfinite(a.re) && isfinite(a.im); }

// result[0] = |a|^2 (FP64 field as a flat array)
__global__ void __launch_bounds__(kRedBlock) k_norm2_flat(long long n, const double2 *a, ReduceScratch rs)
{
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> ai = ld(a, i);
        acc[0] += ai.re * ai.re + ai.im * ai.im;
    }
    grid_reduce<1>(acc, rs, rs.result);
}

// r = b - r (r holds M x on entry), rhat = r, p = v = 0;  rr = |r|^2
__global__ void __launch_bounds__(kRedBlock) k_bicg_init(long long n, const double2 *b, double2 *r, double2 *rhat,
                                                         double2 *p, double2 *v, ReduceScratch rs,
                                                         SolverScalars *sc)
{
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> ri = ld(b, i) - ld(r, i);
        st(r, i, ri);
        st(rhat, i, ri);
        p[i] = make_double2(0.0, 0.0);
        v[i] = make_double2(0.0, 0.0);
        acc[0] += ri.re * ri.re + ri.im * ri.im;
    }
    if (grid_reduce<1>(acc, rs, rs.result)) {
        const double rr = rs.result[0];
        sc->rr = rr;
        sc->rho = make_double2(rr, 0.0);   // <rhat, r> with rhat = r
        sc->rho0 = make_double2(1.0, 0.0);
        sc->alpha = make_double2(1.0, 0.0);
        sc->omega = make_double2(1.0, 0.0);
        sc->beta = make_double2(rr, 0.0);  // (rho/rho0)(alpha/omega)
        sc->flags = isfinite(rr) ? 0 : FLAG_NAN;
        if (rr == 0.0) sc->flags |= FLAG_BREAKDOWN;
    }
}

// p = r + beta (p - omega v);  pp = |p|^2
__global__ void __launch_bounds__(kRedBlock) k_bicg_p(long long n, const double2 *r, const double2 *v, double2 *p,
                                                      ReduceScratch rs, SolverScalars *sc)
{
    const cx<double> beta = c_of(sc->beta), omega = c_of(sc->omega);
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> pi = ld(r, i) + beta * (ld(p, i) - omega * ld(v, i));
        st(p, i, pi);
        acc[0] += pi.re * pi.re + pi.im * pi.im;
    }
    if (grid_reduce<1>(acc, rs, rs.result)) {
        sc->pp = rs.result[0];
        if (!isfinite(sc->pp)) sc->flags |= FLAG_NAN;
    }
}

// alpha = rho / <rhat, v>
__global__ void __launch_bounds__(kRedBlock) k_bicg_alpha(long long n, const double2 *rhat, const double2 *v,
                                                          ReduceScratch rs, SolverScalars *sc)
{
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> a = ld(rhat, i), b = ld(v, i);
        acc[0] += a.re * b.re + a.im * b.im;
        acc[1] += a.re * b.im - a.im * b.re;
    }
    if (grid_reduce<2>(acc, rs, rs.result)) {
        const cx<double> rv = mkc(rs.result[0], rs.result[1]);
        if (!finite2(rv)) sc->flags |= FLAG_NAN;
        if (rv.re == 0.0 && rv.im == 0.0) {
            sc->flags |= FLAG_BREAKDOWN;
            sc->alpha = make_double2(0.0, 0.0);
        } else {
            sc->alpha = d2_of(cdiv(c_of(sc->rho), rv));
        }
    }
}

// s = r - alpha v;  ss = |s|^2
__global__ void __launch_bounds__(kRedBlock) k_bicg_s(long long n, const double2 *r, const double2 *v, double2 *s,
                                                      ReduceScratch rs, SolverScalars *sc)
{
    const cx<double> alpha = c_of(sc->alpha);
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> si = ld(r, i) - alpha * ld(v, i);
        st(s, i, si);
        acc[0] += si.re * si.re + si.im * si.im;
    }
    if (grid_reduce<1>(acc, rs, rs.result)) {
        sc->ss = rs.result[0];
        if (!isfinite(sc->ss)) sc->flags |= FLAG_NAN;
    }
}

// omega = <t, s> / <t, t>
__global__ void __launch_bounds__(kRedBlock) k_bicg_omega(long long n, const double2 *t, const double2 *s,
                                                          ReduceScratch rs, SolverScalars *sc)
{
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> a = ld(t, i), b = ld(s, i);
        acc[0] += a.re * b.re + a.im * b.im;
        acc[1] += a.re * b.im - a.im * b.re;
        acc[2] += a.re * a.re + a.im * a.im;
    }
    if (grid_reduce<3>(acc, rs, rs.result)) {
        const double tt = rs.result[2];
        sc->tt = tt;
        if (!isfinite(tt) || !isfinite(rs.result[0]) || !isfinite(rs.result[1])) sc->flags |= FLAG_NAN;
        if (tt > 0.0)
            sc->omega = make_double2(rs.result[0] / tt, rs.result[1] / tt);
        else
            sc->omega = make_double2(0.0, 0.0);
    }
}

// x += alpha phat + omega shat;  r = s - omega t;  rho' = <rhat, r>, rr = |r|^2,
// beta = (rho'/rho)(alpha/omega), rho0 = rho, rho = rho'
__global__ void __launch_bounds__(kRedBlock) k_bicg_xr(long long n, double2 *x, const double2 *phat,
                                                       const double2 *shat, const double2 *s, const double2 *t,
                                                       double2 *r, const double2 *rhat, ReduceScratch rs,
                                                       SolverScalars *sc)
{
    const cx<double> alpha = c_of(sc->alpha), omega = c_of(sc->omega);
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cx<double> xi = ld(x, i);
        xi = cfma(alpha, ld(phat, i), xi);
        xi = cfma(omega, ld(shat, i), xi);
        st(x, i, xi);
        const cx<double> ri = ld(s, i) - omega * ld(t, i);
        st(r, i, ri);
        const cx<double> h = ld(rhat, i);
        acc[0] += h.re * ri.re + h.im * ri.im;
        acc[1] += h.re * ri.im - h.im * ri.re;
        acc[2] += ri.re * ri.re + ri.im * ri.im;
    }
    if (grid_reduce<3>(acc, rs, rs.result)) {
        const cx<double> rho_new = mkc(rs.result[0], rs.result[1]);
        const cx<double> rho = c_of(sc->rho);
        sc->rr = rs.result[2];
        if (!isfinite(sc->rr) || !finite2(rho_new)) sc->flags |= FLAG_NAN;
        if ((omega.re == 0.0 && omega.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
            sc->flags |= FLAG_BREAKDOWN;
        } else {
            sc->beta = d2_of(cdiv(rho_new, rho) * cdiv(alpha, omega));
        }
        if (rho_new.re == 0.0 && rho_new.im == 0.0 && sc->rr > 0.0) sc->flags |= FLAG_BREAKDOWN;
        sc->rho0 = sc->rho;
        sc->rho = d2_of(rho_new);
    }
}

// r = b - r (r holds M x);  rr = |r|^2  (true residual)
__global__ void __launch_bounds__(kRedBlock) k_residual(long long n, const double2 *b, double2 *r,
                                                        ReduceScratch rs, SolverScalars *sc)
{
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx<double> ri = ld(b, i) - ld(r, i);
        st(r, i, ri);
        acc[0] += ri.re * ri.re + ri.im * ri.im;
    }
    if (grid_reduce<1>(acc, rs, rs.result)) sc->rr = rs.result[0];
}

}  // namespace

// ------------------------------------------------------------------------
// Low-precision BiCGStab vector updates (FP32 fields, FP32 arithmetic) for
// the reliable-update solver.  Per-thread partial sums are FP32; blocks add
// them in FP32 and the last block adds the block partials in FP64, so the
// FP64 pipe is used once per block rather than once per element.
// ------------------------------------------------------------------------

namespace {

__device__ __forceinline__ cx<float> f2c(float2 a) { return {a.x, a.y}; }

// Fields are flat arrays of n = 6 V float4 (two complex each).
__device__ __forceinline__ void ld4(const float4 *p, long long i, cx<float> &a, cx<float> &b)
{
    const float4 v = p[i];
    a = {v.x, v.y};
    b = {v.z, v.w};
}
__device__ __forceinline__ void st4(float4 *p, long long i, cx<float> a, cx<float> b)
{
    p[i] = make_float4(a.re, a.im, b.re, b.im);
}

// Grid sum of per-thread FP32 partials: lanes and warps in FP32, the block
// partials (one per block) in FP64 by the last block, in block order.
// Returns true in thread 0 of the last block once out[0..N) is final.
template <int N>
__device__ __forceinline__ bool grid_reduce_f(float (&v)[N], const ReduceScratch &rs, double *out)
{
    __shared__ float sm[32][N];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) sm[wid][i] = v[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float t = lane < nw ? sm[lane][i] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) rs.partials[(size_t)blockIdx.x * 8 + i] = (double)t;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(rs.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    __shared__ double smd[32 * N];
    final_sum<N>(rs, out, smd);
    return threadIdx.x == 0;
}

__device__ __forceinline__ cx<double> c_of2(double2 a) { return {a.x, a.y}; }
__device__ __forceinline__ double2 d2_of2(cx<double> a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ cx<double> cdiv2(cx<double> a, cx<double> b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// Scalar updates of the low-precision BiCGStab, run by one thread of the
// last block once the grid sums res[] are final (shared by the FP32 and the
// FP16-storage kernels).
__device__ void lo_init_update(const double *res, SolverScalars *sc)
{
    const double rr = res[0];
    sc->rr = rr;
    sc->rho = make_double2(rr, 0.0);
    sc->rho0 = make_double2(1.0, 0.0);
    sc->alpha = make_double2(1.0, 0.0);
    sc->omega = make_double2(1.0, 0.0);
    sc->beta = make_double2(rr, 0.0);
    sc->flags = isfinite(rr) ? 0 : FLAG_NAN;
    if (rr == 0.0) sc->flags |= FLAG_BREAKDOWN;
}

// alpha = rho / <rhat, v>
__device__ void lo_alpha_update(const double *res, SolverScalars *sc)
{
    const cx<double> rv = mkc(res[0], res[1]);
    if (!isfinite(rv.re) || !isfinite(rv.im)) sc->flags |= FLAG_NAN;
    if (rv.re == 0.0 && rv.im == 0.0) {
        sc->flags |= FLAG_BREAKDOWN;
        sc->alpha = make_double2(0.0, 0.0);
    } else {
        sc->alpha = d2_of2(cdiv2(c_of2(sc->rho), rv));
    }
}

// omega from <t, s>, <t, t>, <s, s>
__device__ void lo_omega_update(const double *res, SolverScalars *sc)
{
    const double tr = res[0], ti = res[1], tt = res[2], ss = res[3];
    sc->tt = tt;
    if (!isfinite(tt) || !isfinite(tr) || !isfinite(ti) || !isfinite(ss)) sc->flags |= FLAG_NAN;
    double2 om = tt > 0.0 ? make_double2(tr / tt, ti / tt) : make_double2(0.0, 0.0);
    // omega stabilisation (Sleijpen & van der Vorst): when t and s are
    // nearly orthogonal, |<t,s>| / (|t||s|) < 0.7, the minimising omega is
    // tiny and BiCGStab loses accuracy in finite precision; enlarge it
    const double rho_t = (tt > 0.0 && ss > 0.0) ? sqrt(tr * tr + ti * ti) / sqrt(tt * ss) : 1.0;
    if (rho_t > 0.0 && rho_t < 0.7) {
        const double f = 0.7 / rho_t;
        om.x *= f;
        om.y *= f;
    }
    sc->omega = om;
}

// rho' = <rhat, r>, rr = |r|^2, beta
__device__ void lo_xr_update(const double *res, SolverScalars *sc)
{
    const cx<double> rho_new = mkc(res[0], res[1]);
    const cx<double> rho = c_of2(sc->rho), om = c_of2(sc->omega), al = c_of2(sc->alpha);
    sc->rr = res[2];
    if (!isfinite(sc->rr) || !isfinite(rho_new.re) || !isfinite(rho_new.im)) sc->flags |= FLAG_NAN;
    if ((om.re == 0.0 && om.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0))
        sc->flags |= FLAG_BREAKDOWN;
    else
        sc->beta = d2_of2(cdiv2(rho_new, rho) * cdiv2(al, om));
    if (rho_new.re == 0.0 && rho_new.im == 0.0 && sc->rr > 0.0) sc->flags |= FLAG_BREAKDOWN;
    sc->rho0 = sc->rho;
    sc->rho = d2_of2(rho_new);
}

// after r was replaced: rho = <rhat, r>, beta from rho0 (rr untouched)
__device__ void lo_rho_update(const double *res, SolverScalars *sc)
{
    const cx<double> rho_new = mkc(res[0], res[1]);
    const cx<double> rho0 = c_of2(sc->rho0), om = c_of2(sc->omega), al = c_of2(sc->alpha);
    if ((om.re != 0.0 || om.im != 0.0) && (rho0.re != 0.0 || rho0.im != 0.0))
        sc->beta = d2_of2(cdiv2(rho_new, rho0) * cdiv2(al, om));
    sc->rho = d2_of2(rho_new);
}

// rhat = r, p = v = 0, xlo = 0; rr = |r|^2, rho = rr, alpha = omega = rho0 = 1
__global__ void __launch_bounds__(kRedBlock) k_lo_init(long long n, const float4 *r, float4 *rhat, float4 *p,
                                                       float4 *v, float4 *xlo, ReduceScratch rs, SolverScalars *sc)
{
    float acc[1] = {0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 ri = r[i];
        rhat[i] = ri;
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        xlo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        acc[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, fmaf(ri.z, ri.z, fmaf(ri.w, ri.w, acc[0]))));
    }
    if (grid_reduce_f<1>(acc, rs, rs.result)) lo_init_update(rs.result, sc);
}

// p = r + beta (p - omega v)
__device__ __forceinline__ void body_lo_p(long long n, const float4 *r, const float4 *v, float4 *p,
                                                    const SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    const cx<float> beta = mkc((float)sc->beta.x, (float)sc->beta.y);
    const cx<float> omega = mkc((float)sc->omega.x, (float)sc->omega.y);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cx<float> r0, r1, v0, v1, p0, p1;
        ld4(r, i, r0, r1);
        ld4(v, i, v0, v1);
        ld4(p, i, p0, p1);
        p0 = r0 + beta * (p0 - omega * v0);
        p1 = r1 + beta * (p1 - omega * v1);
        st4(p, i, p0, p1);
    }
}
__global__ void __launch_bounds__(kRedBlock) k_lo_p(long long n, const float4 *r, const float4 *v, float4 *p,
                                                    const SolverScalars *sc)
{
    body_lo_p(n, r, v, p, sc);
}

// alpha = rho / <rhat, v>
__device__ __forceinline__ void body_lo_alpha(long long n, const float4 *rhat, const float4 *v,
                                                        ReduceScratch rs, SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    float acc[2] = {0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 a = rhat[i], b = v[i];
        acc[0] = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc[0]))));
        acc[1] = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, acc[1]))));
    }
    if (grid_reduce_f<2>(acc, rs, rs.result)) lo_alpha_update(rs.result, sc);
}
__global__ void __launch_bounds__(kRedBlock) k_lo_alpha(long long n, const float4 *rhat, const float4 *v,
                                                        ReduceScratch rs, SolverScalars *sc)
{
    body_lo_alpha(n, rhat, v, rs, sc);
}

// s = r - alpha v
__device__ __forceinline__ void body_lo_s(long long n, const float4 *r, const float4 *v, float4 *s,
                                                    const SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    const cx<float> alpha = mkc((float)sc->alpha.x, (float)sc->alpha.y);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cx<float> r0, r1, v0, v1;
        ld4(r, i, r0, r1);
        ld4(v, i, v0, v1);
        st4(s, i, r0 - alpha * v0, r1 - alpha * v1);
    }
}
__global__ void __launch_bounds__(kRedBlock) k_lo_s(long long n, const float4 *r, const float4 *v, float4 *s,
                                                    const SolverScalars *sc)
{
    body_lo_s(n, r, v, s, sc);
}

// omega = <t, s> / <t, t>
__device__ __forceinline__ void body_lo_omega(long long n, const float4 *t, const float4 *s,
                                                        ReduceScratch rs, SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 a = t[i], b = s[i];
        acc[0] = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc[0]))));
        acc[1] = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, acc[1]))));
        acc[2] = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, acc[2]))));
        acc[3] = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, acc[3]))));
    }
    if (grid_reduce_f<4>(acc, rs, rs.result)) lo_omega_update(rs.result, sc);
}
__global__ void __launch_bounds__(kRedBlock) k_lo_omega(long long n, const float4 *t, const float4 *s,
                                                        ReduceScratch rs, SolverScalars *sc)
{
    body_lo_omega(n, t, s, rs, sc);
}

// xlo += alpha phat + omega shat; r = s - omega t; rho' = <rhat, r>, rr = |r|^2
__device__ __forceinline__ void body_lo_xr(long long n, float4 *xlo, const float4 *phat,
                                                     const float4 *shat, const float4 *s, const float4 *t,
                                                     float4 *r, const float4 *rhat, ReduceScratch rs,
                                                     SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    const cx<float> alpha = mkc((float)sc->alpha.x, (float)sc->alpha.y);
    const cx<float> omega = mkc((float)sc->omega.x, (float)sc->omega.y);
    float acc[3] = {0.f, 0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cx<float> x0, x1, a0, a1, b0, b1, s0, s1, t0, t1, h0, h1;
        ld4(xlo, i, x0, x1);
        ld4(phat, i, a0, a1);
        ld4(shat, i, b0, b1);
        x0 = cfma(omega, b0, cfma(alpha, a0, x0));
        x1 = cfma(omega, b1, cfma(alpha, a1, x1));
        st4(xlo, i, x0, x1);
        ld4(s, i, s0, s1);
        ld4(t, i, t0, t1);
        const cx<float> r0 = s0 - omega * t0, r1 = s1 - omega * t1;
        st4(r, i, r0, r1);
        ld4(rhat, i, h0, h1);
        acc[0] += h0.re * r0.re + h0.im * r0.im + h1.re * r1.re + h1.im * r1.im;
        acc[1] += h0.re * r0.im - h0.im * r0.re + h1.re * r1.im - h1.im * r1.re;
        acc[2] += r0.re * r0.re + r0.im * r0.im + r1.re * r1.re + r1.im * r1.im;
    }
    if (grid_reduce_f<3>(acc, rs, rs.result)) lo_xr_update(rs.result, sc);
}
__global__ void __launch_bounds__(kRedBlock) k_lo_xr(long long n, float4 *xlo, const float4 *phat,
                                                     const float4 *shat, const float4 *s, const float4 *t,
                                                     float4 *r, const float4 *rhat, ReduceScratch rs,
                                                     SolverScalars *sc)
{
    body_lo_xr(n, xlo, phat, shat, s, t, r, rhat, rs, sc);
}

// ------------------------------------------------------------------------
// The same updates with FP16 storage (per-site scale) of the BiCGStab
// vectors: one site per thread, FP32 arithmetic, FP32 partial sums; the
// accumulated correction xlo stays FP32.  The scalar updates are shared.
// ------------------------------------------------------------------------

struct HF {   // FP16 field: values and per-site scales
    void *d;
    float *n;
};

__device__ __forceinline__ void hld(const HF &f, int V, int x, cx<float> s[12]) { P16::load_spinor(f.d, f.n, V, x, s); }
__device__ __forceinline__ void hst(const HF &f, int V, int x, const cx<float> s[12])
{
    P16::store_spinor(f.d, f.n, V, x, s);
}

__global__ void __launch_bounds__(kRedBlock) k_lo_init_h(int V, HF r, HF rhat, HF p, HF v, float4 *xlo,
                                                         ReduceScratch rs, SolverScalars *sc)
{
    float acc[1] = {0.f};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<float> a[12], z[12];
        hld(r, V, x, a);
        hst(rhat, V, x, a);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            z[k] = mkc(0.f, 0.f);
            acc[0] = fmaf(a[k].re, a[k].re, fmaf(a[k].im, a[k].im, acc[0]));
        }
        hst(p, V, x, z);
        hst(v, V, x, z);
        P32::store_spinor(xlo, nullptr, V, x, z);
    }
    if (grid_reduce_f<1>(acc, rs, rs.result)) lo_init_update(rs.result, sc);
}

__device__ __forceinline__ void body_lo_p_h(int V, HF r, HF v, HF p, const SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    const cx<float> beta = mkc((float)sc->beta.x, (float)sc->beta.y);
    const cx<float> omega = mkc((float)sc->omega.x, (float)sc->omega.y);
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<float> a[12], b[12], c[12];
        hld(r, V, x, a);
        hld(v, V, x, b);
        hld(p, V, x, c);
#pragma unroll
        for (int k = 0; k < 12; ++k) c[k] = a[k] + beta * (c[k] - omega * b[k]);
        hst(p, V, x, c);
    }
}
__global__ void __launch_bounds__(kRedBlock) k_lo_p_h(int V, HF r, HF v, HF p, const SolverScalars *sc)
{
    body_lo_p_h(V, r, v, p, sc);
}

// acc[0] + i acc[1] += <a, b> over 12 components
__device__ __forceinline__ void cdot_acc(const cx<float> a[12], const cx<float> b[12], float acc[2])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        acc[0] = fmaf(a[k].re, b[k].re, fmaf(a[k].im, b[k].im, acc[0]));
        acc[1] = fmaf(a[k].re, b[k].im, fmaf(-a[k].im, b[k].re, acc[1]));
    }
}

__device__ __forceinline__ void body_lo_alpha_h(int V, HF rhat, HF v, ReduceScratch rs,
                                                          SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    float acc[2] = {0.f, 0.f};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<float> a[12], b[12];
        hld(rhat, V, x, a);
        hld(v, V, x, b);
        cdot_acc(a, b, acc);
    }
    if (grid_reduce_f<2>(acc, rs, rs.result)) lo_alpha_update(rs.result, sc);
}
__global__ void __launch_bounds__(kRedBlock) k_lo_alpha_h(int V, HF rhat, HF v, ReduceScratch rs,
                                                          SolverScalars *sc)
{
    body_lo_alpha_h(V, rhat, v, rs, sc);
}

__device__ __forceinline__ void body_lo_s_h(int V, HF r, HF v, HF s, const SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    const cx<float> alpha = mkc((float)sc->alpha.x, (float)sc->alpha.y);
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<float> a[12], b[12];
        hld(r, V, x, a);
        hld(v, V, x, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) a[k] = a[k] - alpha * b[k];
        hst(s, V, x, a);
    }
}
__global__ void __launch_bounds__(kRedBlock) k_lo_s_h(int V, HF r, HF v, HF s, const SolverScalars *sc)
{
    body_lo_s_h(V, r, v, s, sc);
}

__device__ __forceinline__ void body_lo_omega_h(int V, HF t, HF s, ReduceScratch rs, SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<float> a[12], b[12];
        hld(t, V, x, a);
        hld(s, V, x, b);
        cdot_acc(a, b, acc);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[2] = fmaf(a[k].re, a[k].re, fmaf(a[k].im, a[k].im, acc[2]));
            acc[3] = fmaf(b[k].re, b[k].re, fmaf(b[k].im, b[k].im, acc[3]));
        }
    }
    if (grid_reduce_f<4>(acc, rs, rs.result)) lo_omega_update(rs.result, sc);
}
__global__ void __launch_bounds__(kRedBlock) k_lo_omega_h(int V, HF t, HF s, ReduceScratch rs, SolverScalars *sc)
{
    body_lo_omega_h(V, t, s, rs, sc);
}

__device__ __forceinline__ void body_lo_xr_h(int V, float4 *xlo, HF phat, HF shat, HF s, HF t, HF r,
                                                       HF rhat, ReduceScratch rs, SolverScalars *sc)
{
    if (sc->skip) return;   // a stopped right-hand side of a lockstep batch
    const cx<float> alpha = mkc((float)sc->alpha.x, (float)sc->alpha.y);
    const cx<float> omega = mkc((float)sc->omega.x, (float)sc->omega.y);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<float> xs[12], a[12], b[12];
        P32::load_spinor(xlo, nullptr, V, x, xs);
        hld(phat, V, x, a);
        hld(shat, V, x, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) xs[k] = cfma(omega, b[k], cfma(alpha, a[k], xs[k]));
        P32::store_spinor(xlo, nullptr, V, x, xs);
        hld(s, V, x, a);
        hld(t, V, x, b);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            a[k] = a[k] - omega * b[k];
            acc[2] = fmaf(a[k].re, a[k].re, fmaf(a[k].im, a[k].im, acc[2]));
        }
        hst(r, V, x, a);
        hld(rhat, V, x, b);
        cdot_acc(b, a, acc);
    }
    if (grid_reduce_f<3>(acc, rs, rs.result)) lo_xr_update(rs.result, sc);
}
__global__ void __launch_bounds__(kRedBlock) k_lo_xr_h(int V, float4 *xlo, HF phat, HF shat, HF s, HF t, HF r,
                                                       HF rhat, ReduceScratch rs, SolverScalars *sc)
{
    body_lo_xr_h(V, xlo, phat, shat, s, t, r, rhat, rs, sc);
}

// End of a reliable update in one pass (the FP64 residual, its
// low-precision copy and the new rho of the recurrence): r = b - r (r holds
// op x), rr = |r|^2; rlo = r rounded to the Krylov storage PL (FP32, or
// FP16 with its per-site scale); rho = <rhat, rlo> of the stored rlo and
// beta from rho0, alpha, omega of the last step (lo_rho_update).  One site
// per thread.
template <class PL>
__global__ void __launch_bounds__(kRedBlock) k_refresh_tail(int V, const void *b, void *r, void *rlo, float *rlo_n,
                                                            const void *rhat, const float *rhat_n, ReduceScratch rs,
                                                            SolverScalars *sc)
{
    double acc[3] = {0.0, 0.0, 0.0};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        cx<double> bv[12], rv[12];
        P64::load_spinor(b, nullptr, V, x, bv);
        P64::load_spinor(r, nullptr, V, x, rv);
        cx<float> lo[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            rv[k] = bv[k] - rv[k];
            acc[0] += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
            lo[k] = mkc((float)rv[k].re, (float)rv[k].im);
        }
        P64::store_spinor(r, nullptr, V, x, rv);
        PL::store_spinor(rlo, rlo_n, V, x, lo);
        PL::as_stored(lo);
        cx<float> h[12];
        PL::load_spinor(rhat, rhat_n, V, x, h);
        float d[2] = {0.f, 0.f};
        cdot_acc(h, lo, d);
        acc[1] += d[0];
        acc[2] += d[1];
    }
    if (grid_reduce<3>(acc, rs, rs.result)) {
        sc->rr = rs.result[0];
        lo_rho_update(rs.result + 1, sc);
    }
}

// The step kernels for all members of a lockstep group: member blockIdx.y,
// its part of the grid blockIdx.x (grid-stride loops and the block-partial
// reductions use only the x extent).
template <bool HALF, int STEP>
__global__ void __launch_bounds__(kRedBlock) k_lo_group(int V, const LoMember *members)
{
    const LoMember &a = members[blockIdx.y];
    const long long n = 6LL * V;
    auto h = [](void *d, float *nrm) { return HF{d, nrm}; };
    auto c4 = [](void *d) { return static_cast<const float4 *>(d); };
    auto m4 = [](void *d) { return static_cast<float4 *>(d); };
    switch (STEP) {
    case LO_STEP_P:
        if (HALF) body_lo_p_h(V, h(a.r, a.rn), h(a.v, a.vn), h(a.p, a.pn), a.sc);
        else body_lo_p(n, c4(a.r), c4(a.v), m4(a.p), a.sc);
        break;
    case LO_STEP_ALPHA:
        if (HALF) body_lo_alpha_h(V, h(a.rhat, a.rhatn), h(a.v, a.vn), a.rs, a.sc);
        else body_lo_alpha(n, c4(a.rhat), c4(a.v), a.rs, a.sc);
        break;
    case LO_STEP_S:
        if (HALF) body_lo_s_h(V, h(a.r, a.rn), h(a.v, a.vn), h(a.s, a.sn), a.sc);
        else body_lo_s(n, c4(a.r), c4(a.v), m4(a.s), a.sc);
        break;
    case LO_STEP_OMEGA:
        if (HALF) body_lo_omega_h(V, h(a.t, a.tn), h(a.s, a.sn), a.rs, a.sc);
        else body_lo_omega(n, c4(a.t), c4(a.s), a.rs, a.sc);
        break;
    default:
        if (HALF)
            body_lo_xr_h(V, a.xlo, h(a.phat, a.phatn), h(a.shat, a.shatn), h(a.s, a.sn), h(a.t, a.tn),
                         h(a.r, a.rn), h(a.rhat, a.rhatn), a.rs, a.sc);
        else
            body_lo_xr(n, a.xlo, c4(a.phat), c4(a.shat), c4(a.s), c4(a.t), m4(a.r), c4(a.rhat), a.rs, a.sc);
        break;
    }
}

// The alpha or omega scalars of every member from the partial sums the
// even multi-RHS Schur pass wrote (one member per CTA, the partials summed
// in a fixed order, so the result does not depend on scheduling).
template <int STEP>
__global__ void __launch_bounds__(256) k_lo_group_finalize(int nblk, const double *part, const LoMember *members)
{
    const LoMember &a = members[blockIdx.x];
    if (a.sc->skip) return;   // its partials were not written
    const double *p = part + (size_t)blockIdx.x * nblk * 4;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < 4; ++c) t[c] += p[(size_t)b * 4 + c];
    __shared__ double sm[8][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) t[c] = warp_sum(t[c]);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) sm[wid][c] = t[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double res[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
            for (int c = 0; c < 4; ++c) res[c] += sm[w][c];
        if (STEP == LO_STEP_ALPHA)
            lo_alpha_update(res, a.sc);
        else
            lo_omega_update(res, a.sc);
    }
}

// x (FP64) += xlo (FP32); xlo = 0.  FP32 plane j holds components 2j and
// 2j+1 of each site; FP64 plane k holds component k.
__global__ void k_hp_add_lo(long long n, int V, double2 *x, float4 *xlo)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / V, site = i - j * V;
        const float4 a = xlo[i];
        double2 *x0 = x + (2 * j) * V + site;
        double2 *x1 = x0 + V;
        const double2 u = *x0, w = *x1;
        *x0 = make_double2(u.x + (double)a.x, u.y + (double)a.y);
        *x1 = make_double2(w.x + (double)a.z, w.y + (double)a.w);
        xlo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

}  // namespace

#define WC_GRID(n) reduce_grid(S.red, (n)), kRedBlock, 0, S.stream

cudaError_t bicg_init(wc_lattice lat, SolverState &S, const double2 *b, double2 *r, double2 *rhat, double2 *p,
                      double2 *v)
{
    const long long n = 12LL * lat->g.V;
    k_bicg_init<<<WC_GRID(n)>>>(n, b, r, rhat, p, v, S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t bicg_p(wc_lattice lat, SolverState &S, const double2 *r, const double2 *v, double2 *p)
{
    const long long n = 12LL * lat->g.V;
    k_bicg_p<<<WC_GRID(n)>>>(n, r, v, p, S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t bicg_alpha(wc_lattice lat, SolverState &S, const double2 *rhat, const double2 *v)
{
    const long long n = 12LL * lat->g.V;
    k_bicg_alpha<<<WC_GRID(n)>>>(n, rhat, v, S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t bicg_s(wc_lattice lat, SolverState &S, const double2 *r, const double2 *v, double2 *s)
{
    const long long n = 12LL * lat->g.V;
    k_bicg_s<<<WC_GRID(n)>>>(n, r, v, s, S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t bicg_omega(wc_lattice lat, SolverState &S, const double2 *t, const double2 *s)
{
    const long long n = 12LL * lat->g.V;
    k_bicg_omega<<<WC_GRID(n)>>>(n, t, s, S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t bicg_xr(wc_lattice lat, SolverState &S, double2 *x, const double2 *phat, const double2 *shat,
                    const double2 *s, const double2 *t, double2 *r, const double2 *rhat)
{
    const long long n = 12LL * lat->g.V;
    k_bicg_xr<<<WC_GRID(n)>>>(n, x, phat, shat, s, t, r, rhat, S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t residual(wc_lattice lat, SolverState &S, const double2 *b, double2 *r)
{
    const long long n = 12LL * lat->g.V;
    k_residual<<<WC_GRID(n)>>>(n, b, r, S.red, S.scal);
    return cudaGetLastError();
}
namespace {
float4 *f4(wc_field f) { return static_cast<float4 *>(f->data); }
HF hf(wc_field f) { return HF{f->data, f->nrm}; }
bool half_vectors(wc_field f) { return f->prec == WC_F16; }
}  // namespace

#define WC_GRID_SITES(V) reduce_grid(S.red, (V)), kRedBlock, 0, S.stream

cudaError_t lo_init(wc_lattice lat, SolverState &S, wc_field r, wc_field rhat, wc_field p, wc_field v, wc_field xlo)
{
    const int V = lat->g.V;
    const long long n = 6LL * V;
    if (half_vectors(r))
        k_lo_init_h<<<WC_GRID_SITES(V)>>>(V, hf(r), hf(rhat), hf(p), hf(v), f4(xlo), S.red, S.scal);
    else
        k_lo_init<<<WC_GRID(n)>>>(n, f4(r), f4(rhat), f4(p), f4(v), f4(xlo), S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t lo_p(wc_lattice lat, SolverState &S, wc_field r, wc_field v, wc_field p)
{
    const int V = lat->g.V;
    const long long n = 6LL * V;
    if (half_vectors(r))
        k_lo_p_h<<<WC_GRID_SITES(V)>>>(V, hf(r), hf(v), hf(p), S.scal);
    else
        k_lo_p<<<WC_GRID(n)>>>(n, f4(r), f4(v), f4(p), S.scal);
    return cudaGetLastError();
}
cudaError_t lo_alpha(wc_lattice lat, SolverState &S, wc_field rhat, wc_field v)
{
    const int V = lat->g.V;
    const long long n = 6LL * V;
    if (half_vectors(v))
        k_lo_alpha_h<<<WC_GRID_SITES(V)>>>(V, hf(rhat), hf(v), S.red, S.scal);
    else
        k_lo_alpha<<<WC_GRID(n)>>>(n, f4(rhat), f4(v), S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t lo_s(wc_lattice lat, SolverState &S, wc_field r, wc_field v, wc_field s)
{
    const int V = lat->g.V;
    const long long n = 6LL * V;
    if (half_vectors(r))
        k_lo_s_h<<<WC_GRID_SITES(V)>>>(V, hf(r), hf(v), hf(s), S.scal);
    else
        k_lo_s<<<WC_GRID(n)>>>(n, f4(r), f4(v), f4(s), S.scal);
    return cudaGetLastError();
}
cudaError_t lo_omega(wc_lattice lat, SolverState &S, wc_field t, wc_field s)
{
    const int V = lat->g.V;
    const long long n = 6LL * V;
    if (half_vectors(t))
        k_lo_omega_h<<<WC_GRID_SITES(V)>>>(V, hf(t), hf(s), S.red, S.scal);
    else
        k_lo_omega<<<WC_GRID(n)>>>(n, f4(t), f4(s), S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t lo_xr(wc_lattice lat, SolverState &S, wc_field xlo, wc_field phat, wc_field shat, wc_field s,
                  wc_field t, wc_field r, wc_field rhat)
{
    const int V = lat->g.V;
    const long long n = 6LL * V;
    if (half_vectors(r))
        k_lo_xr_h<<<WC_GRID_SITES(V)>>>(V, f4(xlo), hf(phat), hf(shat), hf(s), hf(t), hf(r), hf(rhat), S.red,
                                         S.scal);
    else
        k_lo_xr<<<WC_GRID(n)>>>(n, f4(xlo), f4(phat), f4(shat), f4(s), f4(t), f4(r), f4(rhat), S.red, S.scal);
    return cudaGetLastError();
}
cudaError_t refresh_tail(wc_lattice lat, SolverState &S, const wc_field b, wc_field r_hp, wc_field r, wc_field rhat)
{
    const int V = lat->g.V;
    if (half_vectors(r))
        k_refresh_tail<P16><<<WC_GRID_SITES(V)>>>(V, b->data, r_hp->data, r->data, r->nrm, rhat->data, rhat->nrm,
                                                  S.red, S.scal);
    else
        k_refresh_tail<P32><<<WC_GRID_SITES(V)>>>(V, b->data, r_hp->data, r->data, nullptr, rhat->data, nullptr,
                                                  S.red, S.scal);
    return cudaGetLastError();
}
LoMember lo_member(SolverState &S, wc_field r, wc_field rhat, wc_field p, wc_field v, wc_field s, wc_field t,
                   wc_field phat, wc_field shat, wc_field xlo)
{
    LoMember m{};
    m.r = r->data, m.rhat = rhat->data, m.p = p->data, m.v = v->data;
    m.s = s->data, m.t = t->data, m.phat = phat->data, m.shat = shat->data;
    m.rn = r->nrm, m.rhatn = rhat->nrm, m.pn = p->nrm, m.vn = v->nrm;
    m.sn = s->nrm, m.tn = t->nrm, m.phatn = phat->nrm, m.shatn = shat->nrm;
    m.xlo = f4(xlo);
    m.rs = S.red;
    m.sc = S.scal;
    return m;
}

cudaError_t lo_group(LoStep step, wc_lattice lat, int m, const LoMember *members, bool half, int max_blocks,
                     cudaStream_t stream)
{
    if (m < 1 || m > 65535) return cudaErrorInvalidValue;
    const int V = lat->g.V;
    // about max_blocks blocks in all (each member reduces over its own
    // gridDim.x partials, at most max_blocks of them)
    const long long work = half ? (long long)V : 6LL * V;
    long long gx = (work + kRedBlock - 1) / kRedBlock;
    const long long share = std::max<long long>(1, (max_blocks + m - 1) / m);
    const long long floor_blocks = std::max(1, max_blocks / 8);   // one per SM
    gx = std::max<long long>(1, std::min<long long>(std::min<long long>(gx, max_blocks),
                                                    std::max<long long>(share, floor_blocks)));
    const dim3 grid((unsigned)gx, (unsigned)m);
#define WC_GROUP_LAUNCH(S)                                                     \
    if (half) k_lo_group<true, S><<<grid, kRedBlock, 0, stream>>>(V, members); \
    else k_lo_group<false, S><<<grid, kRedBlock, 0, stream>>>(V, members)
    switch (step) {
    case LO_STEP_P: WC_GROUP_LAUNCH(LO_STEP_P); break;
    case LO_STEP_ALPHA: WC_GROUP_LAUNCH(LO_STEP_ALPHA); break;
    case LO_STEP_S: WC_GROUP_LAUNCH(LO_STEP_S); break;
    case LO_STEP_OMEGA: WC_GROUP_LAUNCH(LO_STEP_OMEGA); break;
    case LO_STEP_XR: WC_GROUP_LAUNCH(LO_STEP_XR); break;
    default: return cudaErrorInvalidValue;
    }
#undef WC_GROUP_LAUNCH
    return cudaGetLastError();
}

cudaError_t lo_group_finalize(LoStep step, int m, int nblk, const double *part, const LoMember *members,
                              cudaStream_t stream)
{
    if (m < 1 || nblk < 1) return cudaErrorInvalidValue;
    if (step == LO_STEP_ALPHA)
        k_lo_group_finalize<LO_STEP_ALPHA><<<m, 256, 0, stream>>>(nblk, part, members);
    else if (step == LO_STEP_OMEGA)
        k_lo_group_finalize<LO_STEP_OMEGA><<<m, 256, 0, stream>>>(nblk, part, members);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t hp_add_lo(wc_lattice lat, SolverState &S, double2 *x, wc_field xlo_f)
{
    float4 *xlo = f4(xlo_f);
    const long long n = 6LL * lat->g.V;
    k_hp_add_lo<<<WC_GRID(n)>>>(n, lat->g.V, x, xlo);
    return cudaGetLastError();
}

cudaError_t norm2_to_result(wc_lattice lat, SolverState &S, const double2 *a)
{
    const long long n = 12LL * lat->g.V;
    k_norm2_flat<<<WC_GRID(n)>>>(n, a, S.red);
    return cudaGetLastError();
}

}  // namespace wc
