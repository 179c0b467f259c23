// C ABI entry points: lattices, fields, gauge/clover loading, applies.
//
// Field transfers convert between the caller's canonical layout (complex128
// or complex64, site-major) and the plane-major device layouts in one kernel
// per call.  The synchronous calls stage host data in a lattice-owned
// buffer and return when the caller's memory may be reused; the
// asynchronous calls take device or page-locked host memory, copy host data
// in on a second stream of the lattice (so that the next input crosses the
// host link while the current step computes and copies its result out) and
// leave the caller to wc_sync.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <new>

#include <vector>

#include "wc_internal.cuh"

namespace wc {

namespace {
thread_local std::string g_global_error;
}

wc_status set_error(wc_lattice lat, wc_status st, const std::string &msg)
{
    if (st == WC_OK) return st;
    if (lat)
        lat->err = msg;
    else
        g_global_error = msg;
    return st;
}

wc_status check_cuda(wc_lattice lat, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return WC_OK;
    return set_error(lat, WC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

wc_status check_launch(wc_lattice lat, const char *what) { return check_cuda(lat, cudaGetLastError(), what); }

int sm_count()
{
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    });
    return n;
}

namespace {

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------------
// canonical <-> internal
// ------------------------------------------------------------------------

// T: double2 (canonical complex128) or float2 (canonical complex64)
template <class P, class T>
__global__ void k_import(int V, const T *src, void *dst, float *nrm)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    using R = typename P::real;
    cx<R> s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const T v = src[(size_t)x * 12 + k];
        s[k] = mkc((R)v.x, (R)v.y);
    }
    P::store_spinor(dst, nrm, V, x, s);
}

template <class P, class T>
__global__ void k_export(int V, const void *src, const float *nrm, T *dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    using E = decltype(T::x);
    cx<typename P::real> s[12];
    P::load_spinor(src, nrm, V, x, s);
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[(size_t)x * 12 + k] = T{(E)s[k].re, (E)s[k].im};
}

// canonical U[V][4][3][3] -> two-row stores in three precisions
__global__ void k_pack_gauge(int V, const double2 *U, GaugeStore g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * V) return;
    const int x = i % V, mu = i / V;
    const double2 *u = U + ((size_t)x * 4 + mu) * 9;  // rows 0 and 1 = entries 0..5
    double2 a[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = u[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        g.u64[((size_t)mu * 9 + k) * V + x] = a[k];
        g.udf[((size_t)mu * 9 + k) * V + x] = df_pack(a[k]);
    }
    cx<double> r01[6], r2[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) r01[k] = mkc(a[k].x, a[k].y);
    reconstruct_row2(r01, r2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 v = make_double2(r2[k].re, r2[k].im);
        g.u64[((size_t)mu * 9 + 6 + k) * V + x] = v;
        g.udf[((size_t)mu * 9 + 6 + k) * V + x] = df_pack(v);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
        g.u32[((size_t)mu * 3 + j) * V + x] =
            make_float4((float)a[2 * j].x, (float)a[2 * j].y, (float)a[2 * j + 1].x, (float)a[2 * j + 1].y);
    uint4 h;
    h.x = c2h((float)a[0].x, (float)a[0].y);
    h.y = c2h((float)a[1].x, (float)a[1].y);
    h.z = c2h((float)a[2].x, (float)a[2].y);
    h.w = c2h((float)a[3].x, (float)a[3].y);
    uint2 h2;
    h2.x = c2h((float)a[4].x, (float)a[4].y);
    h2.y = c2h((float)a[5].x, (float)a[5].y);
    g.u16a[(size_t)mu * V + x] = h;
    g.u16b[(size_t)mu * V + x] = h2;
}

// ------------------------------------------------------------------------
// clover term (FP64 arithmetic)
// ------------------------------------------------------------------------

struct M3 {
    cx<double> m[3][3];
};

__device__ M3 m3_mul(const M3 &a, const M3 &b)
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

__device__ M3 m3_dag(const M3 &a)
{
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

__device__ M3 load_u(const GaugeStore &g, int V, int mu, int x)
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

__device__ int shifted(const Geom &g, const int c[4], int mu, int dmu, int nu, int dnu)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + dmu + g.L[mu]) % g.L[mu];
    d[nu] = (d[nu] + dnu + g.L[nu]) % g.L[nu];
    return d[0] + g.stride[1] * d[1] + g.stride[2] * d[2] + g.stride[3] * d[3];
}

// Fhat_munu(x) = (1/8)[(Q - Q^+) - tr(Q - Q^+)/3], Q the four-leaf clover
__device__ M3 field_strength(const Geom &g, const GaugeStore &G, int x, const int c[4], int mu, int nu)
{
    const int V = g.V;
    const int xpm = shifted(g, c, mu, 1, nu, 0), xpn = shifted(g, c, mu, 0, nu, 1);
    const int xmm = shifted(g, c, mu, -1, nu, 0), xmn = shifted(g, c, mu, 0, nu, -1);
    const int xmm_pn = shifted(g, c, mu, -1, nu, 1), xmm_mn = shifted(g, c, mu, -1, nu, -1);
    const int xpm_mn = shifted(g, c, mu, 1, nu, -1);
    M3 Q;
    // leaf x -> x+mu -> x+mu+nu -> x+nu -> x
    M3 l = m3_mul(m3_mul(load_u(G, V, mu, x), load_u(G, V, nu, xpm)),
                  m3_mul(m3_dag(load_u(G, V, mu, xpn)), m3_dag(load_u(G, V, nu, x))));
    Q = l;
    // leaf x -> x+nu -> x+nu-mu -> x-mu -> x
    l = m3_mul(m3_mul(load_u(G, V, nu, x), m3_dag(load_u(G, V, mu, xmm_pn))),
               m3_mul(m3_dag(load_u(G, V, nu, xmm)), load_u(G, V, mu, xmm)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + l.m[i][j];
    // leaf x -> x-mu -> x-mu-nu -> x-nu -> x
    l = m3_mul(m3_mul(m3_dag(load_u(G, V, mu, xmm)), m3_dag(load_u(G, V, nu, xmm_mn))),
               m3_mul(load_u(G, V, mu, xmm_mn), load_u(G, V, nu, xmn)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + l.m[i][j];
    // leaf x -> x-nu -> x-nu+mu -> x+mu -> x
    l = m3_mul(m3_mul(m3_dag(load_u(G, V, nu, xmn)), load_u(G, V, mu, xmn)),
               m3_mul(load_u(G, V, nu, xpm_mn), m3_dag(load_u(G, V, mu, x))));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + l.m[i][j];
    M3 F;
    cx<double> tr = mkc(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            F.m[i][j] = Q.m[i][j] - conj(Q.m[j][i]);
            if (i == j) tr = tr + F.m[i][i];
        }
    const cx<double> t3 = (1.0 / 3.0) * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i) F.m[i][i] = F.m[i][i] - t3;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F.m[i][j] = 0.125 * F.m[i][j];
    return F;
}

// Block b of A = 1 + T.  In the chiral basis sigma_munu restricted to spin
// pair b is (eta = -1 for b = 0, +1 for b = 1):
//   sigma_xy = -s3, sigma_xz = s2, sigma_yz = -s1,
//   sigma_xt = eta s1, sigma_yt = eta s2, sigma_zt = eta s3,
// so the block is 1 + i csw kappa [[E3, E1 - i E2], [E1 + i E2, -E3]] with
// E1 = -F_yz + eta F_xt, E2 = F_xz + eta F_yt, E3 = -F_xy + eta F_zt.
__global__ void k_build_clover(Geom g, GaugeStore G, CloverStore C, double csw, double kappa)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    int c[4];
    site_coords(g, x, c);
    const M3 Fxy = field_strength(g, G, x, c, 0, 1), Fxz = field_strength(g, G, x, c, 0, 2);
    const M3 Fxt = field_strength(g, G, x, c, 0, 3), Fyz = field_strength(g, G, x, c, 1, 2);
    const M3 Fyt = field_strength(g, G, x, c, 1, 3), Fzt = field_strength(g, G, x, c, 2, 3);
    const double ck = csw * kappa;
    const int V = g.V;
    for (int b = 0; b < 2; ++b) {
        const double eta = b == 0 ? -1.0 : 1.0;
        cx<double> blk[6][6];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const cx<double> e1 = (-1.0) * Fyz.m[i][j] + eta * Fxt.m[i][j];
                const cx<double> e2 = Fxz.m[i][j] + eta * Fyt.m[i][j];
                const cx<double> e3 = (-1.0) * Fxy.m[i][j] + eta * Fzt.m[i][j];
                // i*ck*(...) for the four spin sub-blocks
                blk[i][j] = ck * times_i(e3);
                blk[3 + i][3 + j] = (-ck) * times_i(e3);
                blk[i][3 + j] = ck * times_i(e1 - times_i(e2));
                blk[3 + i][j] = ck * times_i(e1 + times_i(e2));
            }
        double r[36];
#pragma unroll
        for (int i = 0; i < 6; ++i) r[i] = 1.0 + blk[i][i].re;
        int k = 6;
#pragma unroll
        for (int i = 1; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j) {
                r[k++] = blk[i][j].re;
                r[k++] = blk[i][j].im;
            }
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const double2 v = make_double2(r[2 * q], r[2 * q + 1]);
            C.c64[((size_t)b * 18 + q) * V + x] = v;
            C.cdf[((size_t)b * 18 + q) * V + x] = df_pack(v);
        }
#pragma unroll
        for (int q = 0; q < 9; ++q)
            C.c32[((size_t)b * 9 + q) * V + x] =
                make_float4((float)r[4 * q], (float)r[4 * q + 1], (float)r[4 * q + 2], (float)r[4 * q + 3]);
        // FP16: 18 half2 per block, global half2 index 18b + q, 4 per uint4
        unsigned hw[18];
#pragma unroll
        for (int q = 0; q < 18; ++q) hw[q] = c2h((float)r[2 * q], (float)r[2 * q + 1]);
        unsigned *c16 = reinterpret_cast<unsigned *>(C.c16);
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const int gq = 18 * b + q;
            c16[((size_t)(gq >> 2) * V + x) * 4 + (gq & 3)] = hw[q];
        }
    }
}

template <class T>
cudaError_t dalloc(T **p, size_t bytes)
{
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

void free_gauge(GaugeStore &g)
{
    cudaFree(g.u64);
    cudaFree(g.udf);
    cudaFree(g.u32);
    cudaFree(g.u16a);
    cudaFree(g.u16b);
    g = GaugeStore{};
}

void free_clover(CloverStore &c)
{
    cudaFree(c.c64);
    cudaFree(c.cdf);
    cudaFree(c.c32);
    cudaFree(c.c16);
    c = CloverStore{};
}

wc_status need_staging(wc_lattice lat, size_t bytes)
{
    if (lat->staging_bytes >= bytes) return WC_OK;
    cudaFree(lat->staging);
    lat->staging = nullptr;
    lat->staging_bytes = 0;
    wc_status st = check_cuda(lat, dalloc(&lat->staging, bytes), "cudaMalloc(staging)");
    if (st == WC_OK) lat->staging_bytes = bytes;
    return st;
}

wc_status check_field(wc_lattice lat, wc_field f, const char *name)
{
    if (!f) return set_error(lat, WC_ERR_ARG, std::string(name) + " is NULL");
    if (f->lat != lat) return set_error(lat, WC_ERR_ARG, std::string(name) + " belongs to another lattice");
    return WC_OK;
}

}  // namespace

// readers of the per-translation-unit violation counters (checked build)
std::vector<cudaError_t (*)(unsigned *)> &check_readers()
{
    static std::vector<cudaError_t (*)(unsigned *)> r;
    return r;
}

void register_check_counter(cudaError_t (*read)(unsigned *)) { check_readers().push_back(read); }

wc_status require_operator(wc_lattice lat, bool need_clover)
{
    if (lat->split_mask)
        return set_error(lat, WC_ERR_ARG,
                         "sub-domain lattice: its operator needs the neighbours' face data (wc_halo_pack, "
                         "wc_apply_interior, wc_apply_surface)");
    if (!lat->gauge_loaded) return set_error(lat, WC_ERR_STATE, "gauge field not loaded");
    if (need_clover && !lat->clover_loaded) return set_error(lat, WC_ERR_STATE, "clover term not loaded");
    return WC_OK;
}

wc_status state_init(wc_lattice lat, SolverState &s)
{
    const int max_blocks = 8 * sm_count();
    s.red.max_blocks = max_blocks;
    wc_status st = check_cuda(lat, dalloc(&s.red.partials, sizeof(double) * 8 * max_blocks), "cudaMalloc");
    if (st == WC_OK) st = check_cuda(lat, dalloc(&s.red.ticket, sizeof(unsigned)), "cudaMalloc");
    if (st == WC_OK) st = check_cuda(lat, dalloc(&s.red.result, sizeof(double) * 8), "cudaMalloc");
    if (st == WC_OK)
        st = check_cuda(lat, cudaMallocHost(reinterpret_cast<void **>(&s.red.host_result), sizeof(double) * 8),
                        "cudaMallocHost");
    if (st == WC_OK) st = check_cuda(lat, dalloc(&s.scal, sizeof(SolverScalars)), "cudaMalloc");
    if (st == WC_OK)
        st = check_cuda(lat, cudaMallocHost(reinterpret_cast<void **>(&s.scal_host), sizeof(SolverScalars)),
                        "cudaMallocHost");
    if (st == WC_OK) st = check_cuda(lat, cudaMemset(s.red.ticket, 0, sizeof(unsigned)), "cudaMemset");
    if (st == WC_OK) st = check_cuda(lat, cudaMemset(s.scal, 0, sizeof(SolverScalars)), "cudaMemset");
    if (st != WC_OK) state_free(s);
    return st;
}

void state_free(SolverState &s)
{
    if (s.inner) {
        state_free(*s.inner);
        delete s.inner;
        s.inner = nullptr;
    }
    for (auto &w : s.work) {
        wc_field_destroy(w);
        w = nullptr;
    }
    cudaFree(s.red.partials);
    cudaFree(s.red.ticket);
    cudaFree(s.red.result);
    cudaFreeHost(s.red.host_result);
    cudaFree(s.scal);
    cudaFreeHost(s.scal_host);
    s = SolverState{};
}

wc_field state_work(wc_lattice lat, SolverState &s, int slot, wc_prec prec, wc_status *st)
{
    if (!s.work[slot]) {
        *st = wc_field_create(lat, prec, &s.work[slot]);
        if (*st != WC_OK) return nullptr;
    }
    *st = WC_OK;
    return s.work[slot];
}

namespace {
}  // namespace
}  // namespace wc

using namespace wc;

namespace {

template <class T>
wc_status field_import(wc_field f, const T *data)
{
    if (!f) return set_error(nullptr, WC_ERR_ARG, "field is NULL");
    wc_lattice lat = f->lat;
    if (!data) return set_error(lat, WC_ERR_ARG, "data is NULL");
    const int V = lat->g.V;
    const size_t bytes = sizeof(T) * 12 * (size_t)V;
    const T *src = data;
    wc_status st = WC_OK;
    const bool host = !is_device_pointer(data);
    if (host) {
        st = need_staging(lat, bytes);
        if (st != WC_OK) return st;
        st = check_cuda(lat, cudaMemcpyAsync(lat->staging, data, bytes, cudaMemcpyHostToDevice, lat->stream),
                        "cudaMemcpyAsync(import)");
        if (st != WC_OK) return st;
        src = reinterpret_cast<const T *>(lat->staging);
    }
    dim3 grid((V + 255) / 256), block(256);
    if (f->prec == WC_F64)
        k_import<P64, T><<<grid, block, 0, lat->stream>>>(V, src, f->data, f->nrm);
    else if (f->prec == WC_F32)
        k_import<P32, T><<<grid, block, 0, lat->stream>>>(V, src, f->data, f->nrm);
    else
        k_import<P16, T><<<grid, block, 0, lat->stream>>>(V, src, f->data, f->nrm);
    st = check_launch(lat, "import");
    if (st == WC_OK && host) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync(import)");
    return st;
}

template <class T>
wc_status field_export(wc_field f, T *data)
{
    if (!f) return set_error(nullptr, WC_ERR_ARG, "field is NULL");
    wc_lattice lat = f->lat;
    if (!data) return set_error(lat, WC_ERR_ARG, "data is NULL");
    const int V = lat->g.V;
    const size_t bytes = sizeof(T) * 12 * (size_t)V;
    const bool host = !is_device_pointer(data);
    T *dst = data;
    wc_status st = WC_OK;
    if (host) {
        st = need_staging(lat, bytes);
        if (st != WC_OK) return st;
        dst = reinterpret_cast<T *>(lat->staging);
    }
    dim3 grid((V + 255) / 256), block(256);
    if (f->prec == WC_F64)
        k_export<P64, T><<<grid, block, 0, lat->stream>>>(V, f->data, f->nrm, dst);
    else if (f->prec == WC_F32)
        k_export<P32, T><<<grid, block, 0, lat->stream>>>(V, f->data, f->nrm, dst);
    else
        k_export<P16, T><<<grid, block, 0, lat->stream>>>(V, f->data, f->nrm, dst);
    st = check_launch(lat, "export");
    if (st == WC_OK && host) {
        st = check_cuda(lat, cudaMemcpyAsync(data, lat->staging, bytes, cudaMemcpyDeviceToHost, lat->stream),
                        "cudaMemcpyAsync(export)");
        if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync(export)");
    }
    return st;
}

bool is_pinned_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// copy stream, events and the two staging buffers of the asynchronous path.
// Everything is created into locals and handed to the lattice only when
// every step succeeded (the copy stream is set last: it marks the set-up as
// done); after a failure the partial resources are released and the next
// asynchronous call tries again.
wc_status async_setup(wc_lattice lat)
{
    if (lat->copy_stream) return WC_OK;
    const size_t bytes = sizeof(double2) * 12 * (size_t)lat->g.V;
    cudaStream_t cs = nullptr, co = nullptr;
    cudaEvent_t ev[6] = {};   // in ready, in free, out ready 0/1, out free 0/1
    double2 *in = nullptr, *out[2] = {nullptr, nullptr};
    wc_status st = check_cuda(lat, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate(copy)");
    if (st == WC_OK)
        st = check_cuda(lat, cudaStreamCreateWithFlags(&co, cudaStreamNonBlocking), "cudaStreamCreate(copy out)");
    for (int k = 0; k < 6 && st == WC_OK; ++k)
        st = check_cuda(lat, cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming), "cudaEventCreate");
    if (st == WC_OK) st = check_cuda(lat, dalloc(&in, bytes), "cudaMalloc(staging)");
    for (int b = 0; b < 2 && st == WC_OK; ++b) st = check_cuda(lat, dalloc(&out[b], bytes), "cudaMalloc(staging)");
    // nothing to wait for before the first copies
    if (st == WC_OK) st = check_cuda(lat, cudaEventRecord(ev[1], lat->stream), "cudaEventRecord");
    for (int b = 0; b < 2 && st == WC_OK; ++b)
        st = check_cuda(lat, cudaEventRecord(ev[4 + b], co), "cudaEventRecord");
    if (st != WC_OK) {
        if (cs) cudaStreamDestroy(cs);
        if (co) cudaStreamDestroy(co);
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        cudaFree(in);
        cudaFree(out[0]);
        cudaFree(out[1]);
        return st;
    }
    lat->ev_in_ready = ev[0];
    lat->ev_in_free = ev[1];
    for (int b = 0; b < 2; ++b) {
        lat->ev_out_ready[b] = ev[2 + b];
        lat->ev_out_free[b] = ev[4 + b];
        lat->astage_out[b] = out[b];
    }
    lat->astage_in = in;
    lat->out_buf = 0;
    lat->copy_out_stream = co;
    lat->copy_stream = cs;
    return WC_OK;
}

template <class T>
wc_status field_import_async(wc_field f, const T *data)
{
    if (!f) return set_error(nullptr, WC_ERR_ARG, "field is NULL");
    wc_lattice lat = f->lat;
    if (!data) return set_error(lat, WC_ERR_ARG, "data is NULL");
    const bool dev = is_device_pointer(data);
    if (!dev && !is_pinned_host(data))
        return set_error(lat, WC_ERR_ARG, "asynchronous import needs device or page-locked host memory");
    const int V = lat->g.V;
    const T *src = data;
    wc_status st = WC_OK;
    if (!dev) {
        st = async_setup(lat);
        if (st != WC_OK) return st;
        // the previous import kernel must have read the staging buffer
        st = check_cuda(lat, cudaStreamWaitEvent(lat->copy_stream, lat->ev_in_free, 0), "wait");
        if (st == WC_OK)
            st = check_cuda(lat, cudaMemcpyAsync(lat->astage_in, data, sizeof(T) * 12 * (size_t)V,
                                                 cudaMemcpyHostToDevice, lat->copy_stream), "cudaMemcpyAsync(import)");
        if (st == WC_OK) st = check_cuda(lat, cudaEventRecord(lat->ev_in_ready, lat->copy_stream), "record");
        if (st == WC_OK) st = check_cuda(lat, cudaStreamWaitEvent(lat->stream, lat->ev_in_ready, 0), "wait");
        if (st != WC_OK) return st;
        src = reinterpret_cast<const T *>(lat->astage_in);
    }
    dim3 grid((V + 255) / 256), block(256);
    if (f->prec == WC_F64)
        k_import<P64, T><<<grid, block, 0, lat->stream>>>(V, src, f->data, f->nrm);
    else if (f->prec == WC_F32)
        k_import<P32, T><<<grid, block, 0, lat->stream>>>(V, src, f->data, f->nrm);
    else
        k_import<P16, T><<<grid, block, 0, lat->stream>>>(V, src, f->data, f->nrm);
    st = check_launch(lat, "import");
    if (st == WC_OK && !dev) st = check_cuda(lat, cudaEventRecord(lat->ev_in_free, lat->stream), "record");
    return st;
}

template <class T>
wc_status field_export_async(wc_field f, T *data)
{
    if (!f) return set_error(nullptr, WC_ERR_ARG, "field is NULL");
    wc_lattice lat = f->lat;
    if (!data) return set_error(lat, WC_ERR_ARG, "data is NULL");
    const bool dev = is_device_pointer(data);
    if (!dev && !is_pinned_host(data))
        return set_error(lat, WC_ERR_ARG, "asynchronous export needs device or page-locked host memory");
    const int V = lat->g.V;
    T *dst = data;
    wc_status st = WC_OK;
    const int b = lat->out_buf;
    if (!dev) {
        st = async_setup(lat);
        if (st != WC_OK) return st;
        // the copy out that last used buffer b must be done
        st = check_cuda(lat, cudaStreamWaitEvent(lat->stream, lat->ev_out_free[b], 0), "wait");
        if (st != WC_OK) return st;
        dst = reinterpret_cast<T *>(lat->astage_out[b]);
    }
    dim3 grid((V + 255) / 256), block(256);
    if (f->prec == WC_F64)
        k_export<P64, T><<<grid, block, 0, lat->stream>>>(V, f->data, f->nrm, dst);
    else if (f->prec == WC_F32)
        k_export<P32, T><<<grid, block, 0, lat->stream>>>(V, f->data, f->nrm, dst);
    else
        k_export<P16, T><<<grid, block, 0, lat->stream>>>(V, f->data, f->nrm, dst);
    st = check_launch(lat, "export");
    if (st == WC_OK && !dev) {
        st = check_cuda(lat, cudaEventRecord(lat->ev_out_ready[b], lat->stream), "record");
        if (st == WC_OK)
            st = check_cuda(lat, cudaStreamWaitEvent(lat->copy_out_stream, lat->ev_out_ready[b], 0), "wait");
        if (st == WC_OK)
            st = check_cuda(lat, cudaMemcpyAsync(data, lat->astage_out[b], sizeof(T) * 12 * (size_t)V,
                                                 cudaMemcpyDeviceToHost, lat->copy_out_stream),
                            "cudaMemcpyAsync(export)");
        if (st == WC_OK) st = check_cuda(lat, cudaEventRecord(lat->ev_out_free[b], lat->copy_out_stream), "record");
        if (st == WC_OK) lat->out_buf = b ^ 1;
    }
    return st;
}

}  // namespace

extern "C" {

wc_status wc_create_lattice(const int dims[4], int t_bc, void *cuda_stream, wc_lattice *out)
{
    if (!dims || !out) return set_error(nullptr, WC_ERR_ARG, "dims and out must not be NULL");
    *out = nullptr;
    long long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2) return set_error(nullptr, WC_ERR_ARG, "every lattice extent must be >= 2");
        V *= dims[m];
    }
    if (V > (1LL << 30)) return set_error(nullptr, WC_ERR_ARG, "lattice volume above 2^30 sites");
    if (t_bc != 1 && t_bc != -1) return set_error(nullptr, WC_ERR_ARG, "t_bc must be +1 or -1");
    wc_lattice lat = new (std::nothrow) wc_lattice_s();
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "out of host memory");
    for (int m = 0; m < 4; ++m) lat->g.L[m] = dims[m];
    lat->g.stride[0] = 1;
    lat->g.stride[1] = dims[0];
    lat->g.stride[2] = dims[0] * dims[1];
    lat->g.stride[3] = dims[0] * dims[1] * dims[2];
    lat->g.V = (int)V;
    lat->g.tbc = t_bc;
    geom_set_div(lat->g);
    lat->stream = static_cast<cudaStream_t>(cuda_stream);
    wc_status st = state_init(lat, lat->st);
    if (st != WC_OK) {
        set_error(nullptr, st, lat->err);
        wc_destroy_lattice(lat);
        return st;
    }
    *out = lat;
    return WC_OK;
}

wc_status wc_destroy_lattice(wc_lattice lat)
{
    if (!lat) return WC_OK;
    cudaStreamSynchronize(lat->stream);
    free_batch_pool(lat);
    free_half(lat);
    state_free(lat->st);
    free_gauge(lat->gauge);
    free_clover(lat->clover);
    free_clover(lat->cinv);
    free_clover(lat->ceo);
    cudaFree(lat->staging);
    for (cudaStream_t cs : {lat->copy_stream, lat->copy_out_stream})
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
    for (cudaEvent_t e : {lat->ev_in_ready, lat->ev_in_free, lat->ev_out_ready[0], lat->ev_out_ready[1],
                          lat->ev_out_free[0], lat->ev_out_free[1]})
        if (e) cudaEventDestroy(e);
    cudaFree(lat->astage_in);
    cudaFree(lat->astage_out[0]);
    cudaFree(lat->astage_out[1]);
    wc_destroy_lattice(lat->ext);
    delete lat;
    return WC_OK;
}

wc_status wc_set_stream(wc_lattice lat, void *cuda_stream)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    lat->stream = static_cast<cudaStream_t>(cuda_stream);
    if (lat->ext) lat->ext->stream = lat->stream;
    return WC_OK;
}

wc_status wc_set_fp64_arith(wc_lattice lat, int arith)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (arith != WC_ARITH_F64 && arith != WC_ARITH_DF32) return set_error(lat, WC_ERR_ARG, "unknown FP64 arithmetic");
    lat->fp64_arith = arith;
    return WC_OK;
}

wc_status wc_load_gauge(wc_lattice lat, const double *data)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!data) return set_error(lat, WC_ERR_ARG, "gauge data is NULL");
    const int V = lat->g.V;
    GaugeStore &g = lat->gauge;
    wc_status st = WC_OK;
    if (!g.u64) {
        st = check_cuda(lat, dalloc(&g.u64, sizeof(double2) * 36 * (size_t)V), "cudaMalloc(gauge)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&g.udf, sizeof(float4) * 36 * (size_t)V), "cudaMalloc(gauge)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&g.u32, sizeof(float4) * 12 * (size_t)V), "cudaMalloc(gauge)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&g.u16a, sizeof(uint4) * 4 * (size_t)V), "cudaMalloc(gauge)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&g.u16b, sizeof(uint2) * 4 * (size_t)V), "cudaMalloc(gauge)");
        if (st != WC_OK) {
            free_gauge(g);
            return st;
        }
    }
    if (lat->split_mask) {
        // a sub-domain: data is the gauge field extended by one site across
        // every cut face; it is loaded on the extended lattice (where the
        // clover term will be built) and its interior copied here
        lat->ext->stream = lat->stream;
        st = wc_load_gauge(lat->ext, data);
        if (st != WC_OK) return set_error(lat, st, "extended gauge field: " + lat->ext->err);
        st = check_cuda(lat, extract_gauge(lat, lat->stream), "extract gauge");
        lat->gauge_loaded = (st == WC_OK);
        lat->clover_loaded = false;
        lat->cinv_loaded = false;
        return st;
    }
    const size_t bytes = sizeof(double2) * 36 * (size_t)V;
    const double2 *src = reinterpret_cast<const double2 *>(data);
    if (!is_device_pointer(data)) {
        st = need_staging(lat, bytes);
        if (st != WC_OK) return st;
        st = check_cuda(lat, cudaMemcpyAsync(lat->staging, data, bytes, cudaMemcpyHostToDevice, lat->stream),
                        "cudaMemcpyAsync(gauge)");
        if (st != WC_OK) return st;
        src = lat->staging;
    }
    k_pack_gauge<<<(4 * V + 255) / 256, 256, 0, lat->stream>>>(V, src, g);
    st = check_launch(lat, "pack_gauge");
    if (st != WC_OK) return st;
    // the host buffer must stay valid until the copy ran
    if (src == lat->staging) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync(gauge)");
    lat->gauge_loaded = (st == WC_OK);
    lat->clover_loaded = false;
    lat->cinv_loaded = false;
    return st;
}

wc_status wc_load_clover(wc_lattice lat, double csw, double kappa)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!lat->gauge_loaded) return set_error(lat, WC_ERR_STATE, "wc_load_clover before wc_load_gauge");
    if (!isfinite(csw) || !isfinite(kappa)) return set_error(lat, WC_ERR_ARG, "csw and kappa must be finite");
    const int V = lat->g.V;
    CloverStore &c = lat->clover;
    wc_status st = WC_OK;
    if (!c.c64) {
        st = check_cuda(lat, dalloc(&c.c64, sizeof(double2) * 36 * (size_t)V), "cudaMalloc(clover)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&c.cdf, sizeof(float4) * 36 * (size_t)V), "cudaMalloc(clover)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&c.c32, sizeof(float4) * 18 * (size_t)V), "cudaMalloc(clover)");
        if (st == WC_OK) st = check_cuda(lat, dalloc(&c.c16, sizeof(uint4) * 9 * (size_t)V), "cudaMalloc(clover)");
        if (st != WC_OK) {
            free_clover(c);
            return st;
        }
    }
    if (lat->split_mask) {
        // a sub-domain: built on the extended lattice, whose halo sites hold
        // the neighbours' links the face sites' clover leaves reach
        lat->ext->stream = lat->stream;
        st = wc_load_clover(lat->ext, csw, kappa);
        if (st != WC_OK) return set_error(lat, st, "extended lattice clover: " + lat->ext->err);
        st = check_cuda(lat, extract_clover(lat, lat->stream), "extract clover");
    } else {
        k_build_clover<<<(V + 63) / 64, 64, 0, lat->stream>>>(lat->g, lat->gauge, c, csw, kappa);
        st = check_launch(lat, "build_clover");
    }
    if (st != WC_OK) return st;
    lat->csw = csw;
    lat->kappa = kappa;
    lat->clover_loaded = true;
    lat->cinv_loaded = false;
    return WC_OK;
}

wc_status wc_field_create(wc_lattice lat, wc_prec prec, wc_field *out)
{
    if (!lat || !out) return set_error(lat, WC_ERR_ARG, "lattice and out must not be NULL");
    *out = nullptr;
    if (prec != WC_F64 && prec != WC_F32 && prec != WC_F16) return set_error(lat, WC_ERR_ARG, "bad precision");
    wc_field f = new (std::nothrow) wc_field_s();
    if (!f) return set_error(lat, WC_ERR_ARG, "out of host memory");
    f->lat = lat;
    f->prec = prec;
    wc_status st = check_cuda(lat, cudaMalloc(&f->data, spinor_bytes(prec, lat->g.V)), "cudaMalloc(field)");
    if (st == WC_OK && prec == WC_F16)
        st = check_cuda(lat, dalloc(&f->nrm, sizeof(float) * (size_t)lat->g.V), "cudaMalloc(field)");
    if (st == WC_OK) st = check_cuda(lat, cudaMemsetAsync(f->data, 0, spinor_bytes(prec, lat->g.V), lat->stream),
                                     "cudaMemset(field)");
    if (st == WC_OK && f->nrm)
        st = check_cuda(lat, cudaMemsetAsync(f->nrm, 0, sizeof(float) * (size_t)lat->g.V, lat->stream),
                        "cudaMemset(field)");
    if (st != WC_OK) {
        wc_field_destroy(f);
        return st;
    }
    *out = f;
    return WC_OK;
}

wc_status wc_field_destroy(wc_field f)
{
    if (!f) return WC_OK;
    // cudaFree waits for outstanding device work that may use the buffers
    cudaFree(f->data);
    cudaFree(f->nrm);
    delete f;
    return WC_OK;
}

wc_status wc_field_import(wc_field f, const double *data)
{
    return field_import(f, reinterpret_cast<const double2 *>(data));
}

wc_status wc_field_export(wc_field f, double *data)
{
    return field_export(f, reinterpret_cast<double2 *>(data));
}

wc_status wc_field_import_f32(wc_field f, const float *data)
{
    return field_import(f, reinterpret_cast<const float2 *>(data));
}

wc_status wc_field_import_async(wc_field f, const void *data, int complex64)
{
    return complex64 ? field_import_async(f, static_cast<const float2 *>(data))
                     : field_import_async(f, static_cast<const double2 *>(data));
}

wc_status wc_field_export_async(wc_field f, void *data, int complex64)
{
    return complex64 ? field_export_async(f, static_cast<float2 *>(data))
                     : field_export_async(f, static_cast<double2 *>(data));
}

wc_status wc_sync(wc_lattice lat)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    wc_status st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync");
    if (st == WC_OK && lat->copy_stream) st = check_cuda(lat, cudaStreamSynchronize(lat->copy_stream), "sync");
    if (st == WC_OK && lat->copy_out_stream)
        st = check_cuda(lat, cudaStreamSynchronize(lat->copy_out_stream), "sync");
    return st;
}

wc_status wc_field_export_f32(wc_field f, float *data)
{
    return field_export(f, reinterpret_cast<float2 *>(data));
}

wc_status wc_field_copy(wc_field dst, wc_field src, double scale)
{
    if (!dst || !src) return set_error(nullptr, WC_ERR_ARG, "field is NULL");
    wc_lattice lat = dst->lat;
    if (src->lat != lat) return set_error(lat, WC_ERR_ARG, "fields belong to different lattices");
    if (!isfinite(scale)) return set_error(lat, WC_ERR_ARG, "scale must be finite");
    return check_cuda(lat, launch_copy(lat, dst, src, scale, nullptr, 0, lat->stream), "field_copy");
}

static wc_status apply_common(wc_lattice lat, wc_field out, wc_field in, int kind)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    wc_status st = check_field(lat, out, "out");
    if (st == WC_OK) st = check_field(lat, in, "in");
    if (st != WC_OK) return st;
    if (out == in || out->data == in->data) return set_error(lat, WC_ERR_ARG, "out and in must be distinct fields");
    if (out->prec != in->prec) return set_error(lat, WC_ERR_ARG, "out and in must have the same precision");
    st = require_operator(lat, kind != 2);
    if (st != WC_OK) return st;
    return check_cuda(lat, launch_apply(lat, out, in, kind, lat->stream), "apply");
}

wc_status wc_apply_M(wc_lattice lat, wc_field out, wc_field in) { return apply_common(lat, out, in, 0); }

wc_status wc_apply_multi(wc_lattice lat, int n, wc_field *outs, wc_field *ins, int dagger)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (n < 1 || n > kMrhsMax || !outs || !ins)
        return set_error(lat, WC_ERR_ARG, "n must be in 1.." + std::to_string(kMrhsMax) + ", outs/ins non-NULL");
    for (int r = 0; r < n; ++r) {
        wc_status st = check_field(lat, outs[r], "out");
        if (st == WC_OK) st = check_field(lat, ins[r], "in");
        if (st != WC_OK) return st;
        if (outs[r]->prec != WC_F32 || ins[r]->prec != WC_F32)
            return set_error(lat, WC_ERR_ARG, "the multi-RHS operator takes FP32 fields");
        for (int q = 0; q < n; ++q)
            if (outs[r] == ins[q] || (q < r && outs[r] == outs[q]))
                return set_error(lat, WC_ERR_ARG, "out fields must be distinct from each other and from the inputs");
    }
    wc_status st = require_operator(lat);
    if (st != WC_OK) return st;
    return check_cuda(lat, launch_apply_multi(lat, n, outs, ins, dagger ? 1 : 0, nullptr, lat->stream),
                      "apply_multi");
}

wc_status wc_apply_schur(wc_lattice lat, wc_field out, wc_field in, int dagger)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    wc_status st = check_field(lat, out, "out");
    if (st == WC_OK) st = check_field(lat, in, "in");
    if (st != WC_OK) return st;
    if (out == in || out->prec != in->prec)
        return set_error(lat, WC_ERR_ARG, "out and in must be distinct fields of one precision");
    st = require_operator(lat);
    if (st != WC_OK) return st;
    wc_lattice h = nullptr;
    st = half_lattice(lat, &h);
    if (st != WC_OK) return st;
    wc_field e = nullptr, o = nullptr, r = nullptr;
    st = wc_field_create(h, in->prec, &e);
    if (st == WC_OK) st = wc_field_create(h, in->prec, &o);
    if (st == WC_OK) st = wc_field_create(h, in->prec, &r);
    if (st == WC_OK) st = check_cuda(lat, launch_split(lat, in, e, o, lat->stream), "split");
    if (st == WC_OK) st = check_cuda(lat, launch_schur(h, r, e, dagger ? 1 : 0, lat->stream), "schur");
    if (st == WC_OK) st = check_cuda(lat, launch_merge(lat, r, nullptr, out, lat->stream), "merge");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync");
    wc_field_destroy(e);
    wc_field_destroy(o);
    wc_field_destroy(r);
    return st;
}
wc_status wc_apply_Mdag(wc_lattice lat, wc_field out, wc_field in) { return apply_common(lat, out, in, 1); }
wc_status wc_apply_hop(wc_lattice lat, wc_field out, wc_field in) { return apply_common(lat, out, in, 2); }

wc_status wc_apply_shape(wc_lattice lat, wc_prec prec, int kind, int force_index, int shape_out[6])
{
    if (!lat || !shape_out) return set_error(lat, WC_ERR_ARG, "lattice and shape_out must not be NULL");
    if (prec != WC_F64 && prec != WC_F32 && prec != WC_F16) return set_error(lat, WC_ERR_ARG, "bad precision");
    if (kind < 0 || kind > 2) return set_error(lat, WC_ERR_ARG, "kind must be 0 (M), 1 (M^+) or 2 (H)");
    if (force_index < -1 || force_index >= apply_shape_count())
        return set_error(lat, WC_ERR_ARG, "force_index out of range");
    if (!apply_shape(lat, prec, kind, force_index, shape_out))
        return set_error(lat, WC_ERR_ARG, "launch shape does not fit this lattice / precision");
    return WC_OK;
}

wc_status wc_checked_violations(unsigned long long *count)
{
    if (!count) return set_error(nullptr, WC_ERR_ARG, "count is NULL");
    *count = 0;
    if (!kChecked) return set_error(nullptr, WC_ERR_STATE, "not a checked build (compile with -DWC_CHECKED)");
    wc_status st = check_cuda(nullptr, cudaDeviceSynchronize(), "sync");
    for (auto read : check_readers()) {
        if (st != WC_OK) break;
        unsigned v = 0;
        st = check_cuda(nullptr, read(&v), "read violation counter");
        *count += v;
    }
    return st;
}

const char *wc_last_error(wc_lattice lat)
{
    if (lat) return lat->err.c_str();
    return g_global_error.c_str();
}

}  // extern "C"
