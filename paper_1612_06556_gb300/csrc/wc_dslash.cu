// Wilson-Clover operator kernels: out = M in, M^+ in, H in; field casts.
//
// One thread per site.  Sites map to threads either in lexicographic order
// or by 4-D tiles (a CTA covers a tx*ty*tz*tt brick, x fastest, so a warp's
// loads stay 128-byte contiguous and the x/y/z neighbours of most sites lie
// in the same CTA); the 8-fold reuse of each input spinor is served by
// L1/L2.  The mapping, CTA size and register cap are picked per lattice
// extent, precision and operator by a small autotuner (first use, timed with
// CUDA events; not while the stream is being captured).  Per direction the neighbour spinor is spin
// projected to a two-spinor before the SU(3) multiply, halving the matvec
// work (paper Sec. 2/3, the hopping multiplication "MULT"); links are read as
// two rows and the third rebuilt in registers (SU(3) reconstruction).  The
// clover term (two packed Hermitian 6x6 blocks) is applied to the centre
// spinor first and the hops are accumulated into that result with the
// coefficient -kappa, so out = (1 + T) in - kappa H in is written once.
//
#include <array>
#include <map>
#include <mutex>
#include <type_traits>

#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

constexpr int kApplyMaxThreads = 256;

// Site of (block, thread) under a launch shape: tile[] = {0,0,0,0} means
// lexicographic order, else tile extents (x fastest) tiling the lattice.
struct TileMap {
    int tile[4];
    int ntile[3];   // tiles along x, y, z
};

__device__ __forceinline__ int site_of_thread(const Geom &g, const TileMap &m, int blk, bool &valid)
{
    if (m.tile[0] == 0) {
        const int x = blk * blockDim.x + threadIdx.x;
        valid = x < g.V;
        return x;
    }
    int t = threadIdx.x, b = blk;
    const int cx = (b % m.ntile[0]) * m.tile[0] + t % m.tile[0];
    t /= m.tile[0];
    b /= m.ntile[0];
    const int cy = (b % m.ntile[1]) * m.tile[1] + t % m.tile[1];
    t /= m.tile[1];
    b /= m.ntile[1];
    const int cz = (b % m.ntile[2]) * m.tile[2] + t % m.tile[2];
    t /= m.tile[2];
    b /= m.ntile[2];
    const int ct = b * m.tile[3] + t;
    valid = true;
    return cx + g.stride[1] * cy + g.stride[2] * cz + g.stride[3] * ct;
}

template <class P, int KIND>
__device__ __forceinline__ void apply_site(const Geom &g, const TileMap &tm, int blk, const GaugeStore &U,
                                           const CloverStore &C, const void *in, const float *in_nrm, void *out,
                                           float *out_nrm, double kappa)
{
    bool valid;
    const int x = site_of_thread(g, tm, blk, valid);
    if (valid) apply_site_at<P, KIND>(g, x, U, C, in, in_nrm, out, out_nrm, kappa);
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream serialization attribute may start while the previous kernel of the
// stream drains; griddepcontrol.wait then blocks until that kernel has
// completed and its writes are visible.  launch_dependents lets the next
// such kernel start once every CTA of this grid is running.  Both are no-ops
// for kernels launched without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// Bulk L2 prefetch of n bytes at p (both 16-byte multiples); only a cache
// hint: L2 is the point of coherence, so data still being written by the
// previous kernel is read correctly by the loads after griddep_wait().
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned n)
{
    if (n >= 16 && (reinterpret_cast<uintptr_t>(p) & 15) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(n & ~15u) : "memory");
}

// The links and clover term of sites [x0, x0 + n) (lexicographic block),
// one contiguous range per component plane; plane i is issued by thread i.
template <class P>
__device__ __forceinline__ void prefetch_block(const Geom &g, const GaugeStore &U, const CloverStore &C, int x0,
                                               int n, int i)
{
    const size_t V = g.V;
    if (std::is_same<P, P32>::value) {
        if (i < 12) prefetch_l2(U.u32 + i * V + x0, 16u * n);                   // [4][3][V] float4
        else if (i < 30) prefetch_l2(C.c32 + (i - 12) * V + x0, 16u * n);      // [18][V] float4
    } else if (std::is_same<P, P16>::value) {
        if (i < 4) prefetch_l2(U.u16a + i * V + x0, 16u * n);                   // [4][V] uint4
        else if (i < 8) prefetch_l2(U.u16b + (i - 4) * V + x0, 8u * n);        // [4][V] uint2
        else if (i < 17) prefetch_l2(C.c16 + (i - 8) * V + x0, 16u * n);       // [9][V] uint4
    }
}

// KIND 0: out = M in, 1: out = M^+ in, 2: out = H in.  MINB: minimum
// resident CTAs of kApplyMaxThreads threads per SM (caps registers).  The
// grid may be smaller than the nlogical logical blocks (persistent launch:
// each CTA walks the logical blocks with stride gridDim.x).  kFlagPdl: the launch is a programmatic
// dependent of the previous kernel (lexicographic site maps only): the CTA
// warms L2 with the links and clover of its first sites, which no kernel of
// a solve writes, before it waits for the previous kernel's output.
constexpr int kFlagPdl = 1;

template <class P, int KIND, int MINB>
__global__ void __launch_bounds__(kApplyMaxThreads, MINB)
    k_apply(Geom g, TileMap tm, int nlogical, GaugeStore U, CloverStore C, const void *in, const float *in_nrm,
            void *out, float *out_nrm, double kappa, int flags)
{
    if (flags & kFlagPdl) {
        const int x0 = blockIdx.x * blockDim.x;
        const int n = g.V - x0 < (int)blockDim.x ? g.V - x0 : (int)blockDim.x;
        if (n > 0) prefetch_block<P>(g, U, C, x0, n, threadIdx.x);
        griddep_wait();
    }
    griddep_launch_dependents();
    for (int blk = blockIdx.x; blk < nlogical; blk += gridDim.x)
        apply_site<P, KIND>(g, tm, blk, U, C, in, in_nrm, out, out_nrm, kappa);
}

// ---- launch shapes and their autotuner ---------------------------------

struct ApplyShape {
    int threads;
    int tile[4];     // {0,0,0,0}: lexicographic
    int capped;      // register cap: 0 none, 1: 64 per thread (4 CTAs of 256), 2: 85 (3 CTAs of 256)
    int persistent;  // 1: grid = resident CTAs, each walks logical blocks
    int pdl;         // 1: programmatic dependent launch (lexicographic only; not inside a capture)
};

constexpr ApplyShape kShapes[] = {
    {128, {0, 0, 0, 0}, 0, 0}, {128, {0, 0, 0, 0}, 1, 0}, {256, {0, 0, 0, 0}, 0, 0}, {256, {0, 0, 0, 0}, 1, 0},
    {128, {8, 4, 4, 1}, 0, 0}, {128, {8, 4, 4, 1}, 1, 0}, {128, {8, 4, 2, 2}, 0, 0}, {128, {4, 4, 4, 2}, 0, 0},
    {256, {8, 4, 4, 2}, 0, 0}, {256, {8, 4, 4, 2}, 1, 0}, {256, {8, 8, 4, 1}, 0, 0}, {128, {0, 0, 0, 0}, 2, 0},
    {256, {0, 0, 0, 0}, 2, 0}, {128, {8, 4, 4, 1}, 2, 0}, {256, {8, 4, 4, 2}, 2, 0}, {128, {8, 4, 2, 2}, 2, 0},
    {128, {0, 0, 0, 0}, 2, 1}, {256, {0, 0, 0, 0}, 2, 1}, {128, {0, 0, 0, 0}, 0, 1}, {256, {0, 0, 0, 0}, 0, 1},
    {128, {0, 0, 0, 0}, 2, 1, 1}, {256, {0, 0, 0, 0}, 2, 1, 1},
    // small lattices: CTAs of 32 or 64 sites spread a few thousand sites
    // over more SMs (the FP64 operator is bound by the FP64 pipe of the SMs
    // it runs on)
    {32, {0, 0, 0, 0}, 0, 0}, {64, {0, 0, 0, 0}, 0, 0},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// caps: bit c-1 set if register cap c is compiled for the operator (P::kCaps)
bool shape_fits(const Geom &g, const ApplyShape &s, int caps)
{
    if (s.capped && !((caps >> (s.capped - 1)) & 1)) return false;
    if (s.tile[0] == 0) return true;
    for (int m = 0; m < 4; ++m)
        if (g.L[m] % s.tile[m] != 0) return false;
    return s.tile[0] * s.tile[1] * s.tile[2] * s.tile[3] == s.threads;
}

// Resident CTAs per SM of one kernel instantiation (cached per function).
template <class K>
int resident_ctas(K kernel, int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <class P>
cudaError_t launch_shape(wc_lattice lat, wc_field out, wc_field in, int kind, const ApplyShape &sh,
                         cudaStream_t stream)
{
    const Geom &g = lat->g;
    TileMap tm{};
    int nlogical;
    if (sh.tile[0] == 0) {
        nlogical = (g.V + sh.threads - 1) / sh.threads;
    } else {
        for (int m = 0; m < 4; ++m) tm.tile[m] = sh.tile[m];
        for (int m = 0; m < 3; ++m) tm.ntile[m] = g.L[m] / sh.tile[m];
        nlogical = g.V / sh.threads;
    }
    int pdl = 0;
    if (sh.pdl && sh.tile[0] == 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(stream, &cs);
        pdl = cs == cudaStreamCaptureStatusNone;
    }
#define WC_LAUNCH(K, MB)                                                                                      \
    do {                                                                                                      \
        auto kern = k_apply<P, K, MB>;                                                                        \
        int grid = nlogical;                                                                                  \
        if (sh.persistent) {                                                                                  \
            const int cap = resident_ctas(kern, sh.threads) * sm_count();                                   \
            grid = nlogical < cap ? nlogical : cap;                                                           \
        }                                                                                                     \
        if (pdl) {                                                                                            \
            cudaLaunchConfig_t cfg = {};                                                                      \
            cudaLaunchAttribute attr[1];                                                                      \
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                                  \
            attr[0].val.programmaticStreamSerializationAllowed = 1;                                           \
            cfg.gridDim = dim3(grid);                                                                         \
            cfg.blockDim = dim3(sh.threads);                                                                  \
            cfg.stream = stream;                                                                              \
            cfg.attrs = attr;                                                                                 \
            cfg.numAttrs = 1;                                                                                 \
            return cudaLaunchKernelEx(&cfg, kern, g, tm, nlogical, lat->gauge, lat->clover, in->data,         \
                                      (const float *)in->nrm, out->data, out->nrm, lat->kappa, kFlagPdl);    \
        }                                                                                                     \
        kern<<<grid, sh.threads, 0, stream>>>(g, tm, nlogical, lat->gauge, lat->clover, in->data, in->nrm,    \
                                              out->data, out->nrm, lat->kappa, 0);                            \
    } while (0)
    // minimum resident CTAs of 256 threads for caps 1 and 2 (1: not compiled)
    constexpr bool c1 = P::kCaps & 1, c2 = P::kCaps & 2;
    constexpr int MB1 = c1 ? P::kCap1MinBlocks : 1, MB2 = c2 ? 3 : 1;
    if (kind == 0) {
        if (c1 && sh.capped == 1) WC_LAUNCH(0, MB1);
        else if (c2 && sh.capped == 2) WC_LAUNCH(0, MB2);
        else WC_LAUNCH(0, 1);
    } else if (kind == 1) {
        if (c1 && sh.capped == 1) WC_LAUNCH(1, MB1);
        else if (c2 && sh.capped == 2) WC_LAUNCH(1, MB2);
        else WC_LAUNCH(1, 1);
    } else {
        if (c1 && sh.capped == 1) WC_LAUNCH(2, MB1);
        else if (c2 && sh.capped == 2) WC_LAUNCH(2, MB2);
        else WC_LAUNCH(2, 1);
    }
#undef WC_LAUNCH
    return cudaGetLastError();
}

std::mutex g_shape_mutex;
std::map<std::array<int, 6>, int> g_shape_choice;   // (L, prec, kind) -> shape index

// Time every fitting shape (three rounds of 16 launches after one warm-up,
// best round kept, candidates interleaved so that clock drift affects all
// alike) and keep the fastest.  Needs an uncaptured stream; out is
// overwritten by the real launch that follows.
template <class P>
int tune_shape(wc_lattice lat, wc_field out, wc_field in, int kind, cudaStream_t stream)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    // the candidates are timed on four input / output pairs in turn (the
    // caller's and three copies of its input), so that on lattices whose
    // fields outgrow L2 every launch streams its spinors from HBM as the
    // solvers' applies do; without memory for the copies, on the caller's
    // pair alone
    const size_t bytes = spinor_bytes(in->prec, lat->g.V);
    wc_field ins[4] = {in, nullptr, nullptr, nullptr}, outs[4] = {out, nullptr, nullptr, nullptr};
    int npair = 1;
    for (int k = 1; k < 4; ++k) {
        if (wc_field_create(lat, in->prec, &ins[k]) != WC_OK) break;
        if (wc_field_create(lat, in->prec, &outs[k]) != WC_OK) {
            wc_field_destroy(ins[k]);
            ins[k] = nullptr;
            break;
        }
        cudaMemcpyAsync(ins[k]->data, in->data, bytes, cudaMemcpyDeviceToDevice, stream);
        if (in->nrm) cudaMemcpyAsync(ins[k]->nrm, in->nrm, sizeof(float) * lat->g.V, cudaMemcpyDeviceToDevice, stream);
        npair = k + 1;
    }
    cudaGetLastError();
    float best_ms[kNumShapes];
    for (int i = 0; i < kNumShapes; ++i) best_ms[i] = 1e30f;
    for (int round = 0; round < 3; ++round) {
        for (int i = 0; i < kNumShapes; ++i) {
            if (!shape_fits(lat->g, kShapes[i], P::kCaps)) continue;
            if (launch_shape<P>(lat, out, in, kind, kShapes[i], stream) != cudaSuccess) continue;
            cudaEventRecord(e0, stream);
            for (int r = 0; r < 16; ++r)
                launch_shape<P>(lat, outs[r % npair], ins[r % npair], kind, kShapes[i], stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms[i]) best_ms[i] = ms;
        }
    }
    int best = 0;
    for (int i = 1; i < kNumShapes; ++i)
        if (best_ms[i] < best_ms[best]) best = i;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int k = 1; k < npair; ++k) {
        wc_field_destroy(ins[k]);
        wc_field_destroy(outs[k]);
    }
    cudaGetLastError();
    return best;
}

template <class P>
cudaError_t launch_apply_p(wc_lattice lat, wc_field out, wc_field in, int kind, cudaStream_t stream)
{
    // the double-FP32 operator has its own entry (precision code 3)
    const int pcode = std::is_same<P, PDF>::value ? 3 : (int)in->prec;
    const std::array<int, 6> key = {lat->g.L[0], lat->g.L[1], lat->g.L[2], lat->g.L[3], pcode, kind};
    int choice = -1;
    {
        std::lock_guard<std::mutex> lk(g_shape_mutex);
        auto it = g_shape_choice.find(key);
        if (it != g_shape_choice.end()) choice = it->second;
    }
    if (choice < 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(stream, &cs);
        if (cs != cudaStreamCaptureStatusNone) {
            choice = 0;   // no timing inside a capture: default shape, not cached
        } else {
            choice = tune_shape<P>(lat, out, in, kind, stream);
            std::lock_guard<std::mutex> lk(g_shape_mutex);
            g_shape_choice[key] = choice;
        }
    }
    return launch_shape<P>(lat, out, in, kind, kShapes[choice], stream);
}

// ------------------------------------------------------------------------
// precision conversion / scaling: dst = scale * src
// ------------------------------------------------------------------------

template <class PS, class PD>
__global__ void k_copy(int V, const void *src, const float *src_nrm, void *dst, float *dst_nrm, double scale,
                       const double *dev_norm2, int invert)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    double sc = scale;
    if (dev_norm2) {
        const double n2 = *dev_norm2;
        const double n = sqrt(n2);
        sc *= invert ? (n > 0.0 ? 1.0 / n : 0.0) : n;
    }
    cx<typename PS::real> a[12];
    PS::load_spinor(src, src_nrm, V, x, a);
    cx<typename PD::real> b[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        // scale in the wider of the two precisions, then round once
        const double re = sc * (double)a[k].re, im = sc * (double)a[k].im;
        b[k] = mkc((typename PD::real)re, (typename PD::real)im);
    }
    PD::store_spinor(dst, dst_nrm, V, x, b);
}

template <class PS>
cudaError_t launch_copy_s(wc_lattice lat, wc_field dst, wc_field src, double scale, const double *dn, int inv,
                          cudaStream_t stream)
{
    const int V = lat->g.V;
    dim3 grid((V + 255) / 256), block(256);
    switch (dst->prec) {
    case WC_F64:
        k_copy<PS, P64><<<grid, block, 0, stream>>>(V, src->data, src->nrm, dst->data, dst->nrm, scale, dn, inv);
        break;
    case WC_F32:
        k_copy<PS, P32><<<grid, block, 0, stream>>>(V, src->data, src->nrm, dst->data, dst->nrm, scale, dn, inv);
        break;
    default:
        k_copy<PS, P16><<<grid, block, 0, stream>>>(V, src->data, src->nrm, dst->data, dst->nrm, scale, dn, inv);
    }
    return cudaGetLastError();
}

}  // namespace

// Query or pin the launch shape of (lat extent, prec, kind): force >= 0 pins
// shape #force (false if it does not fit); out = {threads, tile[4], capped},
// all -1 when no shape was chosen yet.
bool apply_shape(wc_lattice lat, wc_prec prec, int kind, int force, int out[6])
{
    // FP64 fields on a lattice in double-FP32 mode use that operator's entry
    const int pcode = (prec == WC_F64 && lat->fp64_arith == WC_ARITH_DF32) ? 3 : (int)prec;
    const std::array<int, 6> key = {lat->g.L[0], lat->g.L[1], lat->g.L[2], lat->g.L[3], pcode, kind};
    for (int i = 0; i < 6; ++i) out[i] = -1;
    std::lock_guard<std::mutex> lk(g_shape_mutex);
    if (force >= 0) {
        const int caps = prec != WC_F64 ? P32::kCaps : pcode == 3 ? PDF::kCaps : P64::kCaps;
        if (force >= kNumShapes || !shape_fits(lat->g, kShapes[force], caps)) return false;
        g_shape_choice[key] = force;
    }
    auto it = g_shape_choice.find(key);
    if (it == g_shape_choice.end()) return true;
    const ApplyShape &s = kShapes[it->second];
    out[0] = s.threads;
    for (int m = 0; m < 4; ++m) out[1 + m] = s.tile[m];
    out[5] = s.capped + 4 * s.persistent + 16 * s.pdl;
    return true;
}

int apply_shape_count() { return kNumShapes; }

cudaError_t launch_apply(wc_lattice lat, wc_field out, wc_field in, int kind, cudaStream_t stream)
{
    if (lat->schur_parent) return launch_schur(lat, out, in, kind == 1, stream);   // half lattice: M^
    switch (in->prec) {
    case WC_F64:
        return lat->fp64_arith == WC_ARITH_DF32 ? launch_apply_p<PDF>(lat, out, in, kind, stream)
                                                : launch_apply_p<P64>(lat, out, in, kind, stream);
    case WC_F32: return launch_apply_p<P32>(lat, out, in, kind, stream);
    default: return launch_apply_p<P16>(lat, out, in, kind, stream);
    }
}

cudaError_t launch_copy(wc_lattice lat, wc_field dst, wc_field src, double scale, const double *dev_scale,
                        int invert_scale, cudaStream_t stream)
{
    switch (src->prec) {
    case WC_F64: return launch_copy_s<P64>(lat, dst, src, scale, dev_scale, invert_scale, stream);
    case WC_F32: return launch_copy_s<P32>(lat, dst, src, scale, dev_scale, invert_scale, stream);
    default: return launch_copy_s<P16>(lat, dst, src, scale, dev_scale, invert_scale, stream);
    }
}

}  // namespace wc
