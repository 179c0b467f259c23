// Allocation-free inner product for callers that cannot allocate device
// memory.
//
// Some callers must not call cudaMalloc: code that runs while another
// framework owns the device memory pool and forbids outside allocations,
// code on a latency-critical path where an allocation would synchronise the
// device, or code that is itself queued from a host callback.  wc_dot needs
// a lattice handle, whose creation allocates its reduction scratch; this
// variant takes plain device pointers and keeps its scratch -- the per-block
// partial sums and the completion ticket of the deterministic two-stage
// reduction -- in one file-scope __device__ array of fixed size, so it
// allocates nothing.  Every GPU that loads the library holds that array
// (32 KiB + 256 B) until the process exits.
#include <cuda.h>
#include <stdint.h>

#include <mutex>

#include "wc_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 16;                     // complex values per thread
constexpr int kNaMaxBlocks = 2048;               // capacity of the scratch array
constexpr long long kNaChunk = (long long)kNaThreads * kNaItems;
constexpr long long kNaMaxN = kNaChunk * kNaMaxBlocks;   // 8,388,608 complex values
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    double partial[kNaMaxBlocks][2];
    unsigned ticket;
};

// Shared by every call on this device; see wc_dot_noalloc in wc.h.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block i reduces the n-element chunk [i*kNaChunk, (i+1)*kNaChunk) with
// coalesced loads; the last block to finish adds the block partials in
// block order and writes out[0] + i out[1].
__global__ void __launch_bounds__(kNaThreads) k_dot_noalloc(const double2 *a, const double2 *b, long long n,
                                                           NoAllocScratch *s, double *out)
{
    __shared__ double sm[kNaThreads / 32][2];
    __shared__ bool last;
    double re = 0.0, im = 0.0;
    const long long base = (long long)blockIdx.x * kNaChunk + threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < kNaItems; ++it) {
        const long long i = base + (long long)it * kNaThreads;
        if (i < n) {
            const double2 x = a[i], y = b[i];
            re += x.x * y.x + x.y * y.y;
            im += x.x * y.y - x.y * y.x;
        }
    }
    re = warp_sum(re);
    im = warp_sum(im);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sm[wid][0] = re;
        sm[wid][1] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0, m = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) {
            r += sm[w][0];
            m += sm[w][1];
        }
        s->partial[blockIdx.x][0] = r;
        s->partial[blockIdx.x][1] = m;
        __threadfence();
        last = atomicAdd(&s->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (wid == 0) {
        double r = 0.0, m = 0.0;
        for (int blk = lane; blk < (int)gridDim.x; blk += 32) {
            r += __ldcg(&s->partial[blk][0]);
            m += __ldcg(&s->partial[blk][1]);
        }
        r = warp_sum(r);
        m = warp_sum(m);
        if (lane == 0) {
            out[0] = r;
            out[1] = m;
            s->ticket = 0u;
        }
    }
}

// cuCtxGetId of the driver, looked up through the runtime (no link against
// libcuda); null when the driver does not offer it
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetIdFn ctx_get_id()
{
    static CtxGetIdFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return static_cast<CtxGetIdFn>(nullptr);
        }
        return reinterpret_cast<CtxGetIdFn>(p);
    }();
    return fn;
}

struct ScratchEntry {
    unsigned long long ctx = 0;   // id of the context the address belongs to
    NoAllocScratch *addr = nullptr;
};

std::mutex g_setup_mutex;
ScratchEntry g_scratch[kMaxDevices];

// Device address of the scratch array for the current device and context.
// The name g_noalloc_scratch is only a host-side stand-in; the address is
// looked up with cudaGetSymbolAddress once per device (with that device
// current) and cached together with the context's id, so that a context
// destroyed and created again (cudaDeviceReset) gets a fresh lookup instead
// of a stale address.  Without cuCtxGetId the lookup is repeated every call
// (cheap once the library's module is loaded).
cudaError_t scratch_address(NoAllocScratch **p)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    CtxGetIdFn get_id = ctx_get_id();
    unsigned long long id = 0;
    bool have_id = get_id && get_id(nullptr, &id) == CUDA_SUCCESS;
    ScratchEntry &ent = g_scratch[dev];
    if (have_id && ent.addr && ent.ctx == id) {
        *p = ent.addr;
        return cudaSuccess;
    }
    void *addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // the lookup made the device's primary context current if it was not yet
    if (!have_id) have_id = get_id && get_id(nullptr, &id) == CUDA_SUCCESS;
    ent.addr = static_cast<NoAllocScratch *>(addr);
    ent.ctx = have_id ? id : 0;
    if (!have_id) ent.addr = nullptr;   // no id to validate a cached address against
    *p = static_cast<NoAllocScratch *>(addr);
    return cudaSuccess;
}

}  // namespace

using namespace wc;

extern "C" wc_status wc_dot_noalloc(const double *a, const double *b, long long n, double *out,
                                    void *cuda_stream)
{
    if (!out) return set_error(nullptr, WC_ERR_ARG, "wc_dot_noalloc: out must not be NULL");
    if (n < 0) return set_error(nullptr, WC_ERR_ARG, "wc_dot_noalloc: n must be >= 0");
    if (n > 0 && (!a || !b)) return set_error(nullptr, WC_ERR_ARG, "wc_dot_noalloc: a and b must not be NULL");
    if (((uintptr_t)a | (uintptr_t)b) & 15u)
        return set_error(nullptr, WC_ERR_ARG, "wc_dot_noalloc: a and b must be 16-byte aligned (complex128 arrays)");
    if ((uintptr_t)out & 7u) return set_error(nullptr, WC_ERR_ARG, "wc_dot_noalloc: out must be 8-byte aligned");
    if (n > kNaMaxN)
        return set_error(nullptr, WC_ERR_ARG,
                         "wc_dot_noalloc: n = " + std::to_string(n) +
                             " complex values exceeds the allocation-free maximum of " + std::to_string(kNaMaxN));
    NoAllocScratch *s = nullptr;
    wc_status st = check_cuda(nullptr, scratch_address(&s), "wc_dot_noalloc: cudaGetSymbolAddress");
    if (st != WC_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // the completion ticket must start at zero
    st = check_cuda(nullptr, cudaMemsetAsync(&s->ticket, 0, sizeof(unsigned), stream), "wc_dot_noalloc: memset");
    if (st != WC_OK) return st;
    const long long blocks = n == 0 ? 1 : (n + kNaChunk - 1) / kNaChunk;
    k_dot_noalloc<<<(unsigned)blocks, kNaThreads, 0, stream>>>(reinterpret_cast<const double2 *>(a),
                                                               reinterpret_cast<const double2 *>(b), n, s, out);
    return check_launch(nullptr, "wc_dot_noalloc");
}
