// Checked build (compile every translation unit with -DWC_CHECKED; see
// build.py --checked): the site, neighbour, block-local and shared-memory
// indices the operator, even-odd, RAS and multi-RHS kernels compute are
// tested against the extent of the array they index.  An out-of-range index
// is counted in a device counter of the translation unit and replaced by 0,
// so the access stays inside the array -- the kernel neither faults nor
// traps, its output is simply wrong -- and wc_checked_violations returns the
// count.  The RAS kernels also fill their shared memory with NaN before
// staging it, so that a read of a slot never written shows up as NaN in the
// output.  In the normal build every check compiles to nothing.
#pragma once

#include <cuda_runtime.h>

namespace wc {

// registers a reader of one translation unit's violation counter (checked
// build; called from static initialisers)
void register_check_counter(cudaError_t (*read)(unsigned *));

}  // namespace wc

#ifdef WC_CHECKED

static __device__ unsigned wc_bad_index_count;

namespace {

cudaError_t wc_read_bad_index_count(unsigned *out)
{
    return cudaMemcpyFromSymbol(out, wc_bad_index_count, sizeof(unsigned));
}

struct WcCheckRegistration {
    WcCheckRegistration() { wc::register_check_counter(&wc_read_bad_index_count); }
};
const WcCheckRegistration wc_check_registration;

}  // namespace

namespace wc {
constexpr bool kChecked = true;

// i when 0 <= i < n; otherwise counts a violation and returns 0
__device__ __forceinline__ int wc_idx(int i, int n)
{
    if ((unsigned)i >= (unsigned)n) {
        atomicAdd(&wc_bad_index_count, 1u);
        return 0;
    }
    return i;
}
}  // namespace wc

#else

namespace wc {
constexpr bool kChecked = false;
__device__ __forceinline__ int wc_idx(int i, int) { return i; }
}  // namespace wc

#endif
