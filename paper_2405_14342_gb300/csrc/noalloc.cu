// noalloc.cu -- rogs_sort_pairs_noalloc: the stable radix sort of
// (uint32 key, uint32 value) pairs without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// sort: code that only enqueues work into a stream owned by a host framework
// that has reserved all device memory up front, real-time loops that forbid
// allocator calls for latency reasons, or plugin hooks that run while another
// component holds the allocator.  Such callers cannot create a rogs_ctx
// (rogs_create allocates its scratch).  This entry point therefore keeps its
// scratch in a fixed-size array in the library's own device image, which the
// CUDA runtime materialises on every device that loads the library and keeps
// until the process exits.
//
// The host side of this file must not pass the array's name to a kernel: in
// host code that name denotes a host-side shadow, not the device copy.  The
// device address is looked up with cudaGetSymbolAddress on every call, with
// the caller's device current: the lookup is a host-side table read once the
// library's device code is loaded (the first call on a device loads it), and
// no address is kept across calls, so a context that was reset and re-created
// (where the array may sit elsewhere) is never handed a stale address.

#include "kernels.h"

namespace rogs {

constexpr unsigned long long kNoallocMaxPairs = ROGS_NOALLOC_MAX_PAIRS;
// histogram words as the sort lays them out (sized for its smallest keys-per-CTA)
constexpr unsigned long long kNoallocHistWords = radix_hist_words(kNoallocMaxPairs);   // histograms + digit totals
constexpr unsigned long long kNoallocWords = 2ull * kNoallocMaxPairs + kNoallocHistWords;

// alternate keys | alternate values | digit histograms (9.44 MB for 2^20 pairs)
static __device__ __align__(256) uint32_t g_sort_scratch[kNoallocWords];

namespace {
// Device address of g_sort_scratch in the current device's context.
cudaError_t scratch_on_current_device(uint32_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<uint32_t*>(p);
    return cudaSuccess;
}
}  // namespace

}  // namespace rogs

extern "C" rogs_status rogs_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n,
                                               int32_t key_bits, uint32_t* keys_out, uint32_t* vals_out,
                                               rogs_stream stream) {
    using namespace rogs;
    if (n < 0 || key_bits < 0 || key_bits > 32) return ROGS_ERR_INVALID;
    if ((unsigned long long)n > kNoallocMaxPairs) return ROGS_ERR_CAPACITY;
    if (n == 0) return ROGS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return ROGS_ERR_INVALID;
    // an error already pending from some earlier, unrelated call is left for
    // its owner: only an error that appears during this call is reported (and
    // consumed) here
    const bool clean_on_entry = cudaPeekAtLastError() == cudaSuccess;
    uint32_t* base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess) {
        if (clean_on_entry) (void)cudaGetLastError();
        return ROGS_ERR_CUDA;
    }
    // Every histogram word the sort reads is written earlier in the same pass,
    // so nothing in the shared array has to be cleared between calls.
    uint32_t* kalt = base;
    uint32_t* valt = base + kNoallocMaxPairs;
    uint32_t* hist = base + 2 * kNoallocMaxPairs;
    radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, kalt, valt, nullptr, (unsigned long long)n, key_bits, hist,
                     (cudaStream_t)stream, 4096);
    if (clean_on_entry && cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return ROGS_ERR_CUDA;
    }
    return ROGS_OK;
}
