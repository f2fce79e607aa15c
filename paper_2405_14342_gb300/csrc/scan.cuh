// scan.cuh -- device-wide exclusive prefix sum with a device-resident length.
//
// Three launches with fixed grids (sized by a host-known capacity), so the
// whole sequence can be captured in a CUDA graph although the real length
// is only known on the device:
//   1. scan_reduce_k   : per 4096-element tile, sum of f(i)
//   2. scan_tiles_k    : one block, exclusive scan of the tile sums; writes the
//                        total (and, when asked, the total clamped to a
//                        capacity with an overflow bit, so that no separate
//                        kernel has to finish the count)
//   3. scan_down_k     : per tile, block-wide exclusive scan plus the tile offset
// f(i) is a functor giving the value of element i (no input array needs to
// be materialised).  No kernel waits on another block.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rogs {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x == kScanThreads);
// sh must hold 33 T.  Every thread receives the block total.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* sh, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = sh[lane];
        T wi = warp_incl_scan(w);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    T r = sh[warp] + inc - v;
    total = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned long long scan_len(const unsigned long long* n_ptr, unsigned long long cap) {
    if (!n_ptr) return cap;
    unsigned long long n = *n_ptr;
    return n < cap ? n : cap;
}

template <class F, class T>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_k(F f, const unsigned long long* n_ptr,
                                                               unsigned long long cap, T* tile_sums) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ T sh[33];
    const unsigned long long n = scan_len(n_ptr, cap);
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile;
    T s = 0;
    if (base < n) {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            unsigned long long i = base + (unsigned long long)threadIdx.x * kScanItems + k;
            if (i < n) s += (T)f(i);
        }
    }
    T tot;
    block_excl_scan<T>(s, sh, tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Where the one-block pass leaves the scan's total: the total itself and,
// optionally, min(total, cap), with overflow_bit set in *status when the
// total exceeds cap.  Null pointers are skipped.
struct ScanTotal {
    unsigned long long* total;
    unsigned long long* clamped;
    unsigned long long cap;
    unsigned int* status;
    unsigned int overflow_bit;
};

// One block: exclusive scan of n_tiles tile sums in place; the sum as `out` asks.
template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_tiles_k(T* tile_sums, int n_tiles, ScanTotal out) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ T sh[33];
    T carry = 0;
    for (int base = 0; base < n_tiles; base += kScanThreads) {
        int i = base + threadIdx.x;
        T v = i < n_tiles ? tile_sums[i] : T(0);
        T tot;
        T ex = block_excl_scan<T>(v, sh, tot);
        if (i < n_tiles) tile_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        const unsigned long long t = (unsigned long long)carry;
        if (out.total) *out.total = t;
        if (out.clamped) *out.clamped = t < out.cap ? t : out.cap;
        if (out.status && t > out.cap) *out.status |= out.overflow_bit;
    }
}

template <class F, class T>
__global__ void __launch_bounds__(kScanThreads) scan_down_k(F f, const unsigned long long* n_ptr,
                                                             unsigned long long cap, const T* tile_offs, T* out) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ T sh[33];
    const unsigned long long n = scan_len(n_ptr, cap);
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile;
    if (base >= n) return;  // uniform per block
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        unsigned long long i = base + (unsigned long long)threadIdx.x * kScanItems + k;
        v[k] = (i < n) ? (T)f(i) : T(0);
        s += v[k];
    }
    T tot;
    T ex = block_excl_scan<T>(s, sh, tot) + tile_offs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        unsigned long long i = base + (unsigned long long)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
}

inline int scan_tiles_for(unsigned long long cap) {
    int nt = (int)((cap + kScanTile - 1) / kScanTile);
    return nt > 0 ? nt : 1;
}

// Launch the three-stage scan.  tile_sums must hold scan_tiles_for(cap) T.
template <class F, class T>
inline void device_exclusive_scan(F f, const unsigned long long* n_ptr, unsigned long long cap, T* tile_sums,
                                  T* out, ScanTotal total, cudaStream_t s) {
    int nt = scan_tiles_for(cap);
    launch_pdl(scan_reduce_k<F, T>, dim3(nt), dim3(kScanThreads), 0, s, f, n_ptr, cap, tile_sums);
    launch_pdl(scan_tiles_k<T>, dim3(1), dim3(kScanThreads), 0, s, tile_sums, nt, total);
    launch_pdl(scan_down_k<F, T>, dim3(nt), dim3(kScanThreads), 0, s, f, n_ptr, cap, tile_sums, out);
    note_launches(3);
}

}  // namespace rogs
