// sort.cu -- hand-written stable LSD radix sort of (uint32 key, uint32 value)
// pairs with a device-resident length (8-bit digits, 1024-8192 keys per CTA).
//
// Keys per CTA (the sort "chunk") is 1024, 2048, 4096 or 8192 (4/8/16/32
// keys per thread), chosen by the caller: the context configuration for the
// pair sort, 1024 for the depth sort of the records.  Per pass, three launches
// with fixed grids:
//   rs_upsweep_k   per-tile digit histograms, digit-major [256][tiles]
//   rs_rowscan_k   one block per digit: exclusive scan across tiles + digit total
//   rs_downsweep_k stable scatter: the rank of a key inside its tile is built
//                  warp by warp in key order (one ballot per digit bit
//                  groups equal digits, lanes below a lane come first), then warps in
//                  order, so equal keys keep their input order.
// No block waits on another block.  Used for the depth sort of visible
// records and the tile sort of (tile, record) pairs (RoGs Sec. 3.3.1: sort by
// ascending original depth; ties by surfel index come from stability).
#include "kernels.h"
#include "scan.cuh"

namespace rogs {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ unsigned long long rs_len(const unsigned long long* n_ptr, unsigned long long cap) {
    return scan_len(n_ptr, cap);
}

template <int IPT>
__global__ void __launch_bounds__(kRsThreads) rs_upsweep_k(const uint32_t* __restrict__ keys,
                                                            const unsigned long long* n_ptr, unsigned long long cap,
                                                            int shift, uint32_t mask, uint32_t* __restrict__ hist) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    constexpr int kRsWarpItems = 32 * IPT;
    constexpr int kRsTile = kRsThreads * IPT;
    __shared__ uint32_t sh[kRsWarps][256];
    const unsigned long long n = rs_len(n_ptr, cap);
    const unsigned ntiles = (unsigned)((n + kRsTile - 1) / kRsTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) sh[w][threadIdx.x] = 0;
        __syncthreads();
        const unsigned long long base = (unsigned long long)tile * kRsTile + (unsigned long long)warp * kRsWarpItems;
        uint32_t key[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {   // every load in flight before the first count
            unsigned long long i = base + k * 32 + lane;
            key[k] = i < n ? keys[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k)
            if (base + k * 32 + lane < n) atomicAdd(&sh[warp][(key[k] >> shift) & mask], 1u);
        __syncthreads();
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) s += sh[w][threadIdx.x];
        hist[(unsigned long long)threadIdx.x * ntiles + tile] = s;
        __syncthreads();
    }
}

// One block per digit: exclusive scan of hist[d][0..ntiles) in place.
__global__ void __launch_bounds__(kScanThreads) rs_rowscan_k(uint32_t* __restrict__ hist,
                                                              const unsigned long long* n_ptr, unsigned long long cap,
                                                              int tile_keys, uint32_t* __restrict__ row_total) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ uint32_t sh[33];
    const unsigned long long n = rs_len(n_ptr, cap);
    const unsigned ntiles = (unsigned)((n + tile_keys - 1) / tile_keys);
    uint32_t* row = hist + (unsigned long long)blockIdx.x * ntiles;
    uint32_t carry = 0;
    for (unsigned base = 0; base < ntiles; base += kScanThreads) {
        unsigned i = base + threadIdx.x;
        uint32_t v = i < ntiles ? row[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan<uint32_t>(v, sh, tot);
        if (i < ntiles) row[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) row_total[blockIdx.x] = carry;
}

// Dynamic shared memory of rs_downsweep_k: the tile's keys and values in digit order.
__host__ __device__ constexpr size_t rs_stage_bytes(int ipt) { return (size_t)2 * 4 * kRsThreads * ipt; }

template <int IPT>
__global__ void __launch_bounds__(kRsThreads) rs_downsweep_k(const uint32_t* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin,
                                                              uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                              const unsigned long long* n_ptr, unsigned long long cap,
                                                              int shift, uint32_t mask, const uint32_t* __restrict__ hist,
                                                              const uint32_t* __restrict__ row_total) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    constexpr int kRsWarpItems = 32 * IPT;
    constexpr int kRsTile = kRsThreads * IPT;
    extern __shared__ uint32_t rs_stage[];   // [kRsTile] keys, then [kRsTile] values
    __shared__ uint32_t digit_base[256];
    __shared__ uint32_t wh[kRsWarps][256];   // per-warp digit counts, then per-warp tile-local starts
    __shared__ uint32_t tile_start[256];     // tile-local start of each digit
    __shared__ uint32_t out_base[256];       // global position of each digit's first key of the tile
    __shared__ uint32_t scan_w[kRsWarps + 1];
    uint32_t* sk = rs_stage;
    uint32_t* sv = rs_stage + kRsTile;
    const unsigned long long n = rs_len(n_ptr, cap);
    const unsigned ntiles = (unsigned)((n + kRsTile - 1) / kRsTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d0 = threadIdx.x;
    const unsigned lt = lanemask_lt();

    // block-wide exclusive scan of one value per thread (256 threads)
    auto block_scan = [&](uint32_t v) -> uint32_t {
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) scan_w[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t c = 0;
            for (int w = 0; w < kRsWarps; ++w) { uint32_t t = scan_w[w]; scan_w[w] = c; c += t; }
        }
        __syncthreads();
        const uint32_t r = scan_w[warp] + inc - v;
        __syncthreads();
        return r;
    };
    // exclusive scan of the 256 digit totals
    digit_base[d0] = block_scan(row_total[d0]);

    for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) wh[w][threadIdx.x] = 0;
        __syncthreads();
        const unsigned long long base = (unsigned long long)tile * kRsTile + (unsigned long long)warp * kRsWarpItems;
        const unsigned long long left = n - (unsigned long long)tile * kRsTile;
        const int tile_n = (int)(left < (unsigned long long)kRsTile ? left : (unsigned long long)kRsTile);
        uint32_t key[IPT], val[IPT], rank[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {   // every load in flight before the first rank
            unsigned long long i = base + k * 32 + lane;
            key[k] = i < n ? kin[i] : 0u;
            val[k] = i < n ? vin[i] : 0u;
        }
        // rank in key order: warp by warp, and inside a warp item row by item row,
        // lanes below a lane first, so equal digits keep their input order
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const bool valid = base + k * 32 + lane < n;
            const unsigned vm = __ballot_sync(kFull, valid);
            const uint32_t d = (key[k] >> shift) & mask;
            const unsigned peers = warp_digit_peers(d, mask, vm);
            rank[k] = 0;
            if (valid) rank[k] = wh[warp][d] + __popc(peers & lt);
            __syncwarp();
            if (valid && (peers & lt) == 0) wh[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            uint32_t cnt = 0;
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) {   // per-warp counts -> starts inside the digit's run
                const uint32_t c = wh[w][d0];
                wh[w][d0] = cnt;
                cnt += c;
            }
            const uint32_t ts = block_scan(cnt);
            tile_start[d0] = ts;
            out_base[d0] = digit_base[d0] + hist[(unsigned long long)d0 * ntiles + tile];
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) wh[w][d0] += ts;
        }
        __syncthreads();
        // keys into shared memory in digit order, then out in runs of equal digits
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            if (base + k * 32 + lane < n) {
                const uint32_t d = (key[k] >> shift) & mask;
                const uint32_t lp = wh[warp][d] + rank[k];
                sk[lp] = key[k];
                sv[lp] = val[k];
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < tile_n; j += kRsThreads) {
            const uint32_t kk = sk[j];
            const uint32_t d = (kk >> shift) & mask;
            const uint32_t pos = out_base[d] + (uint32_t)j - tile_start[d];
            if (rogs_ok(pos < n, 301u)) {
                kout[pos] = kk;
                vout[pos] = sv[j];
            }
        }
        __syncthreads();
    }
}

__global__ void copy_pairs_k(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                             const unsigned long long* n_ptr, unsigned long long cap) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    const unsigned long long n = rs_len(n_ptr, cap);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        kout[i] = kin[i];
        vout[i] = vin[i];
    }
}

void prepare_sort() {
    cudaFuncSetAttribute(rs_downsweep_k<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_stage_bytes(4));
    cudaFuncSetAttribute(rs_downsweep_k<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_stage_bytes(8));
    cudaFuncSetAttribute(rs_downsweep_k<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_stage_bytes(16));
    cudaFuncSetAttribute(rs_downsweep_k<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_stage_bytes(32));
}

template <int IPT>
static void radix_passes(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t* kalt,
                         uint32_t* valt, const unsigned long long* n_ptr, unsigned long long cap, int key_bits,
                         uint32_t* hist, uint32_t* row_total, cudaStream_t s) {
    constexpr int tile_keys = kRsThreads * IPT;
    const int passes = (key_bits + 7) / 8;
    unsigned long long tiles = (cap + tile_keys - 1) / tile_keys;
    const int grid = (int)(tiles < 1 ? 1 : (tiles > 2048 ? 2048 : tiles));
    const uint32_t* sk = kin;
    const uint32_t* sv = vin;
    for (int p = 0; p < passes; ++p) {
        // the last pass must land in (kout, vout)
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t* dk = to_out ? kout : kalt;
        uint32_t* dv = to_out ? vout : valt;
        const int shift = 8 * p;
        const int bits = key_bits - shift < 8 ? key_bits - shift : 8;
        const uint32_t mask = (bits >= 32) ? 0xffffffffu : ((1u << bits) - 1u);
        launch_pdl(rs_upsweep_k<IPT>, dim3(grid), dim3(kRsThreads), 0, s, sk, n_ptr, cap, shift, mask, hist);
        launch_pdl(rs_rowscan_k, dim3(256), dim3(kScanThreads), 0, s, hist, n_ptr, cap, tile_keys, row_total);
        launch_pdl(rs_downsweep_k<IPT>, dim3(grid), dim3(kRsThreads), rs_stage_bytes(IPT), s, sk, sv, dk, dv, n_ptr, cap,
                   shift, mask, hist, row_total);
        note_launches(3);
        sk = dk;
        sv = dv;
    }
}

void radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t* kalt,
                      uint32_t* valt, const unsigned long long* n_ptr, unsigned long long cap, int key_bits,
                      uint32_t* hist, cudaStream_t s, int sort_tile) {
    uint32_t* row_total = hist + (radix_hist_words(cap) - 256);
    if ((key_bits + 7) / 8 == 0) {
        unsigned long long blocks = (cap + 255) / 256;
        const int grid = (int)(blocks < 1 ? 1 : (blocks > 2048 ? 2048 : blocks));
        launch_pdl(copy_pairs_k, dim3(grid), dim3(256), 0, s, kin, vin, kout, vout, n_ptr, cap);
        note_launches(1);
        return;
    }
    if (sort_tile == 1024)
        radix_passes<4>(kin, vin, kout, vout, kalt, valt, n_ptr, cap, key_bits, hist, row_total, s);
    else if (sort_tile == 2048)
        radix_passes<8>(kin, vin, kout, vout, kalt, valt, n_ptr, cap, key_bits, hist, row_total, s);
    else if (sort_tile == 8192)
        radix_passes<32>(kin, vin, kout, vout, kalt, valt, n_ptr, cap, key_bits, hist, row_total, s);
    else
        radix_passes<16>(kin, vin, kout, vout, kalt, valt, n_ptr, cap, key_bits, hist, row_total, s);
}

#ifdef ROGS_CHECKED
unsigned check_word_sort() { return rogs_check_word_take(); }
#endif

}  // namespace rogs
