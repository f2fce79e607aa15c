// bin.cu -- stage 2: tile binning of the depth-sorted records.
//
// RoGs Sec. 3.3.1 composites, at each pixel, the surfels covering it in
// ascending order of original depth.  After the depth sort of the records
// (stable, so equal depths keep (view, surfel) order), every record emits one
// (global tile id, record id) pair per tile of its conservative footprint
// rectangle, in depth order.  A stable radix sort on the tile id then leaves
// each tile's list ordered by (depth, surfel index), and tile_ranges_k finds
// each tile's [start, end).
#include "kernels.h"
#include "scan.cuh"

namespace rogs {

__device__ __forceinline__ unsigned long long rect_tiles(uint2 r) {
    const int x0 = (int)(r.x & 0xffffu), y0 = (int)(r.x >> 16);
    const int x1 = (int)(r.y & 0xffffu), y1 = (int)(r.y >> 16);
    if (x1 < x0 || y1 < y0) return 0ull;
    return (unsigned long long)(x1 - x0 + 1) * (unsigned long long)(y1 - y0 + 1);
}

struct RectTilesF {
    const uint32_t* sorted_rec;
    const uint2* rects;
    __device__ unsigned long long operator()(unsigned long long j) const { return rect_tiles(rects[sorted_rec[j]]); }
};

// The scan's one-block pass also leaves the pair count: need_pairs, the
// count clamped to the capacity, and the overflow bit.
void scan_pairs(const uint32_t* sorted_rec, const uint2* rects, const StateHeader* hdr_n_records,
                unsigned long long rec_cap, unsigned long long* pair_off, unsigned long long* tile_sums,
                StateHeader* hdr, unsigned long long pair_cap, cudaStream_t s) {
    const ScanTotal total{&hdr->need_pairs, &hdr->n_pairs, pair_cap, &hdr->status, kStatusPairOverflow};
    device_exclusive_scan<RectTilesF, unsigned long long>(RectTilesF{sorted_rec, rects}, &hdr_n_records->n_records,
                                                          rec_cap, tile_sums, pair_off, total, s);
}

// The views' first tile ids and tile columns, staged in shared memory: the
// per-entry kernels below read them once per list entry.
__device__ __forceinline__ void load_tile_geometry(long long* s_base, int* s_cols, const ViewParams* views,
                                                   int n_views) {
    for (int v = threadIdx.x; v < n_views; v += blockDim.x) {
        s_base[v] = views[v].tile_base;
        s_cols[v] = views[v].tiles_x;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) emit_pairs_k(const ViewParams* __restrict__ views, int n_views,
                                                    const uint32_t* __restrict__ sorted_rec,
                                                    const Record* __restrict__ recs, const uint2* __restrict__ rects,
                                                    const unsigned long long* __restrict__ pair_off,
                                                    const StateHeader* __restrict__ hdr, unsigned long long rec_cap,
                                                    uint32_t* __restrict__ pair_keys, uint32_t* __restrict__ pair_vals,
                                                    unsigned long long pair_cap) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ long long s_base[kMaxViews];
    __shared__ int s_cols[kMaxViews];
    load_tile_geometry(s_base, s_cols, views, n_views);
    const unsigned long long n = scan_len(&hdr->n_records, rec_cap);
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t rec = sorted_rec[j];
        if (!rogs_ok(rec < rec_cap, 401u)) continue;
        const uint2 r = rects[rec];
        const int x0 = (int)(r.x & 0xffffu), y0 = (int)(r.x >> 16);
        const int x1 = (int)(r.y & 0xffffu), y1 = (int)(r.y >> 16);
        if (x1 < x0 || y1 < y0) continue;
        const uint32_t vi = recs[rec].view;
        if (!rogs_ok(vi < (uint32_t)n_views, 403u)) continue;
        unsigned long long p = pair_off[j];
        const long long base = s_base[vi];
        const int cols = s_cols[vi];
        for (int ty = y0; ty <= y1; ++ty) {
            for (int tx = x0; tx <= x1; ++tx, ++p) {
                if (p >= pair_cap) return;  // overflow: recorded by the pair scan
                pair_keys[p] = (uint32_t)(base + (long long)ty * cols + tx);
                pair_vals[p] = rec;
            }
        }
    }
}

void emit_pairs(const ViewParams* views, int n_views, const uint32_t* sorted_rec, const Record* recs, const uint2* rects,
                const unsigned long long* pair_off, const StateHeader* hdr, unsigned long long rec_cap,
                uint32_t* pair_keys, uint32_t* pair_vals, unsigned long long pair_cap, cudaStream_t s) {
    unsigned long long blocks = (rec_cap + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_pdl(emit_pairs_k, dim3((int)blocks), dim3(256), 0, s, views, n_views, sorted_rec, recs, rects, pair_off, hdr, rec_cap, pair_keys,
                                              pair_vals, pair_cap);
    note_launches(1);
}

__global__ void __launch_bounds__(256) tile_ranges_k(const uint32_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ pair_rec,
                                                     const Record* __restrict__ recs,
                                                     const ViewParams* __restrict__ views, int n_views, Consts k,
                                                     const StateHeader* __restrict__ hdr, unsigned long long cap,
                                                     uint2* __restrict__ ranges, float4* __restrict__ pair_mc,
                                                     uint8_t* __restrict__ pair_blk) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ long long s_base[kMaxViews];
    __shared__ int s_cols[kMaxViews];
    load_tile_geometry(s_base, s_cols, views, n_views);
    const unsigned long long n = scan_len(&hdr->n_pairs, cap);
    const int bw = block_w(k.tile_w, k.tile_h), bh = 32 / bw;
    const int wx = k.tile_w / bw, wy = k.tile_h / bh;   // the warps' pixel blocks of a tile: wx columns, wy rows
    for (unsigned long long p = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < n;
         p += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t t = keys[p];
        if (p == 0 || keys[p - 1] != t) ranges[t].x = (uint32_t)p;
        if (p + 1 == n || keys[p + 1] != t) ranges[t].y = (uint32_t)(p + 1);
        if (!rogs_ok(pair_rec[p] < k.rec_cap, 402u)) continue;
        const float4* r4 = reinterpret_cast<const float4*>(recs + pair_rec[p]);
        const float4 m = r4[0], c = r4[1];
        const uint32_t vi = __float_as_uint(r4[2].w);   // the record's view: the tile is in it
        pair_mc[2 * p] = m;
        pair_mc[2 * p + 1] = conic_to_exp2(c);   // the form the list walks evaluate
        if (!rogs_ok(vi < (uint32_t)n_views, 404u)) continue;
        const uint32_t lt = (uint32_t)((long long)t - s_base[vi]);   // tile within its view (< 2^31)
        const uint32_t cols = (uint32_t)s_cols[vi];
        const uint32_t ty = lt / cols, tx = lt - ty * cols;
        const float2 r = block_cull_radii(c, k.alpha_min);
        uint32_t bm = 0;
        int w = 0;
        for (int yb = 0; yb < wy; ++yb) {
            const float by = (float)((int)ty * k.tile_h + yb * bh);
            for (int xb = 0; xb < wx; ++xb, ++w)
                if (box_hits_block(m, r, (float)((int)tx * k.tile_w + xb * bw), by, bw, bh)) bm |= 1u << w;
        }
        pair_blk[p] = (uint8_t)bm;
    }
}

void tile_ranges(const uint32_t* sorted_tile, const uint32_t* pair_rec, const Record* recs, const ViewParams* views,
                 int n_views, Consts k, const StateHeader* hdr, unsigned long long pair_cap, uint2* ranges,
                 float4* pair_mc, uint8_t* pair_blk, cudaStream_t s) {
    unsigned long long blocks = (pair_cap + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_pdl(tile_ranges_k, dim3((int)blocks), dim3(256), 0, s, sorted_tile, pair_rec, recs, views, n_views, k, hdr, pair_cap, ranges,
                                              pair_mc, pair_blk);
    note_launches(1);
}

// Tile schedule key: an 8-bit logarithmic length class (steps of 2^(1/16),
// about 4 %, up to 2^16 entries), ascending key = descending list length, so
// one stable pass over it gives the longest-list-first order.
__device__ __forceinline__ uint32_t tile_class_key(const uint2* __restrict__ ranges, long long t) {
    const uint2 r = ranges[t];
    const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
    const float lc = 16.0f * __log2f(1.0f + (float)len);
    return 255u - (lc < 255.0f ? (uint32_t)lc : 255u);
}

__global__ void __launch_bounds__(256) tile_keys_k(const uint2* __restrict__ ranges, long long n_tiles,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                   uint32_t* __restrict__ order, int sort_ok) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_tiles;
         t += (long long)gridDim.x * blockDim.x) {
        if (!sort_ok) {
            order[t] = (uint32_t)t;
            continue;
        }
        keys[t] = tile_class_key(ranges, t);
        vals[t] = (uint32_t)t;
    }
}

// The same stable order in one block when the frame has few tiles: a
// counting sort on the class key.  Warp w owns the w-th contiguous segment of
// tiles; (1) each warp counts its segment's keys, (2) digit-major exclusive
// offsets over (digit, warp), (3) each warp scatters its segment in order,
// ranking equal keys inside 32-tile steps by lane.  No block waits on
// another; one launch replaces the key kernel and a three-launch radix pass.
constexpr int kOrderThreads = 1024;
constexpr long long kOrderOneBlockMax = 32768;

__global__ void __launch_bounds__(kOrderThreads) tile_order_block_k(const uint2* __restrict__ ranges,
                                                                    long long n_tiles,
                                                                    uint32_t* __restrict__ order) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ uint32_t wh[kOrderThreads / 32][256];   // per-warp counts, then write positions
    __shared__ uint32_t scan_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const long long per = (n_tiles + 31) / 32;
    const long long beg = (long long)warp * per;
    const long long end = beg + per < n_tiles ? beg + per : n_tiles;
    for (int i = threadIdx.x; i < 32 * 256; i += kOrderThreads) (&wh[0][0])[i] = 0u;
    __syncthreads();
    for (long long b = beg; b < end; b += 32) {   // (1)
        const long long t = b + lane;
        const bool valid = t < end;
        const unsigned vm = __ballot_sync(kFull, valid);
        if (valid) {
            const uint32_t d = tile_class_key(ranges, t);
            const unsigned peers = __match_any_sync(vm, d);
            if ((peers & lt) == 0u) wh[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    uint32_t tot = 0, inc = 0;   // (2): thread d < 256 owns digit d
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        for (int w = 0; w < 32; ++w) tot += wh[w][d];
        inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += x;
        }
        if (lane == 31) scan_w[warp] = inc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t c = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t x = scan_w[w];
            scan_w[w] = c;
            c += x;
        }
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        uint32_t run = scan_w[warp] + inc - tot;
        for (int w = 0; w < 32; ++w) {
            const uint32_t c = wh[w][d];
            wh[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (long long b = beg; b < end; b += 32) {   // (3)
        const long long t = b + lane;
        const bool valid = t < end;
        const unsigned vm = __ballot_sync(kFull, valid);
        uint32_t d = 0;
        unsigned peers = 0;
        if (valid) {
            d = tile_class_key(ranges, t);
            peers = __match_any_sync(vm, d);
            order[wh[warp][d] + __popc(peers & lt)] = (uint32_t)t;
        }
        __syncwarp();
        if (valid && (peers & lt) == 0u) wh[warp][d] += __popc(peers);
        __syncwarp();
    }
}

void order_tiles(const uint2* ranges, long long n_tiles, uint32_t* order, bool sort_ok, uint32_t* ka, uint32_t* va,
                 uint32_t* kb, uint32_t* vb, uint32_t* kalt, uint32_t* hist, cudaStream_t s, int sort_tile) {
    if (sort_ok && n_tiles <= kOrderOneBlockMax) {
        if (n_tiles > 0) {
            launch_pdl(tile_order_block_k, dim3(1), dim3(kOrderThreads), 0, s, ranges, n_tiles, order);
            note_launches(1);
        }
        return;
    }
    long long blocks = (n_tiles + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    launch_pdl(tile_keys_k, dim3((int)blocks), dim3(256), 0, s, ranges, n_tiles, ka, va, order, sort_ok ? 1 : 0);
    note_launches(1);
    if (sort_ok)
        radix_sort_pairs(ka, va, kb, order, kalt, vb, nullptr, (unsigned long long)n_tiles, 8, hist, s, sort_tile);
}

#ifdef ROGS_CHECKED
unsigned check_word_bin() { return rogs_check_word_take(); }
#endif

}  // namespace rogs
