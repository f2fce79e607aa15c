// kernels.h -- host launchers of the librogs kernels (internal interface
// between the C-ABI in api.cu and the kernel translation units).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace rogs {

// Count kernel launches made by this library (reported by rogs_launch_count).
void note_launches(int n);
// True while the rogs_debug_fail_alloc test hook makes scratch allocations fail.
bool debug_alloc_fails();
#ifdef ROGS_CHECKED
// Error words of the bounds-checked build, one per translation unit (read and cleared).
unsigned check_word_composite();
unsigned check_word_backward();
unsigned check_word_sort();
unsigned check_word_bin();
#endif

struct SurfelPtrs {
    const float *xyz, *scale, *quat, *opacity, *rgb, *sem;
    long long n;
};

// Copy of a record's feature row (rgb, C logits, depth, zeros: NCP floats,
// 16-byte aligned) into a shared-memory row; all loads before the stores.
template <int NCP>
__device__ __forceinline__ void stage_record_features(float* f, const float* __restrict__ feat, uint32_t rec) {
    const float4* src = reinterpret_cast<const float4*>(feat + (unsigned long long)rec * NCP);
    float4 v[NCP / 4];
#pragma unroll
    for (int q = 0; q < NCP / 4; ++q) v[q] = src[q];
#pragma unroll
    for (int q = 0; q < NCP / 4; ++q) reinterpret_cast<float4*>(f)[q] = v[q];
}

// cp.async (global -> shared, 16 bytes, cached in L1) and its group fences.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The same copy as stage_record_features, issued as asynchronous copies; the
// caller commits, waits and synchronises the warp before reading the row.
template <int NCP>
__device__ __forceinline__ void stage_record_features_async(float* f, const float* __restrict__ feat, uint32_t rec) {
    const float4* src = reinterpret_cast<const float4*>(feat + (unsigned long long)rec * NCP);
#pragma unroll
    for (int q = 0; q < NCP / 4; ++q) cp_async16(reinterpret_cast<float4*>(f) + q, src + q);
}

struct GradPtrs {
    float *xyz, *scale, *quat, *opacity, *rgb, *sem, *exposure;
};

// ---- sort.cu
constexpr int kRsMinTile = 1024;   // smallest keys-per-CTA option of the radix sort (sizes the histograms)
// Words of the digit histograms for up to `cap` keys: [256][tiles] counts, then the 256 digit totals.
constexpr size_t radix_hist_words(unsigned long long cap) {
    return (size_t)(256ull * (cap == 0 ? 1ull : (cap + kRsMinTile - 1) / kRsMinTile) + 256ull);
}
void prepare_sort();   // set the dynamic shared-memory limits (before any capture)
void radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t* kalt,
                      uint32_t* valt, const unsigned long long* n_ptr, unsigned long long cap, int key_bits,
                      uint32_t* hist, cudaStream_t s, int sort_tile = 4096);

// ---- project.cu
// Upload per-view parameters into device memory (by-value kernel argument).
void upload_views(const ViewsArg& va, int n_views, ViewParams* dst, StateHeader* hdr, cudaStream_t s);
// Cull + visibility bitmask: bits[v * n_words + w] bit l <=> surfel 32w+l visible in view v.
void cull_views(const ViewParams* views, int n_views, Consts k, SurfelPtrs sp, uint32_t* bits, long long n_words,
                cudaStream_t s);
// Record positions: exclusive scan of popc(bits) (view-major) -> word_off; total -> hdr->need_records,
// n_records clamped to rec_cap (overflow bit in hdr->status).
void scan_visible(const uint32_t* bits, long long n_words_total, uint32_t* word_off, uint32_t* tile_sums,
                  StateHeader* hdr, unsigned long long rec_cap, cudaStream_t s);
size_t scan_tile_sums_words(unsigned long long cap);
// Write records, rects, depth sort keys and values.
// Writes the records, their tile rectangles, sort keys / values and the
// per-record feature rows (padded_channels(C) floats each).
void project_records(const ViewParams* views, int n_views, Consts k, SurfelPtrs sp, const uint32_t* bits,
                     const uint32_t* word_off, long long n_words, Record* recs, uint2* rects, float* feat,
                     uint32_t* keys, uint32_t* vals, unsigned long long rec_cap, cudaStream_t s);

// ---- bin.cu
// Pair offsets per depth-sorted record; total -> hdr->need_pairs, n_pairs clamped to pair_cap
// (overflow bit in hdr->status).
void scan_pairs(const uint32_t* sorted_rec, const uint2* rects, const StateHeader* hdr_n_records,
                unsigned long long rec_cap, unsigned long long* pair_off, unsigned long long* tile_sums,
                StateHeader* hdr, unsigned long long pair_cap, cudaStream_t s);
void emit_pairs(const ViewParams* views, int n_views, const uint32_t* sorted_rec, const Record* recs, const uint2* rects,
                const unsigned long long* pair_off, const StateHeader* hdr, unsigned long long rec_cap,
                uint32_t* pair_keys, uint32_t* pair_vals, unsigned long long pair_cap, cudaStream_t s);
// Tile ranges of the sorted pairs; each pair's record mean + conic copied into
// pair order (pair_mc, two float4 per pair) and its block mask (pair_blk,
// bit w = entry_hits_block for the tile's w-th block).
void tile_ranges(const uint32_t* sorted_tile, const uint32_t* pair_rec, const Record* recs, const ViewParams* views,
                 int n_views, Consts k, const StateHeader* hdr, unsigned long long pair_cap, uint2* ranges,
                 float4* pair_mc, uint8_t* pair_blk, cudaStream_t s);
// Tile order by descending list length (identity when sort_ok is false);
// uses ka/va/kb/vb/kalt (>= n_tiles uint32 each) and the radix histogram.
void order_tiles(const uint2* ranges, long long n_tiles, uint32_t* order, bool sort_ok, uint32_t* ka, uint32_t* va,
                 uint32_t* kb, uint32_t* vb, uint32_t* kalt, uint32_t* hist, cudaStream_t s, int sort_tile);

// ---- composite.cu
int padded_channels(int C);
void prepare_composite_fwd();   // set the dynamic shared-memory limits (before any capture)
void composite_fwd(int tile_w, int tile_h, int C, const ViewParams* views, int n_views, long long total_tiles,
                   Consts k, SurfelPtrs sp, const Record* recs, const float* feat, const float4* pair_mc, const uint8_t* pair_blk, const uint32_t* pair_rec, const uint2* ranges,
                   const uint32_t* tile_order, const float* exposure_ab, float* out, float* pix_T, uint32_t* pix_last, StateHeader* hdr,
                   cudaStream_t s);

// ---- backward.cu
// per-record gradient row (32 or 64 floats): mean 2, conic 3, alpha, rgb 3, semantics C, depth
int grad_channels(int C);

struct BwdArgs {
    const ViewParams* views;
    int n_views;
    Consts k;
    SurfelPtrs sp;
    const Record* recs;
    const float* feat;   // per-record feature rows (padded_channels(C) floats)
    const float4* pair_mc;   // per-pair record mean + conic (two float4), in list order
    const uint8_t* pair_blk;  // per-pair warp-block masks, in list order
    const uint32_t* pair_rec;
    const uint2* ranges;
    const uint32_t* tile_order;
    const float* exposure_ab;
    const float* pix_T;
    const uint32_t* pix_last;
    // dL/dout: either grad_out, or (fused training step) computed from these
    const float* grad_out;
    const float* out;
    Targets tg;   // fused: tg.rgb or tg.rgb8 set
    const unsigned long long* mask_count;
    float lambda_c, lambda_s;
    float* loss_partials;   // one per warp of the launch, or null
    // outputs
    float* rec_grad;
    float* d_exposure;
};

void prepare_composite_bwd();
int bwd_loss_partials(long long total_tiles, int tile_w, int tile_h);
void composite_bwd(int tile_w, int tile_h, long long total_tiles, const BwdArgs& a, cudaStream_t s);
void project_bwd(const ViewParams* views, SurfelPtrs sp, const Record* recs, const StateHeader* hdr,
                 unsigned long long rec_cap, float* rec_grad, int C, GradPtrs g, cudaStream_t s);

// ---- adam.cu
void adam_step(const rogs_adam_group* groups, int n_groups, int step, float b1, float b2, float eps, bool zero_grad,
               cudaStream_t s);

// ---- bev.cu
constexpr int kMaxStitch = 16;   // chunk views per stitch launch
struct StitchViews {
    long long pix_end[kMaxStitch];   // exclusive prefix end of each view's pixels in the batch
    int w[kMaxStitch], h[kMaxStitch], x0[kMaxStitch], y0[kMaxStitch];
};
void stitch_views(const StitchViews& sv, int n_views, int nch, const float* out, float* image, int W, int H,
                  cudaStream_t s);

// ---- lidar.cu
struct LidarScratch {   // point-cloud hash: capacity m points, 2^lidar_bucket_bits(m) buckets
    uint32_t *keys, *vals, *skeys, *svals, *kalt, *valt, *hist;
    uint2* ranges;
    float4* sorted;
};
int lidar_bucket_bits(long long m);
int elev_blocks();   // partials written by elev_loss
void lidar_targets(const float* xyz, long long n, const float* pts, long long m, float radius, LidarScratch& w,
                   float* zbar, cudaStream_t s);
void elev_loss(const float* xyz, long long n, const float* zbar, float lambda, float* loss, float* grad_xyz,
               float* partials, cudaStream_t s);

// ---- smooth.cu
int smooth_blocks();   // partials written by smooth_loss
void smooth_loss(const int32_t* grid_index, int grid_w, int grid_h, const float* xyz, float lambda, float* loss,
                 float* grad_xyz, float* partials, cudaStream_t s);

// ---- loss.cu
void loss_fwd_bwd(const ViewParams* views, int n_views, long long total_pixels, int C, const float* out,
                  const Targets& tg, float lambda_c, float lambda_s,
                  float* loss, float* grad_out, unsigned long long* counter, float* partials, int n_blocks_cap,
                  cudaStream_t s);
int loss_blocks(long long total_pixels);
void mask_count(const uint8_t* mask, long long total_pixels, unsigned long long* counter, cudaStream_t s);
// loss[0] = sum(partials) / |M| (+ extra[0] when extra is not NULL)
void loss_final(const float* partials, int n, const unsigned long long* counter, const float* extra, float* loss,
                cudaStream_t s);

// ---- init.cu
void init_from_poses(const float* grid_xy, long long n, const float* poses_dev, long long n_poses, int exact_plane,
                     float* out_z, float* out_quat, int32_t* out_nearest, cudaStream_t s);

}  // namespace rogs
