// composite.cu -- stage 3: per-tile front-to-back alpha compositing.
//
// RoGs Sec. 3.3.1, Eq. 6:  c(p) = sum_k c_k a_k prod_{i<k} (1 - a_i),
// a_k = min(alpha_max, alpha_k g_k(p)); the same weights composite the C
// semantic logits ("the color c is replaced by the semantic vector") and the
// camera depth; Eq. 7 applies the per-camera exposure e^a c + b to rgb.
//
// One CTA per tile; each warp owns a 32-pixel block of the tile (one pixel
// per lane; 16x2 in 16x16 tiles, 8x4 otherwise) and walks the tile's
// depth-ordered list on its own, 32 entries at a time: the lanes read one
// record each, keep only the entries whose footprint can reach the warp's
// block (a conservative ellipse bounding box), compact them in order into the
// warp's shared-memory slots together with their features (rgb, sem, depth),
// and then every lane walks the compacted entries for its pixel: the scalar
// recursion (alpha, the transmittance stop, w = a T) and the channel sums of
// Eq. 6, out[ch] += w f[ch], as FP32 fused multiply-adds on the lane's own
// accumulators, the feature row read from shared memory as broadcast
// float4s.  A warp stops as soon as all its pixels have stopped, without
// waiting for the rest of the tile: there is no block-wide barrier.
#include "kernels.h"

namespace rogs {

int padded_channels(int C) {
    const int n = 3 + C + 1;   // a multiple of 8: whole float4 rows, 32-byte aligned
    if (n <= 8) return 8;
    if (n <= 16) return 16;
    if (n <= 24) return 24;
    if (n <= 32) return 32;
    return 64;
}

template <int NCP>
__host__ __device__ constexpr int fwd_warp_floats() {
    return 32 * 4 + 32 * 4 + 32 * NCP + 32;
}

// Up to 24 channels 24 warps stay resident per SM with up to 85 registers
// each (measured: 2 % faster than 32 warps at 64 registers, where the walk
// spills); wider rows run 16 warps per SM with up to 128 registers each.
template <int NCP>
constexpr int fwd_threads_per_sm() { return NCP <= 24 ? 768 : 512; }

template <int TW, int TH, int NCP>
__global__ void __launch_bounds__(TW * TH, fwd_threads_per_sm<NCP>() / (TW * TH)) composite_fwd_k(const ViewParams* __restrict__ views, int n_views, Consts k,
                                                           SurfelPtrs sp, const Record* __restrict__ recs,
                                                           const float* __restrict__ feat,
                                                           const float4* __restrict__ pair_mc,
                                                           const uint8_t* __restrict__ pair_blk,
                                                           const uint32_t* __restrict__ pair_rec,
                                                           const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ tile_order,
                                                           const float* __restrict__ exposure_ab,
                                                           float* __restrict__ out, float* __restrict__ pix_T,
                                                           uint32_t* __restrict__ pix_last,
                                                           StateHeader* __restrict__ hdr) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    constexpr int BW = block_w(TW, TH), BH = 32 / BW, WX = TW / BW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ float4 smem_fwd[];
    __shared__ unsigned long long s_comp;   // the CTA's composited pairs
    __shared__ unsigned s_done;             // warps of the CTA that have added theirs
    if (threadIdx.x == 0) { s_comp = 0ull; s_done = 0u; }
    __syncthreads();
    float* wbase = reinterpret_cast<float*>(smem_fwd) + warp * fwd_warp_floats<NCP>();
    float4* s_m = reinterpret_cast<float4*>(wbase);
    float4* s_c = s_m + 32;
    float* s_f = reinterpret_cast<float*>(s_c + 32);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_f + 32 * NCP);

    const long long tile = tile_order[blockIdx.x];
    const int vi = view_of_tile(views, n_views, tile);
    const ViewParams& v = views[vi];
    const int W = v.W, H = v.H;
    const long long lt = tile - v.tile_base;
    const int tx = (int)(lt % v.tiles_x), ty = (int)(lt / v.tiles_x);
    const int bx = tx * TW + (warp % WX) * BW, by = ty * TH + (warp / WX) * BH;
    const int px = bx + lane % BW, py = by + lane / BW;
    const bool inside = px < W && py < H;
    const int2 org = offset_origin(bx, by);   // the same for every pixel of the block
    const float lx = (float)(px - org.x), ly = (float)(py - org.y);
    const uint2 rg = ranges[tile];
    const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
    const int C = k.C;
    const float amin = k.alpha_min, amax = k.alpha_max, tmin = k.t_min;
    const unsigned lt_mask = lanemask_lt();

    float T = 1.0f;
    float acc[NCP];   // this lane's pixel: rgb, C logits, depth, zero padding
#pragma unroll
    for (int ch = 0; ch < NCP; ++ch) acc[ch] = 0.0f;
    uint32_t last = 0, ncomp = 0;
    bool done = !inside;

    // block masks of the next chunk are loaded one chunk ahead
    uint32_t bm_next = start + lane < end ? pair_blk[start + lane] : 0u;
    // the first chunk's records and mean/conic are loaded with its block masks,
    // whether or not the entry reaches the block (one round trip less)
    uint32_t rec_first = 0;
    float4 m_first = make_float4(0.f, 0.f, 0.f, 0.f), c_first = m_first;
    if (start + lane < end && rogs_ok(start + lane < k.pair_cap, 101u)) {
        rec_first = pair_rec[start + lane];
        m_first = pair_mc[2ull * (start + lane)];
        c_first = pair_mc[2ull * (start + lane) + 1];
    }
    for (uint32_t base = start; base < end; base += 32) {
        if (__all_sync(kFull, done)) break;
        const uint32_t j = base + lane;
        const uint32_t bm = bm_next;
        bm_next = j + 32 < end ? pair_blk[j + 32] : 0u;
        bool hit = false;
        uint32_t rec = 0;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f), c = m;
        if (j < end) {   // the block mask says whether the entry can reach this warp's block
            hit = (bm >> warp) & 1u && rogs_ok(j < k.pair_cap, 101u);
            if (hit) {
                const bool first = base == start;
                rec = first ? rec_first : pair_rec[j];
                hit = rogs_ok(rec < k.rec_cap, 102u);
                if (hit) {
                    m = first ? m_first : pair_mc[2ull * j];
                    c = first ? c_first : pair_mc[2ull * j + 1];
                }
            }
        }
        const unsigned mask = __ballot_sync(kFull, hit);
        if (!mask) continue;
        const int h = __popc(mask);
        if (hit) {
            const int slot = __popc(mask & lt_mask);
            s_m[slot] = block_offsets(m, org);
            s_c[slot] = c;
            s_idx[slot] = j - start + 1;
            stage_record_features<NCP>(s_f + slot * NCP, feat, rec);
        }
        __syncwarp();
        // lane = pixel: entries below alpha_min and entries after the stop get
        // w = 0 (branch-free), every entry adds w f to the lane's channels
        int lslot = -1;   // last slot this pixel composited in the chunk
#pragma unroll 2
        for (int jj = 0; jj < h; ++jj) {
            const float4 mm = s_m[jj];
            const float4 cc = s_c[jj];
            const float dx = __fadd_rn(mm.x, lx);
            const float dy = __fadd_rn(mm.y, ly);
            float gp;
            const float a = surfel_alpha(dx, dy, cc.x, cc.y, cc.z, cc.w, amax, gp);
            bool valid = !done && a >= amin;
            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, a));
            const bool stop = valid && Tn < tmin;
            done = done || stop;
            valid = valid && !stop;
            const float w = valid ? __fmul_rn(a, T) : 0.0f;
            T = valid ? Tn : T;
            lslot = valid ? jj : lslot;
            ncomp += valid ? 1u : 0u;
            const float4* f4 = reinterpret_cast<const float4*>(s_f + jj * NCP);
#pragma unroll
            for (int q = 0; q < NCP / 4; ++q) {
                const float4 f = f4[q];
                acc[4 * q] = fmaf(w, f.x, acc[4 * q]);
                acc[4 * q + 1] = fmaf(w, f.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(w, f.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(w, f.w, acc[4 * q + 3]);
            }
        }
        if (lslot >= 0) last = s_idx[lslot];
        __syncwarp();
    }

    const long long plane = (long long)W * H;
    const int nch = 3 + C + 1;
    const float ea = expf(exposure_ab[2 * v.exp_idx]);
    const float eb = exposure_ab[2 * v.exp_idx + 1];
    if (inside) {
        float* op = out + (long long)nch * v.pix_base + (long long)py * W + px;
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch) {
            if (ch < 3) op[ch * plane] = fmaf(ea, acc[ch], eb);
            else if (ch < nch) op[ch * plane] = acc[ch];
        }
    }
    if (inside) {
        const long long pix = v.pix_base + (long long)py * W + px;
        pix_T[pix] = T;
        pix_last[pix] = last;
    }
    // composited-pair counter (E_alg): summed over the CTA in shared memory;
    // the CTA's last warp to finish adds it to the global counter, so the
    // counter takes one atomic per tile instead of one per warp
    unsigned long long cnt = ncomp;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o2);
    if (lane == 0) {
        if (cnt) atomicAdd(&s_comp, cnt);
        __threadfence_block();
        if (atomicAdd(&s_done, 1u) == (unsigned)(TW * TH / 32) - 1u) {
            __threadfence_block();
            const unsigned long long total = atomicAdd(&s_comp, 0ull);
            if (total) atomicAdd(&hdr->composited, total);
        }
    }
}

static size_t fwd_smem_bytes(int blk, int ncp) {
    return (size_t)(blk / 32) * 4 * (size_t)(32 * 4 + 32 * 4 + 32 * ncp + 32);
}

template <int TW, int TH, int NCP>
static void fwd_attr() {
    static unsigned long long done_mask = 0;   // one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !((done_mask >> dev) & 1ull)) {
        cudaFuncSetAttribute(composite_fwd_k<TW, TH, NCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fwd_smem_bytes(TW * TH, NCP));
        done_mask |= 1ull << dev;
    }
}

template <int TW, int TH>
static void prepare_fwd_tile() {
    fwd_attr<TW, TH, 8>(); fwd_attr<TW, TH, 16>();
    fwd_attr<TW, TH, 24>(); fwd_attr<TW, TH, 32>(); fwd_attr<TW, TH, 64>();
}

void prepare_composite_fwd() {
    prepare_fwd_tile<16, 16>();
    prepare_fwd_tile<32, 8>();
    prepare_fwd_tile<8, 8>();
}

template <int TW, int TH>
static void launch_fwd_tile(int ncp, long long total_tiles, cudaStream_t s, const ViewParams* views, int n_views,
                            Consts k, SurfelPtrs sp, const Record* recs, const float* feat, const float4* pair_mc,
                            const uint8_t* pair_blk, const uint32_t* pair_rec, const uint2* ranges,
                            const uint32_t* tile_order, const float* exposure_ab, float* out, float* pix_T,
                            uint32_t* pix_last, StateHeader* hdr) {
    dim3 grid((unsigned)total_tiles);
#define ROGS_FWD(NCP)                                                                                          \
    do {                                                                                                       \
        fwd_attr<TW, TH, NCP>();                                                                               \
        launch_pdl(composite_fwd_k<TW, TH, NCP>, dim3(grid), dim3(TW * TH), fwd_smem_bytes(TW * TH, NCP), s,                      \
            views, n_views, k, sp, recs, feat, pair_mc, pair_blk, pair_rec, ranges, tile_order, exposure_ab, out, \
            pix_T, pix_last, hdr);                                                                             \
        note_launches(1);                                                                                      \
    } while (0)
    switch (ncp) {
        case 8: ROGS_FWD(8); break;
        case 16: ROGS_FWD(16); break;
        case 24: ROGS_FWD(24); break;
        case 32: ROGS_FWD(32); break;
        default: ROGS_FWD(64); break;
    }
#undef ROGS_FWD
}

void composite_fwd(int tile_w, int tile_h, int C, const ViewParams* views, int n_views, long long total_tiles,
                   Consts k, SurfelPtrs sp, const Record* recs, const float* feat, const float4* pair_mc, const uint8_t* pair_blk, const uint32_t* pair_rec, const uint2* ranges,
                   const uint32_t* tile_order, const float* exposure_ab, float* out, float* pix_T, uint32_t* pix_last, StateHeader* hdr,
                   cudaStream_t s) {
    const int ncp = padded_channels(C);
    if (tile_w == 32 && tile_h == 8)
        launch_fwd_tile<32, 8>(ncp, total_tiles, s, views, n_views, k, sp, recs, feat, pair_mc, pair_blk, pair_rec, ranges, tile_order, exposure_ab, out,
                               pix_T, pix_last, hdr);
    else if (tile_w == 8 && tile_h == 8)
        launch_fwd_tile<8, 8>(ncp, total_tiles, s, views, n_views, k, sp, recs, feat, pair_mc, pair_blk, pair_rec, ranges, tile_order, exposure_ab, out,
                              pix_T, pix_last, hdr);
    else
        launch_fwd_tile<16, 16>(ncp, total_tiles, s, views, n_views, k, sp, recs, feat, pair_mc, pair_blk, pair_rec, ranges, tile_order, exposure_ab, out,
                                pix_T, pix_last, hdr);
}

#ifdef ROGS_CHECKED
unsigned check_word_composite() { return rogs_check_word_take(); }
#endif

}  // namespace rogs
