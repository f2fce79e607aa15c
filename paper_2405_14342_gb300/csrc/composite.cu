// composite.cu -- stage 3: per-tile front-to-back alpha compositing.
//
// RoGs Sec. 3.3.1, Eq. 6:  c(p) = sum_k c_k a_k prod_{i<k} (1 - a_i),
// a_k = min(alpha_max, alpha_k g_k(p)); the same weights composite the C
// semantic logits ("the color c is replaced by the semantic vector") and the
// camera depth; Eq. 7 applies the per-camera exposure e^a c + b to rgb.
//
// One CTA per tile; each warp owns an 8x4 pixel block of the tile (one
// pixel per lane) and walks the tile's depth-ordered list on its own, 32
// entries at a time: the lanes read one record each, keep only the entries
// whose footprint can reach the warp's block (a conservative ellipse
// bounding box), compact them in order into the warp's shared-memory slots
// together with their features (rgb, sem, depth), and then every lane walks
// the compacted entries for its pixel, computing only the scalar recursion
// (alpha, the transmittance stop, w = a T) and writing its weights into a
// (entry x pixel) table.  The channel sums of Eq. 6 for the chunk are then
// one dense product, out[pixel][ch] += W[pixel][entry] F[entry][ch]
// (32 x NCP x up to 32), taken on the tensor cores (warp-level TF32 MMA in
// three passes, about FP32 accurate).  A warp stops as soon as all its
// pixels have stopped, without waiting for the rest of the tile: there is no
// block-wide barrier.
#include "kernels.h"

namespace rogs {

int padded_channels(int C) {
    const int n = 3 + C + 1;   // a multiple of 8: the MMA n-tile
    if (n <= 8) return 8;
    if (n <= 16) return 16;
    if (n <= 24) return 24;
    if (n <= 32) return 32;
    return 64;
}

constexpr int kWStride = 40;   // weight table: row = entry, column = pixel (rows 8 banks apart)

template <int NCP>
__host__ __device__ constexpr int fwd_warp_floats() {
    return 32 * 4 + 32 * 4 + 32 * feat_stride<NCP>() + 32 + 32 * kWStride;
}

template <int TW, int TH, int NCP>
__global__ void __launch_bounds__(TW * TH) composite_fwd_k(const ViewParams* __restrict__ views, int n_views, Consts k,
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
    constexpr int WX = TW / 8;
    constexpr int SF = feat_stride<NCP>();
    constexpr int NT = NCP / 8;   // MMA n-tiles over the channels
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;   // MMA fragment coordinates
    extern __shared__ float4 smem_fwd[];
    float* wbase = reinterpret_cast<float*>(smem_fwd) + warp * fwd_warp_floats<NCP>();
    float4* s_m = reinterpret_cast<float4*>(wbase);
    float4* s_c = s_m + 32;
    float* s_f = reinterpret_cast<float*>(s_c + 32);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_f + 32 * SF);
    float* s_w = reinterpret_cast<float*>(s_idx + 32);

    const long long tile = tile_order[blockIdx.x];
    const int vi = view_of_tile(views, n_views, tile);
    const ViewParams& v = views[vi];
    const int W = v.W, H = v.H;
    const long long lt = tile - v.tile_base;
    const int tx = (int)(lt % v.tiles_x), ty = (int)(lt / v.tiles_x);
    const int bx = tx * TW + (warp % WX) * 8, by = ty * TH + (warp / WX) * 4;
    const int px = bx + (lane & 7), py = by + (lane >> 3);
    const bool inside = px < W && py < H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
    const int C = k.C;
    const float amin = k.alpha_min, amax = k.alpha_max, tmin = k.t_min;
    const unsigned lt_mask = lanemask_lt();

    float T = 1.0f;
    float acc[2][NT][4];   // C fragments: pixels 16 mt + g (+8), channels 8 nt + 2t (+1)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.0f;
    uint32_t last = 0, ncomp = 0;
    bool done = !inside;

    // block masks of the next chunk are loaded one chunk ahead
    uint32_t bm_next = start + lane < end ? pair_blk[start + lane] : 0u;
    for (uint32_t base = start; base < end; base += 32) {
        if (__all_sync(kFull, done)) break;
        const uint32_t j = base + lane;
        const uint32_t bm = bm_next;
        bm_next = j + 32 < end ? pair_blk[j + 32] : 0u;
        bool hit = false;
        uint32_t rec = 0;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f), c = m;
        if (j < end) {   // the block mask says whether the entry can reach this warp's block
            hit = (bm >> warp) & 1u;
            if (hit) {
                rec = pair_rec[j];
                m = pair_mc[2ull * j];
                c = pair_mc[2ull * j + 1];
            }
        }
        const unsigned mask = __ballot_sync(kFull, hit);
        if (!mask) continue;
        const int h = __popc(mask);
        const int h8 = (h + 7) & ~7;   // k extent of the product, padded with zero rows
        if (hit) {
            const int slot = __popc(mask & lt_mask);
            s_m[slot] = m;
            s_c[slot] = c;
            s_idx[slot] = j - start + 1;
            stage_record_features<NCP>(s_f + slot * SF, feat, rec);
        }
        if (lane >= h && lane < h8) {   // zero feature rows pad k up to a multiple of 8
#pragma unroll
            for (int ch = 0; ch < NCP; ++ch) s_f[lane * SF + ch] = 0.0f;
        }
        __syncwarp();
        // scalar recursion, lane = pixel: entries below alpha_min and entries
        // after the stop get w = 0
        int lslot = -1;   // last slot this pixel composited in the chunk
#pragma unroll 2
        for (int jj = 0; jj < h; ++jj) {
            const float4 mm = s_m[jj];
            const float4 cc = s_c[jj];
            const float dx = pix_offset(pxc, mm.x, mm.z);
            const float dy = pix_offset(pyc, mm.y, mm.w);
            float gp;
            const float a = surfel_alpha(dx, dy, cc.x, cc.y, cc.z, cc.w, amax, gp);
            bool valid = !done && a >= amin;
            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, a));
            const bool stop = valid && Tn < tmin;
            done = done || stop;
            valid = valid && !stop;
            s_w[jj * kWStride + lane] = valid ? __fmul_rn(a, T) : 0.0f;
            T = valid ? Tn : T;
            lslot = valid ? jj : lslot;
            ncomp += valid ? 1u : 0u;
        }
        if (lslot >= 0) last = s_idx[lslot];
        for (int jj = h; jj < h8; ++jj) s_w[jj * kWStride + lane] = 0.0f;
        __syncwarp();
        // out[pixel][ch] += W[pixel][entry] F[entry][ch] over this chunk's entries
        for (int k0 = 0; k0 < h8; k0 += 8) {
            uint32_t ah[2][4], al[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const float* w0 = s_w + (k0 + t) * kWStride + 16 * mt + g;
                const float* w1 = s_w + (k0 + t + 4) * kWStride + 16 * mt + g;
                split_tf32(w0[0], ah[mt][0], al[mt][0]);
                split_tf32(w0[8], ah[mt][1], al[mt][1]);
                split_tf32(w1[0], ah[mt][2], al[mt][2]);
                split_tf32(w1[8], ah[mt][3], al[mt][3]);
            }
            uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                split_tf32(s_f[(k0 + t) * SF + 8 * nt + g], bh[nt][0], bl[nt][0]);
                split_tf32(s_f[(k0 + t + 4) * SF + 8 * nt + g], bh[nt][1], bl[nt][1]);
            }
            mma_tf32x3_tiles<NT>(acc, ah, al, bh, bl, true);
        }
        __syncwarp();
    }

    const long long plane = (long long)W * H;
    const int nch = 3 + C + 1;
    const float ea = expf(exposure_ab[2 * v.exp_idx]);
    const float eb = exposure_ab[2 * v.exp_idx + 1];
    float* o = out + (long long)nch * v.pix_base;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {
            const int p = 16 * mt + g + 8 * hr;   // this fragment row's pixel
            const int qx = bx + (p & 7), qy = by + (p >> 3);
            if (qx >= W || qy >= H) continue;
            float* op = o + (long long)qy * W + qx;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int ch = 8 * nt + 2 * t + cc;
                    const float val = acc[mt][nt][2 * hr + cc];
                    if (ch < 3) op[ch * plane] = fmaf(ea, val, eb);
                    else if (ch < nch) op[ch * plane] = val;
                }
        }
    if (inside) {
        const long long pix = v.pix_base + (long long)py * W + px;
        pix_T[pix] = T;
        pix_last[pix] = last;
    }
    // composited-pair counter (E_alg)
    unsigned long long cnt = ncomp;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o2);
    if (lane == 0 && cnt) atomicAdd(&hdr->composited, cnt);
}

static size_t fwd_smem_bytes(int blk, int ncp) {
    const int sf = (ncp % 32 == 8 || ncp % 32 == 24) ? ncp : ncp + 8;
    return (size_t)(blk / 32) * 4 * (size_t)(32 * 4 + 32 * 4 + 32 * sf + 32 + 32 * kWStride);
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
        composite_fwd_k<TW, TH, NCP><<<grid, TW * TH, fwd_smem_bytes(TW * TH, NCP), s>>>(                     \
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

}  // namespace rogs
