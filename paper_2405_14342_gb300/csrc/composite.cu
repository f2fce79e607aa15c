// composite.cu -- stage 3: per-tile front-to-back alpha compositing.
//
// RoGs Sec. 3.3.1, Eq. 6:  c(p) = sum_k c_k a_k prod_{i<k} (1 - a_i),
// a_k = min(alpha_max, alpha_k g_k(p)); the same weights composite the C
// semantic logits ("the color c is replaced by the semantic vector") and the
// camera depth; Eq. 7 applies the per-camera exposure e^a c + b to rgb.
//
// One CTA per tile (tile_w x tile_h pixels, one pixel per thread; each warp
// covers an 8x4 pixel block so its lanes see similar lists).  The tile's
// list is processed in chunks of one entry per thread: each thread stages
// one entry's record (two 16-byte loads) and its features (rgb, sem, depth)
// into shared memory; then every thread walks the chunk from shared memory
// (broadcast reads).  A pixel stops before the entry that would take its
// transmittance below t_min; the CTA leaves the list once all its pixels
// have stopped (__syncthreads_count).
#include "kernels.h"

namespace rogs {

int padded_channels(int C) {
    const int n = 3 + C + 1;
    if (n <= 8) return 8;
    if (n <= 12) return 12;
    if (n <= 16) return 16;
    if (n <= 24) return 24;
    if (n <= 32) return 32;
    return 64;
}

template <int NCP>
__device__ __forceinline__ void stage_entry(const Record* __restrict__ recs, const uint32_t rec, const SurfelPtrs& sp,
                                            int C, float4* s_m, float4* s_c, float* s_f, int slot) {
    const float4* r4 = reinterpret_cast<const float4*>(recs + rec);
    const float4 a = r4[0];
    const float4 b = r4[1];
    const float4 c = r4[2];
    s_m[slot] = a;
    s_c[slot] = b;
    const uint32_t s = __float_as_uint(c.z);
    float* f = s_f + slot * NCP;
    f[0] = sp.rgb[3ull * s];
    f[1] = sp.rgb[3ull * s + 1];
    f[2] = sp.rgb[3ull * s + 2];
    const float* sem = sp.sem + (unsigned long long)C * s;
    for (int ch = 0; ch < C; ++ch) f[3 + ch] = sem[ch];
    f[3 + C] = c.x;  // camera depth
#pragma unroll
    for (int ch = 0; ch < NCP; ++ch)
        if (ch > 3 + C) f[ch] = 0.0f;
}

template <int TW, int TH, int NCP>
__global__ void __launch_bounds__(TW * TH) composite_fwd_k(const ViewParams* __restrict__ views, int n_views, Consts k,
                                                           SurfelPtrs sp, const Record* __restrict__ recs,
                                                           const uint32_t* __restrict__ pair_rec,
                                                           const uint2* __restrict__ ranges,
                                                           const float* __restrict__ exposure_ab,
                                                           float* __restrict__ out, float* __restrict__ pix_T,
                                                           uint32_t* __restrict__ pix_last,
                                                           StateHeader* __restrict__ hdr) {
    constexpr int BLK = TW * TH;
    constexpr int WX = TW / 8;
    extern __shared__ float4 smem_fwd[];
    float4* s_m = smem_fwd;
    float4* s_c = s_m + BLK;
    float* s_f = reinterpret_cast<float*>(s_c + BLK);
    __shared__ unsigned long long s_cnt;

    const long long tile = blockIdx.x;
    const int vi = view_of_tile(views, n_views, tile);
    const ViewParams& v = views[vi];
    const int W = v.W, H = v.H;
    const long long lt = tile - v.tile_base;
    const int tx = (int)(lt % v.tiles_x), ty = (int)(lt / v.tiles_x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = tx * TW + (warp % WX) * 8 + (lane & 7);
    const int py = ty * TH + (warp / WX) * 4 + (lane >> 3);
    const bool inside = px < W && py < H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
    const int C = k.C;
    const float amin = k.alpha_min, amax = k.alpha_max, tmin = k.t_min;

    if (threadIdx.x == 0) s_cnt = 0ull;
    float T = 1.0f;
    float acc[NCP];
#pragma unroll
    for (int ch = 0; ch < NCP; ++ch) acc[ch] = 0.0f;
    uint32_t last = 0, ncomp = 0;
    bool done = !inside;

    for (uint32_t base = start; base < end; base += BLK) {
        if (__syncthreads_count(done) == BLK) break;
        const uint32_t j = base + threadIdx.x;
        if (j < end) stage_entry<NCP>(recs, pair_rec[j], sp, C, s_m, s_c, s_f, threadIdx.x);
        __syncthreads();
        const int cnt = (int)min((uint32_t)BLK, end - base);
        if (!done) {
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 m = s_m[jj];
                const float4 c = s_c[jj];
                const float dx = pix_offset(pxc, m.x, m.z);
                const float dy = pix_offset(pyc, m.y, m.w);
                float g;
                const float a = surfel_alpha(dx, dy, c.x, c.y, c.z, c.w, amax, g);
                if (a < amin) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.0f, a));
                if (Tn < tmin) {
                    done = true;
                    break;
                }
                const float w = __fmul_rn(a, T);
                const float4* f4 = reinterpret_cast<const float4*>(s_f + jj * NCP);
#pragma unroll
                for (int q = 0; q < NCP / 4; ++q) {
                    const float4 f = f4[q];
                    acc[4 * q + 0] = fmaf(w, f.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(w, f.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(w, f.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(w, f.w, acc[4 * q + 3]);
                }
                T = Tn;
                last = base + jj + 1 - start;
                ++ncomp;
            }
        }
    }

    if (inside) {
        const long long pix = v.pix_base + (long long)py * W + px;
        const long long plane = (long long)W * H;
        const int nch = 3 + C + 1;
        float* o = out + (long long)nch * v.pix_base + (long long)py * W + px;
        const float ea = expf(exposure_ab[2 * v.exp_idx]);
        const float eb = exposure_ab[2 * v.exp_idx + 1];
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch) {
            if (ch < 3) o[ch * plane] = fmaf(ea, acc[ch], eb);
            else if (ch < nch) o[ch * plane] = acc[ch];
        }
        pix_T[pix] = T;
        pix_last[pix] = last;
    }
    // composited-pair counter (E_alg)
    unsigned long long c = ncomp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    __syncthreads();
    if (lane == 0 && c) atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&hdr->composited, s_cnt);
}

static size_t fwd_smem_bytes(int blk, int ncp) { return (size_t)blk * (32 + 4 * (size_t)ncp); }

template <int TW, int TH>
static void launch_fwd_tile(int ncp, long long total_tiles, cudaStream_t s, const ViewParams* views, int n_views,
                            Consts k, SurfelPtrs sp, const Record* recs, const uint32_t* pair_rec, const uint2* ranges,
                            const float* exposure_ab, float* out, float* pix_T, uint32_t* pix_last, StateHeader* hdr) {
    dim3 grid((unsigned)total_tiles);
#define ROGS_FWD(NCP)                                                                                          \
    do {                                                                                                       \
        const size_t sm = fwd_smem_bytes(TW * TH, NCP);                                                        \
        static bool attr_set = false;                                                                          \
        if (!attr_set) {                                                                                       \
            cudaFuncSetAttribute(composite_fwd_k<TW, TH, NCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)sm);                                                                     \
            attr_set = true;                                                                                   \
        }                                                                                                      \
        composite_fwd_k<TW, TH, NCP><<<grid, TW * TH, sm, s>>>(views, n_views, k, sp, recs, pair_rec, ranges, \
                                                               exposure_ab, out, pix_T, pix_last, hdr);       \
        note_launches(1);                                                                                      \
    } while (0)
    switch (ncp) {
        case 8: ROGS_FWD(8); break;
        case 12: ROGS_FWD(12); break;
        case 16: ROGS_FWD(16); break;
        case 24: ROGS_FWD(24); break;
        case 32: ROGS_FWD(32); break;
        default: ROGS_FWD(64); break;
    }
#undef ROGS_FWD
}

void composite_fwd(int tile_w, int tile_h, int C, const ViewParams* views, int n_views, long long total_tiles,
                   Consts k, SurfelPtrs sp, const Record* recs, const uint32_t* pair_rec, const uint2* ranges,
                   const float* exposure_ab, float* out, float* pix_T, uint32_t* pix_last, StateHeader* hdr,
                   cudaStream_t s) {
    const int ncp = padded_channels(C);
    if (tile_w == 32 && tile_h == 8)
        launch_fwd_tile<32, 8>(ncp, total_tiles, s, views, n_views, k, sp, recs, pair_rec, ranges, exposure_ab, out,
                               pix_T, pix_last, hdr);
    else if (tile_w == 8 && tile_h == 8)
        launch_fwd_tile<8, 8>(ncp, total_tiles, s, views, n_views, k, sp, recs, pair_rec, ranges, exposure_ab, out,
                              pix_T, pix_last, hdr);
    else
        launch_fwd_tile<16, 16>(ncp, total_tiles, s, views, n_views, k, sp, recs, pair_rec, ranges, exposure_ab, out,
                                pix_T, pix_last, hdr);
}

}  // namespace rogs
