// backward.cu -- stage 4: reverse-order backward of the compositing and the
// projection (the adjoint of RoGs Eqs. 2, 5, 6, 7; not written in the paper).
//
// composite_bwd_k: each warp owns a 32-pixel block of a tile (16x2 in 16x16
// tiles, 8x4 otherwise; block_w in common.cuh) and walks the
// tile's list backwards from the largest last-composited index of its pixels,
// 32 entries at a time, keeping only the entries whose footprint can reach its
// block.  For every pixel it recovers T_k = T_{k+1} / (1 - a_k) and carries one
// scalar suffix sum, S_k = sum_{j>k} w_j (G . f_j) with G = dL/dout at the
// pixel, which gives dL/da_k = T_k (G . f_k) - S_k / (1 - a_k) without a
// per-pixel list and without per-channel suffix sums (phase A, lane = pixel).
// The per-(entry, pixel) weights and dL/dpower go to a small shared-memory
// table; then each lane takes one entry and sums its gradient (mean 2, conic
// 3, alpha 1, features 3 + C + 1) over the warp's pixels that received
// anything (phase B, lane = entry), and the warp adds each entry's row to the
// per-record gradient buffer with one coalesced atomic per column.
// Warps run independently (no block barrier); a block holds two warps of one
// tile.  For the fused training step the kernel computes dL/dout itself from
// the forward output and the targets (masked L1 + CE), so no gradient image is
// written or read, and leaves one loss partial per warp.
//
// project_bwd_k: one thread per record chains the 2D gradients through the
// conic inverse, Sigma' = T2 T2^T + eps I, T2 = J W M, the perspective
// Jacobian and mean, the quaternion normalisation and M = R[:, :2] diag(s),
// and adds the per-surfel results (several views touch one surfel) with
// atomics (one vector reduction for a quaternion row and one for a scale
// row); then each warp walks its 32 records with lane = colour/semantic
// column, so the feature gradients leave as coalesced atomics.  Every row is
// cleared after it is read, so the buffer is all zero again for the next
// backward.
#include "kernels.h"

namespace rogs {

int grad_channels(int C) { return padded_channels(C) <= 24 ? 32 : 64; }

constexpr int kSubPad = 33;   // padded row stride of the per-warp tables
// an entry's gradient row (mean 2, conic 3, alpha 1, 3 + C + 1 features) is
// written over its two table rows in phase B
static_assert(2 * kSubPad >= 6 + 3 + ROGS_MAX_CLASSES + 1, "a gradient row must fit the two table rows");
constexpr int kBwdWarpsPerBlock = 2;

// List entries per chunk, and the resident two-warp blocks per SM the kernel
// is compiled for.  Up to 24 channels a chunk of 24 entries keeps a warp's
// shared memory (10.3 KB) and registers (at most 102) small enough for 10 blocks, 20
// warps, per SM (16 with 32-entry chunks); dL/dout is reloaded from its
// shared-memory row after phase B, so it is not live through it.  Measured:
// 32-entry chunks at 16 warps 0.480 ms, 24 at 20 warps 0.478 ms, 16 at 24
// warps 0.553 ms (twice the chunks).
template <int NCP>
__host__ __device__ constexpr int bwd_chunk() { return NCP <= 24 ? 24 : 32; }
template <int NCP>
__host__ __device__ constexpr int bwd_min_blocks() { return NCP <= 24 ? 10 : 1; }

template <int NCP>
__host__ __device__ constexpr int bwd_warp_floats() {
    constexpr int KC = bwd_chunk<NCP>();
    return KC * 4 + KC * 4 + 32 * NCP + KC + 2 * KC * kSubPad;   // s_m, s_c, s_f | s_G, s_rec, tables
}

// The loss gradient at one pixel for the fused training step (Eqs. 8, 9, 12),
// computed in place from the pixel's forward output channels G (loaded by
// the caller together with the targets, in one memory round trip):
//   dL/dc'  = lambda_c / |M| sign(c' - cbar)          (masked L1, three channels)
//   dL/dsem = lambda_s / |M| (softmax(sem) - onehot)   (masked cross entropy)
// (the depth channel carries no loss).  Returns the pixel's unnormalised loss
// term lambda_c |c' - cbar|_1 + lambda_s CE.
template <int NCP>
__device__ __forceinline__ float pixel_loss_grad(const BwdArgs& a, int C, bool in_mask, unsigned long long nm, int lb,
                                                 float t0, float t1, float t2, float (&G)[NCP]) {
    if (!in_mask || nm == 0) {
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch) G[ch] = 0.0f;
        return 0.0f;
    }
    const float inv = 1.0f / (float)nm;
    const float tr[3] = {t0, t1, t2};
    float l1 = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float d = G[ch] - tr[ch];
        l1 += fabsf(d);
        G[ch] = a.lambda_c * inv * (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f));
    }
    float ce = 0.0f;
    if (lb >= 0 && lb < C) {
        float mx = -3.0e38f;
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch)
            if (ch >= 3 && ch < 3 + C) mx = fmaxf(mx, G[ch]);
        // softmax with one exponential per class: e = exp(x - max), p = e / sum e
        float se = 0.0f, xl = 0.0f;
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch)
            if (ch >= 3 && ch < 3 + C) {
                if ((ch - 3) == lb) xl = G[ch];
                G[ch] = __expf(G[ch] - mx);
                se += G[ch];
            }
        const float rse = 1.0f / se;
        const float ls = a.lambda_s * inv;
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch)
            if (ch >= 3 && ch < 3 + C) G[ch] = ls * (G[ch] * rse - ((ch - 3) == lb ? 1.0f : 0.0f));
        ce = mx + logf(se) - xl;
    } else {
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch)
            if (ch >= 3 && ch < 3 + C) G[ch] = 0.0f;
    }
#pragma unroll
    for (int ch = 0; ch < NCP; ++ch)
        if (ch >= 3 + C) G[ch] = 0.0f;   // depth and padding
    return a.lambda_c * l1 + a.lambda_s * ce;
}

// 16-byte vector reduction (add) into global memory; the address is 16-byte aligned.
__device__ __forceinline__ void red_add_v4(float* p, float x, float y, float z, float w) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w)
                 : "memory");
}
// 8-byte vector reduction (add); the address is 8-byte aligned.
__device__ __forceinline__ void red_add_v2(float* p, float x, float y) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x), "f"(y) : "memory");
}

template <int TW, int TH, int NCP, int GP>
__global__ void __launch_bounds__(32 * kBwdWarpsPerBlock, bwd_min_blocks<NCP>()) composite_bwd_k(BwdArgs a) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    constexpr int BW = block_w(TW, TH), BH = 32 / BW, WX = TW / BW;
    constexpr int NW = TW * TH / 32;
    constexpr int GROUPS = NW / kBwdWarpsPerBlock;
    constexpr int SP = kSubPad;
    constexpr int KC = bwd_chunk<NCP>();
    constexpr uint32_t KCu = (uint32_t)KC;
    static_assert(bwd_warp_floats<NCP>() % 4 == 0, "16-byte aligned warp regions");
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const long long tile = a.tile_order[blockIdx.x / GROUPS];
    const int warp = (int)(blockIdx.x % GROUPS) * kBwdWarpsPerBlock + wib;   // warp index inside the tile
    extern __shared__ float4 smem_bwd[];
    float* wbase = reinterpret_cast<float*>(smem_bwd) + wib * bwd_warp_floats<NCP>();
    float4* s_m = reinterpret_cast<float4*>(wbase);
    float4* s_c = s_m + KC;
    float* s_f = reinterpret_cast<float*>(s_c + KC);   // KC feature rows, or 32 dL/dout rows (s_G)
    uint32_t* s_rec = reinterpret_cast<uint32_t*>(s_f + 32 * NCP);
    float* s_w = reinterpret_cast<float*>(s_rec + KC);
    float* s_p = s_w + KC * SP;
    float* s_G = s_f;   // dL/dout rows per pixel, written over the features once phase A is done

    const Consts& k = a.k;
    const SurfelPtrs& sp = a.sp;
    const int vi = view_of_tile(a.views, a.n_views, tile);
    const ViewParams& v = a.views[vi];
    const int W = v.W, H = v.H;
    const long long lt = tile - v.tile_base;
    const int tx = (int)(lt % v.tiles_x), ty = (int)(lt / v.tiles_x);
    const int bx = tx * TW + (warp % WX) * BW, by = ty * TH + (warp / WX) * BH;
    const int px = bx + lane % BW, py = by + lane / BW;
    const bool inside = px < W && py < H;
    const int2 org = offset_origin(bx, by);   // the same for every pixel of the block
    const float lx = (float)(px - org.x), ly = (float)(py - org.y);
    const uint2 trange = a.ranges[tile];
    const uint32_t start = trange.x;
    const int C = k.C;
    const int nch = 3 + C + 1;
    const float amin = k.alpha_min, amax = k.alpha_max;
    const float ea = expf(a.exposure_ab[2 * v.exp_idx]);
    const unsigned lt_mask = lanemask_lt();

    // A tile no surfel reaches (sky, say) passes no gradient to any surfel;
    // with the fused loss its pixels only count if they are in the mask, so a
    // warp there reads the mask first and, if none of its pixels is in it,
    // leaves a zero loss partial without loading anything else.
    const bool fused = a.tg.rgb != nullptr || a.tg.rgb8 != nullptr;
    if (fused && trange.y <= trange.x) {
        const bool m = inside && a.tg.mask[v.pix_base + (long long)py * W + px] != 0;
        if (!__any_sync(kFull, m)) {
            if (a.loss_partials && lane == 0) a.loss_partials[blockIdx.x * kBwdWarpsPerBlock + wib] = 0.0f;
            return;
        }
    }
    // Every input of this lane's pixel is loaded at once, one memory round trip:
    // the forward's transmittance and last contributor, and either dL/dout or
    // (fused loss) the output channels, the targets and the mask
    float T = 1.0f;
    uint32_t last = 0;
    float G[NCP];
    float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f;
    int lb = -1;
    bool in_mask = false;
    if (inside) {
        const long long q = (long long)py * W + px;
        const long long pix = v.pix_base + q;
        const long long plane = (long long)W * H;
        T = a.pix_T[pix];
        last = a.pix_last[pix];
        const float* src = (fused ? a.out : a.grad_out) + (long long)nch * v.pix_base + q;
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch) G[ch] = ch < nch ? src[ch * plane] : 0.0f;
        if (fused) {
            load_pixel_target(a.tg, 3ll * v.pix_base + q, plane, pix, C, t0, t1, t2, lb);
            in_mask = a.tg.mask[pix] != 0;
        }
    } else {
#pragma unroll
        for (int ch = 0; ch < NCP; ++ch) G[ch] = 0.0f;
    }
    const unsigned long long nm = fused ? *a.mask_count : 0ull;
    const uint32_t wmax = __reduce_max_sync(kFull, last);
    // The first chunk (the last 32 list entries up to wmax) is compacted and
    // staged before the loss gradient is computed: its block masks, records and
    // mean/conic are loaded now, and its feature rows are copied into shared
    // memory asynchronously while the loss gradient runs.
    unsigned mask_first = 0;
    {
        const uint32_t cbeg = wmax > KCu ? wmax - KCu : 0u;
        const uint32_t j = cbeg + lane;
        bool hit = false;
        uint32_t rec = 0;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f), c = m;
        if (lane < KC && j < wmax && rogs_ok(start + j < k.pair_cap, 201u)) {
            // records and mean/conic loaded with the block masks (one round trip)
            const uint32_t bm = a.pair_blk[start + j];
            const uint32_t r = a.pair_rec[start + j];
            const float4 m0 = a.pair_mc[2ull * (start + j)], c0 = a.pair_mc[2ull * (start + j) + 1];
            hit = (bm >> warp) & 1u;
            if (hit) {
                rec = r;
                hit = rogs_ok(rec < k.rec_cap, 202u);
                if (hit) {
                    m = m0;
                    c = c0;
                }
            }
        }
        mask_first = __ballot_sync(kFull, hit);
        if (hit) {
            const int slot = __popc(mask_first & lt_mask);
            s_m[slot] = block_offsets(m, org);
            s_c[slot] = c;
            s_rec[slot] = rec;
            stage_record_features_async<NCP>(s_f + slot * NCP, a.feat, rec);
        }
        cp_async_commit();
    }
    float lpix = 0.0f;
    float gsum_rgb = 0.0f;
    if (inside) {
        if (fused) lpix = pixel_loss_grad<NCP>(a, C, in_mask, nm, lb, t0, t1, t2, G);
        gsum_rgb = G[0] + G[1] + G[2];
        G[0] *= ea; G[1] *= ea; G[2] *= ea;   // through c' = e^a c + b
    }
    if (a.loss_partials) {   // fused loss: one partial per warp, summed in a fixed order later
        float l = lpix;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(kFull, l, o);
        if (lane == 0) a.loss_partials[blockIdx.x * kBwdWarpsPerBlock + wib] = l;
    }
    cp_async_wait_all();
    __syncwarp();

    float Ssum = 0.0f;                          // sum_{j>k} w_j (G . f_j)
    float cr0 = 0.0f, cr1 = 0.0f, cr2 = 0.0f;   // raw rgb, for dL/da of Eq. 7

    // block masks of the chunk after the current one are loaded one chunk ahead
    uint32_t bm_next = 0;
    {
        const uint32_t cb = wmax > KCu ? wmax - KCu : 0u;   // the second chunk is [cb - KC, cb)
        const uint32_t j = (cb > KCu ? cb - KCu : 0u) + lane;
        if (lane < KC && j < cb) bm_next = a.pair_blk[start + j];
    }
    for (uint32_t cend = wmax; cend > 0;) {
        const uint32_t cbeg = cend > KCu ? cend - KCu : 0u;
        unsigned mask;
        if (cend == wmax) {
            mask = mask_first;   // staged before the loss gradient
        } else {
            const uint32_t j = cbeg + lane;   // index in the tile list
            const uint32_t bm = bm_next;
            {
                const uint32_t jn = (cbeg > KCu ? cbeg - KCu : 0u) + lane;
                bm_next = lane < KC && jn < cbeg ? a.pair_blk[start + jn] : 0u;
            }
            bool hit = false;
            uint32_t rec = 0;
            float4 m = make_float4(0.f, 0.f, 0.f, 0.f), c = m;
            if (lane < KC && j < cend) {   // the block mask says whether the entry can reach this warp's block
                hit = (bm >> warp) & 1u && rogs_ok(start + j < k.pair_cap, 203u);
                if (hit) {
                    rec = a.pair_rec[start + j];
                    hit = rogs_ok(rec < k.rec_cap, 204u);
                    if (hit) {
                        m = a.pair_mc[2ull * (start + j)];
                        c = a.pair_mc[2ull * (start + j) + 1];
                    }
                }
            }
            mask = __ballot_sync(kFull, hit);
            if (hit) {
                const int slot = __popc(mask & lt_mask);
                s_m[slot] = block_offsets(m, org);
                s_c[slot] = c;
                s_rec[slot] = rec;
                stage_record_features<NCP>(s_f + slot * NCP, a.feat, rec);
            }
            __syncwarp();
        }
        cend = cbeg;
        if (!mask) continue;
        const int h = __popc(mask);
        // phase A (lane = pixel): reverse recursion over the compacted entries.
        // Branch-free: a lane whose entry does not count uses 1 / (1 - a) = 1 and
        // w = 0, which leaves T and S unchanged, so iterations can overlap.
        unsigned pmask = 0;
        // entries this pixel composited: list index < last, a prefix of the compacted slots
        const int rel = (int)last - (int)cbeg;
        const int kmax = rel <= 0 ? 0 : __popc(rel >= 32 ? mask : (mask & ((1u << rel) - 1u)));
#pragma unroll 2
        for (int jj = h - 1; jj >= 0; --jj) {
            const float4 mm = s_m[jj];
            const float4 cc = s_c[jj];
            const float dx = __fadd_rn(mm.x, lx);
            const float dy = __fadd_rn(mm.y, ly);
            float g;
            const float al = surfel_alpha(dx, dy, cc.x, cc.y, cc.z, cc.w, amax, g);
            const bool valid = jj < kmax && al >= amin;
            // 1 / (1 - alpha) off the loop-carried chain: only a multiply links T_k to T_{k+1}
            // (1 - alpha >= 0.01, so the fast reciprocal is within 2 ulp)
            const float roma = valid ? __fdividef(1.0f, __fsub_rn(1.0f, al)) : 1.0f;
            T = T * roma;   // T_k
            const float w = valid ? al * T : 0.0f;
            const float4* f4 = reinterpret_cast<const float4*>(s_f + jj * NCP);
            float D0 = 0.0f, D1 = 0.0f, D2 = 0.0f, D3 = 0.0f;   // four short chains
#pragma unroll
            for (int q = 0; q < NCP / 4; ++q) {
                const float4 f = f4[q];
                D0 = fmaf(G[4 * q], f.x, D0);
                D1 = fmaf(G[4 * q + 1], f.y, D1);
                D2 = fmaf(G[4 * q + 2], f.z, D2);
                D3 = fmaf(G[4 * q + 3], f.w, D3);
            }
            const float D = (D0 + D1) + (D2 + D3);
            const float da = fmaf(T, D, -Ssum * roma);
            Ssum = fmaf(w, D, Ssum);
            const float4 f0 = f4[0];
            cr0 = fmaf(w, f0.x, cr0);
            cr1 = fmaf(w, f0.y, cr1);
            cr2 = fmaf(w, f0.z, cr2);
            const float ag = cc.w * g;
            const float dpw = (valid && ag < amax) ? da * ag : 0.0f;   // d alpha = dpw / alpha
            s_w[jj * SP + lane] = w;
            s_p[jj * SP + lane] = dpw;
            pmask |= __ballot_sync(kFull, w != 0.0f);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NCP / 4; ++q)   // row per pixel: phase B reads it as broadcast float4s
            reinterpret_cast<float4*>(s_G + lane * NCP)[q] = make_float4(G[4 * q], G[4 * q + 1], G[4 * q + 2], G[4 * q + 3]);
        __syncwarp();
        // phase B (lane = entry): sum the entry's gradient over the pixels that got
        // anything, two pixels per step and without branches (w = 0 adds nothing).
        // With h <= 16 (8) entries the warp splits into 2 (4) groups of E lanes,
        // group g taking the g-th quarter or half of the pixels, and the groups'
        // sums are added with shuffles: fewer pixel steps for short chunks.
        bool any = false;
        {
            const int E = h <= 8 ? 8 : (h <= 16 ? 16 : 32);   // lanes per group (h is warp-uniform)
            const int e = lane & (E - 1), grp = lane / E;
            const bool act = e < h;
            const unsigned gmask = E == 32 ? kFull : (((1u << E) - 1u) << (grp * E));
            float acc[NCP];
#pragma unroll
            for (int ch = 0; ch < NCP; ++ch) acc[ch] = 0.0f;
            // The conic and mean gradients need sums over the pixels of dp times
            // (1, dx, dy, dx^2, dx dy, dy^2), with (dx, dy) the pixel's offset
            // from the mean.  Written as (dxc + ux, dyc + uy), with (ux, uy) the
            // pixel's offset from the block centre (a half-integer constant per
            // pixel) and (dxc, dyc) the centre's offset from the mean, they
            // follow from six moments of dp over (ux, uy), expanded once per
            // entry after the loop.
            constexpr float hx = 0.5f * (float)(BW - 1), hy = 0.5f * (float)(BH - 1);
            float m0 = 0.0f, mx = 0.0f, my = 0.0f, mxx = 0.0f, mxy = 0.0f, myy = 0.0f;
            if (act) {
                for (unsigned q = pmask & gmask; q;) {
                    const int p1 = __ffs(q) - 1;
                    q &= q - 1;
                    const int p2 = q ? __ffs(q) - 1 : p1;
                    const float w1 = s_w[e * SP + p1];
                    const float w2 = q ? s_w[e * SP + p2] : 0.0f;
                    const float dp1 = s_p[e * SP + p1];
                    const float dp2 = q ? s_p[e * SP + p2] : 0.0f;
                    q &= q - 1;
                    any |= (w1 != 0.0f) | (w2 != 0.0f);
                    const float4* r1 = reinterpret_cast<const float4*>(s_G + p1 * NCP);
                    const float4* r2 = reinterpret_cast<const float4*>(s_G + p2 * NCP);
#pragma unroll
                    for (int k4 = 0; k4 < NCP / 4; ++k4) {
                        const float4 a1 = r1[k4], a2 = r2[k4];
                        acc[4 * k4] = fmaf(w2, a2.x, fmaf(w1, a1.x, acc[4 * k4]));
                        acc[4 * k4 + 1] = fmaf(w2, a2.y, fmaf(w1, a1.y, acc[4 * k4 + 1]));
                        acc[4 * k4 + 2] = fmaf(w2, a2.z, fmaf(w1, a1.z, acc[4 * k4 + 2]));
                        acc[4 * k4 + 3] = fmaf(w2, a2.w, fmaf(w1, a1.w, acc[4 * k4 + 3]));
                    }
                    const float ux1 = (float)(p1 % BW) - hx, uy1 = (float)(p1 / BW) - hy;
                    const float ux2 = (float)(p2 % BW) - hx, uy2 = (float)(p2 / BW) - hy;
                    m0 += dp1 + dp2;
                    mx = fmaf(dp1, ux1, fmaf(dp2, ux2, mx));
                    my = fmaf(dp1, uy1, fmaf(dp2, uy2, my));
                    const float ex1 = dp1 * ux1, ex2 = dp2 * ux2;
                    mxx = fmaf(ex1, ux1, fmaf(ex2, ux2, mxx));
                    mxy = fmaf(ex1, uy1, fmaf(ex2, uy2, mxy));
                    myy = fmaf(dp1 * uy1, uy1, fmaf(dp2 * uy2, uy2, myy));
                }
            }
            for (int o = E; o < 32; o <<= 1) {   // add the groups' sums (all lanes)
#pragma unroll
                for (int ch = 0; ch < NCP; ++ch) acc[ch] += __shfl_xor_sync(kFull, acc[ch], o);
                m0 += __shfl_xor_sync(kFull, m0, o);
                mx += __shfl_xor_sync(kFull, mx, o);
                my += __shfl_xor_sync(kFull, my, o);
                mxx += __shfl_xor_sync(kFull, mxx, o);
                mxy += __shfl_xor_sync(kFull, mxy, o);
                myy += __shfl_xor_sync(kFull, myy, o);
                any = __shfl_xor_sync(kFull, (int)any, o) != 0 || any;
            }
            any = any && act && grp == 0;
            if (any) {   // the entry's row of the tables becomes its gradient row
                const float4 mm = s_m[e];   // offsets of pixel org's centre from the mean
                const float4 cc = conic_from_exp2(s_c[e]);   // (A, B, C, alpha)
                const float dx0 = mm.x + (float)(bx - org.x), dy0 = mm.y + (float)(by - org.y);   // block's first pixel
                const float dxc = dx0 + hx, dyc = dy0 + hy;
                const float sx = fmaf(dxc, m0, mx), sy = fmaf(dyc, m0, my);   // sum dp dx, sum dp dy
                const float sxx = fmaf(dxc, fmaf(dxc, m0, 2.0f * mx), mxx);     // sum dp dx^2
                const float sxy = fmaf(dxc, fmaf(dyc, m0, my), fmaf(dyc, mx, mxy));   // sum dp dx dy
                const float syy = fmaf(dyc, fmaf(dyc, m0, 2.0f * my), myy);     // sum dp dy^2
                float* r0 = s_w + e * SP;
                float* r1 = s_p + e * SP;
                r0[0] = fmaf(cc.x, sx, cc.y * sy);
                r0[1] = fmaf(cc.y, sx, cc.z * sy);
                r0[2] = -0.5f * sxx;
                r0[3] = -sxy;
                r0[4] = -0.5f * syy;
                r0[5] = m0 / cc.w;
                // the padded channels are zero and never flushed; the widest rows
                // (6 + 64 > 2 * SP) keep only the real ones, the others write all
#pragma unroll
                for (int ch = 0; ch < NCP; ++ch) {
                    const int col = 6 + ch;
                    if (6 + NCP > 2 * SP && ch >= nch) break;
                    if (col < SP) r0[col] = acc[ch];
                    else r1[col - SP] = acc[ch];
                }
            }
        }
        const unsigned anym = __ballot_sync(kFull, any);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NCP / 4; ++q) {   // dL/dout back from its row: not live through phase B
            const float4 g4 = reinterpret_cast<const float4*>(s_G + lane * NCP)[q];
            G[4 * q] = g4.x; G[4 * q + 1] = g4.y; G[4 * q + 2] = g4.z; G[4 * q + 3] = g4.w;
        }
        // flush: each gradient row that received anything is added into the
        // record's row with 16-byte vector reductions, GP/4 lanes per row and
        // 128/GP rows per instruction (columns past 6 + nch add zeros)
        {
            constexpr int QPR = GP / 4;       // 16-byte pieces per row
            constexpr int RPI = 32 / QPR;     // rows per instruction
            const int ncol = 6 + nch;
            const int sub = lane / QPR, col0 = 4 * (lane % QPR);
            for (unsigned q = anym; q;) {
                int e = -1;
#pragma unroll
                for (int r = 0; r < RPI; ++r) {
                    if (!q) break;
                    const int bit = __ffs(q) - 1;
                    q &= q - 1;
                    if (r == sub) e = bit;
                }
                if (e >= 0 && col0 < ncol) {
                    float x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int col = col0 + u;
                        x[u] = col < ncol ? (col < SP ? s_w[e * SP + col] : s_p[e * SP + col - SP]) : 0.0f;
                    }
                    if (x[0] != 0.0f || x[1] != 0.0f || x[2] != 0.0f || x[3] != 0.0f)
                        red_add_v4(a.rec_grad + (unsigned long long)s_rec[e] * GP + col0, x[0], x[1], x[2], x[3]);
                }
            }
        }
        __syncwarp();
    }

    // exposure (Eq. 7): dL/db = sum g', dL/da = sum g' e^a c_raw
    float e_a = 0.0f, e_b = 0.0f;
    if (inside) {
        e_b = gsum_rgb;
        e_a = G[0] * cr0 + G[1] * cr1 + G[2] * cr2;   // G[0..2] hold e^a g'
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_a += __shfl_xor_sync(kFull, e_a, o);
        e_b += __shfl_xor_sync(kFull, e_b, o);
    }
    if (lane == 0 && a.d_exposure) {
        if (e_a != 0.0f) atomicAdd(&a.d_exposure[2 * v.exp_idx], e_a);
        if (e_b != 0.0f) atomicAdd(&a.d_exposure[2 * v.exp_idx + 1], e_b);
    }
}

template <int NCP>
static size_t bwd_smem_bytes() {
    return (size_t)kBwdWarpsPerBlock * 4 * (size_t)bwd_warp_floats<NCP>();
}

int bwd_loss_partials(long long total_tiles, int tile_w, int tile_h) {
    return (int)(total_tiles * (tile_w * tile_h / 32));
}

template <int TW, int TH, int NCP, int GP>
static void bwd_attr() {
    static unsigned long long done_mask = 0;   // one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !((done_mask >> dev) & 1ull)) {
        cudaFuncSetAttribute(composite_bwd_k<TW, TH, NCP, GP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bwd_smem_bytes<NCP>());
        done_mask |= 1ull << dev;
    }
}

template <int TW, int TH>
static void prepare_bwd_tile() {
    bwd_attr<TW, TH, 8, 32>(); bwd_attr<TW, TH, 16, 32>();
    bwd_attr<TW, TH, 24, 32>(); bwd_attr<TW, TH, 32, 64>(); bwd_attr<TW, TH, 64, 64>();
}

void prepare_composite_bwd() {
    prepare_bwd_tile<16, 16>();
    prepare_bwd_tile<32, 8>();
    prepare_bwd_tile<8, 8>();
}

template <int TW, int TH>
static void launch_bwd_tile(int ncp, long long total_tiles, const BwdArgs& a, cudaStream_t s) {
    constexpr int groups = TW * TH / 32 / kBwdWarpsPerBlock;
    dim3 grid((unsigned)(total_tiles * groups));
#define ROGS_BWD(NCP, GP)                                                                           \
    do {                                                                                            \
        bwd_attr<TW, TH, NCP, GP>();                                                                \
        launch_pdl(composite_bwd_k<TW, TH, NCP, GP>, dim3(grid), dim3(32 * kBwdWarpsPerBlock), bwd_smem_bytes<NCP>(), s, a); \
        note_launches(1);                                                                           \
    } while (0)
    switch (ncp) {
        case 8: ROGS_BWD(8, 32); break;
        case 16: ROGS_BWD(16, 32); break;
        case 24: ROGS_BWD(24, 32); break;
        case 32: ROGS_BWD(32, 64); break;
        default: ROGS_BWD(64, 64); break;
    }
#undef ROGS_BWD
}

void composite_bwd(int tile_w, int tile_h, long long total_tiles, const BwdArgs& a, cudaStream_t s) {
    const int ncp = padded_channels(a.k.C);
    if (tile_w == 32 && tile_h == 8) launch_bwd_tile<32, 8>(ncp, total_tiles, a, s);
    else if (tile_w == 8 && tile_h == 8) launch_bwd_tile<8, 8>(ncp, total_tiles, a, s);
    else launch_bwd_tile<16, 16>(ncp, total_tiles, a, s);
}

// ----------------------------------------------------------- project_bwd

// Geometry part of one record's backward (row cols 0-5 and the depth column).
__device__ __forceinline__ void project_bwd_record(const ViewParams* __restrict__ views, const SurfelPtrs& sp,
                                                   const Record* __restrict__ recs, float* __restrict__ gr, int dcol,
                                                   const GradPtrs& gp, unsigned long long r) {
    const float4 ga = *reinterpret_cast<const float4*>(gr);
    const float2 gb = *reinterpret_cast<const float2*>(gr + 4);
    const float dz_feat = gr[dcol];   // depth-channel gradient
    const float g6[6] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y};
    const bool any = ga.x != 0.0f || ga.y != 0.0f || ga.z != 0.0f || ga.w != 0.0f || gb.x != 0.0f || gb.y != 0.0f ||
                     dz_feat != 0.0f;
    if (!any) return;
    *reinterpret_cast<float4*>(gr) = make_float4(0.f, 0.f, 0.f, 0.f);   // leave the row zero for the next backward
    *reinterpret_cast<float2*>(gr + 4) = make_float2(0.f, 0.f);
    gr[dcol] = 0.0f;
    const Record rec = recs[r];
    const uint32_t i = rec.surfel;
    if (!rogs_ok(i < sp.n, 205u)) return;
        if (gp.opacity && g6[5] != 0.0f) atomicAdd(&gp.opacity[i], g6[5]);

        const ViewParams& v = views[rec.view];
        // recompute the forward quantities in FP32
        const float x = sp.xyz[3ull * i], y = sp.xyz[3ull * i + 1], z = sp.xyz[3ull * i + 2];
        float p[3];
        for (int rr = 0; rr < 3; ++rr) {
            df a = two_prod(v.R[3 * rr], x);
            a = df_add(a, two_prod(v.R[3 * rr + 1], y));
            a = df_add(a, two_prod(v.R[3 * rr + 2], z));
            a = df_add_f(a, v.t[rr]);
            p[rr] = __fadd_rn(a.hi, a.lo);
        }
        float J00, J02, J11, J12, uc = 0.0f, vc = 0.0f;
        bool clx = false, cly = false;
        const bool persp = v.kind == ROGS_PERSP;
        if (persp) {
            const float inv = 1.0f / p[2];
            const float u = p[0] * inv, vv = p[1] * inv;
            uc = fminf(fmaxf(u, -v.lim_x), v.lim_x);
            vc = fminf(fmaxf(vv, -v.lim_y), v.lim_y);
            clx = uc != u;
            cly = vc != vv;
            J00 = v.fx * inv; J02 = -v.fx * uc * inv; J11 = v.fy * inv; J12 = -v.fy * vc * inv;
        } else {
            J00 = v.fx; J02 = 0.0f; J11 = v.fy; J12 = 0.0f;
        }
        const float4 q4 = reinterpret_cast<const float4*>(sp.quat)[i];
        const float qnorm2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
        const float qinv = rsqrtf(qnorm2);
        const float w = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
        const float2 s = reinterpret_cast<const float2*>(sp.scale)[i];
        // R(q) columns 0, 1
        const float R00 = 1.0f - 2.0f * (qy * qy + qz * qz), R10 = 2.0f * (qx * qy + w * qz), R20 = 2.0f * (qx * qz - w * qy);
        const float R01 = 2.0f * (qx * qy - w * qz), R11 = 1.0f - 2.0f * (qx * qx + qz * qz), R21 = 2.0f * (qy * qz + w * qx);
        const float m0[3] = {R00 * s.x, R10 * s.x, R20 * s.x};
        const float m1[3] = {R01 * s.y, R11 * s.y, R21 * s.y};
        float V0[3], V1[3];
        for (int rr = 0; rr < 3; ++rr) {
            V0[rr] = v.R[3 * rr] * m0[0] + v.R[3 * rr + 1] * m0[1] + v.R[3 * rr + 2] * m0[2];
            V1[rr] = v.R[3 * rr] * m1[0] + v.R[3 * rr + 1] * m1[1] + v.R[3 * rr + 2] * m1[2];
        }
        // T2 = J V (2x2): columns t0 = J V0, t1 = J V1
        const float t00 = J00 * V0[0] + J02 * V0[2], t10 = J11 * V0[1] + J12 * V0[2];
        const float t01 = J00 * V1[0] + J02 * V1[2], t11 = J11 * V1[1] + J12 * V1[2];
        // conic Q (recomputed as in the forward record)
        const float A = rec.ca, B = rec.cb, Cc = rec.cc;
        // dL/dSigma = -Q dQ Q, dQ symmetric with the shared off-diagonal split
        const float q00 = g6[2], q01 = 0.5f * g6[3], q11 = g6[4];
        const float a00 = A * q00 + B * q01, a01 = A * q01 + B * q11;
        const float a10 = B * q00 + Cc * q01, a11 = B * q01 + Cc * q11;
        const float dS00 = -(a00 * A + a01 * B), dS01 = -(a00 * B + a01 * Cc), dS11 = -(a10 * B + a11 * Cc);
        // Sigma = T2 T2^T -> dT2 = 2 dS T2
        const float dT00 = 2.0f * (dS00 * t00 + dS01 * t10), dT01 = 2.0f * (dS00 * t01 + dS01 * t11);
        const float dT10 = 2.0f * (dS01 * t00 + dS11 * t10), dT11 = 2.0f * (dS01 * t01 + dS11 * t11);
        // T2 = J V: dJ = dT2 V^T, dV = J^T dT2
        const float dJ00 = dT00 * V0[0] + dT01 * V1[0];
        const float dJ02 = dT00 * V0[2] + dT01 * V1[2];
        const float dJ11 = dT10 * V0[1] + dT11 * V1[1];
        const float dJ12 = dT10 * V0[2] + dT11 * V1[2];
        float dV0[3], dV1[3];
        dV0[0] = J00 * dT00; dV0[1] = J11 * dT10; dV0[2] = J02 * dT00 + J12 * dT10;
        dV1[0] = J00 * dT01; dV1[1] = J11 * dT11; dV1[2] = J02 * dT01 + J12 * dT11;
        // V = W M -> dM = W^T dV
        float dm0[3], dm1[3];
        for (int cc = 0; cc < 3; ++cc) {
            dm0[cc] = v.R[cc] * dV0[0] + v.R[3 + cc] * dV0[1] + v.R[6 + cc] * dV0[2];
            dm1[cc] = v.R[cc] * dV1[0] + v.R[3 + cc] * dV1[1] + v.R[6 + cc] * dV1[2];
        }
        const float dsx = dm0[0] * R00 + dm0[1] * R10 + dm0[2] * R20;
        const float dsy = dm1[0] * R01 + dm1[1] * R11 + dm1[2] * R21;
        // dR entries (row-major) for columns 0, 1
        const float dR0 = dm0[0] * s.x, dR3 = dm0[1] * s.x, dR6 = dm0[2] * s.x;
        const float dR1 = dm1[0] * s.y, dR4 = dm1[1] * s.y, dR7 = dm1[2] * s.y;
        // derivative of R(q) entries w.r.t. the unit quaternion (columns 0, 1 only)
        const float dw = 2.0f * (qz * dR3 - qy * dR6 - qz * dR1 + qx * dR7);
        const float dx_ = 2.0f * (qy * dR3 + qz * dR6 + qy * dR1 - 2.0f * qx * dR4 + w * dR7);
        const float dy_ = 2.0f * (-2.0f * qy * dR0 + qx * dR3 - w * dR6 + qx * dR1 + qz * dR7);
        const float dz_ = 2.0f * (-2.0f * qz * dR0 + w * dR3 + qx * dR6 - w * dR1 - 2.0f * qz * dR4 + qy * dR7);
        const float dot = w * dw + qx * dx_ + qy * dy_ + qz * dz_;
        const float invn = qinv;
        // position
        float dp0 = 0.0f, dp1 = 0.0f, dp2 = dz_feat;
        if (persp) {
            const float iz = 1.0f / p[2], iz2 = iz * iz;
            dp0 += g6[0] * v.fx * iz;
            dp1 += g6[1] * v.fy * iz;
            dp2 += -g6[0] * v.fx * p[0] * iz2 - g6[1] * v.fy * p[1] * iz2;
            dp2 += dJ00 * (-v.fx * iz2) + dJ11 * (-v.fy * iz2);
            if (!clx) { dp0 += dJ02 * (-v.fx * iz2); dp2 += dJ02 * (2.0f * v.fx * p[0] * iz2 * iz); }
            else { dp2 += dJ02 * (v.fx * uc * iz2); }
            if (!cly) { dp1 += dJ12 * (-v.fy * iz2); dp2 += dJ12 * (2.0f * v.fy * p[1] * iz2 * iz); }
            else { dp2 += dJ12 * (v.fy * vc * iz2); }
        } else {
            dp0 += g6[0] * v.fx;
            dp1 += g6[1] * v.fy;
        }
        if (gp.xyz) {
            for (int cc = 0; cc < 3; ++cc) {
                const float val = v.R[cc] * dp0 + v.R[3 + cc] * dp1 + v.R[6 + cc] * dp2;
                if (val != 0.0f) atomicAdd(&gp.xyz[3ull * i + cc], val);
            }
        }
        // one vector reduction per row where the row is aligned (quaternion
        // rows always are: the call checks 16-byte alignment)
        if (gp.scale && (dsx != 0.0f || dsy != 0.0f)) {
            if (((uintptr_t)gp.scale & 7u) == 0u) {
                red_add_v2(gp.scale + 2ull * i, dsx, dsy);
            } else {
                atomicAdd(&gp.scale[2ull * i], dsx);
                atomicAdd(&gp.scale[2ull * i + 1], dsy);
            }
        }
        if (gp.quat)
            red_add_v4(gp.quat + 4ull * i, (dw - w * dot) * invn, (dx_ - qx * dot) * invn, (dy_ - qy * dot) * invn,
                       (dz_ - qz * dot) * invn);
}

__global__ void __launch_bounds__(256) project_bwd_k(const ViewParams* __restrict__ views, SurfelPtrs sp,
                                                     const Record* __restrict__ recs,
                                                     const StateHeader* __restrict__ hdr, unsigned long long rec_cap,
                                                     float* __restrict__ rec_grad, int C, int GP, GradPtrs gp) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    unsigned long long n = hdr->n_records;
    if (n > rec_cap) n = rec_cap;
    const int lane = threadIdx.x & 31;
    const int nf = 3 + C;                 // feature columns 6 .. 6 + nf - 1 (rgb, semantics)
    const int dcol = 6 + nf;              // depth column
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long base = (blockIdx.x * (unsigned long long)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32ull;
         base < n; base += warps * 32ull) {
        const unsigned long long r = base + lane;
        uint32_t sid = 0;
        if (r < n) {
            sid = recs[r].surfel;
            if (!rogs_ok(sid < sp.n, 206u)) sid = 0;
            project_bwd_record(views, sp, recs, rec_grad + r * (unsigned long long)GP, dcol, gp, r);
        }
        const int cnt = n - base < 32ull ? (int)(n - base) : 32;
        // four records per step, their row loads issued together
        for (int j0 = 0; j0 < cnt; j0 += 4) {
            uint32_t sj4[4];   // surfel ids of the four records (all lanes shuffle)
#pragma unroll
            for (int u = 0; u < 4; ++u) sj4[u] = __shfl_sync(kFull, sid, (j0 + u) & 31);
            for (int c = lane; c < nf; c += 32) {
                float val[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    val[u] = j0 + u < cnt ? rec_grad[(base + j0 + u) * (unsigned long long)GP + 6 + c] : 0.0f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t sj = sj4[u];
                    if (val[u] == 0.0f) continue;
                    rec_grad[(base + j0 + u) * (unsigned long long)GP + 6 + c] = 0.0f;
                    if (c < 3) { if (gp.rgb) atomicAdd(&gp.rgb[3ull * sj + c], val[u]); }
                    else if (gp.sem) atomicAdd(&gp.sem[(unsigned long long)C * sj + (c - 3)], val[u]);
                }
            }
        }
    }
}

void project_bwd(const ViewParams* views, SurfelPtrs sp, const Record* recs, const StateHeader* hdr,
                 unsigned long long rec_cap, float* rec_grad, int C, GradPtrs g, cudaStream_t s) {
    unsigned long long blocks = (rec_cap + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_pdl(project_bwd_k, dim3((int)blocks), dim3(256), 0, s, views, sp, recs, hdr, rec_cap, rec_grad, C, grad_channels(C), g);
    note_launches(1);
}

#ifdef ROGS_CHECKED
unsigned check_word_backward() { return rogs_check_word_take(); }
#endif

}  // namespace rogs
