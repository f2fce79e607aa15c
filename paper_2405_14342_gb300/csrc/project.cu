// project.cu -- stage 1: cull and EWA projection of surfels into views.
//
// RoGs Sec. 3.1 (Eq. 2 with s_z = 0: Sigma = M M^T, M = R[:, :2] diag(s_x, s_y)),
// Sec. 3.3.1 (Eq. 5: Sigma' = J W Sigma W^T J^T; orthographic J = pixel
// scale; the 2D covariance drops the third row and column) and the
// supplementary's perspective box cull.
//
// Three launches, all over surfels with one thread per surfel looping over
// the views:
//   cull_k       visibility bitmask, one 32-bit word per (view, 32 surfels)
//   scan         exclusive scan of the word popcounts, view-major
//   project_k    the records of the visible (view, surfel) pairs, written in
//                (view, surfel) order at their scanned positions, plus the
//                depth sort keys.  A warp first loads, lane = view, the
//                visibility words and first positions of its 32 surfels in
//                up to 32 views, then its surfels' inputs, then projects view
//                by view.
// The projection is evaluated again in project_k rather than carried from
// cull_k; only cull_k's bit decides whether a record exists, so the two
// evaluations never need to agree bit for bit.
#include "kernels.h"
#include "scan.cuh"

namespace rogs {

struct ProjOut {
    df mx, my;
    float depth, key, A, B, C, alpha;
    int tx0, ty0, tx1, ty1;
};

// One surfel's inputs to the projection.  Position and opacity are loaded
// once per surfel for all views; rotation and scales when a view first gets
// past the cheap tests (box, near plane, opacity).
struct SurfelIn {
    float x, y, z, alpha;
    float4 q;
    float2 s;
    bool has_shape;
};

__device__ __forceinline__ SurfelIn load_surfel_pos(const SurfelPtrs& sp, long long i) {
    SurfelIn in;
    in.x = sp.xyz[3 * i];
    in.y = sp.xyz[3 * i + 1];
    in.z = sp.xyz[3 * i + 2];
    in.alpha = sp.opacity[i];
    in.q = make_float4(0.f, 0.f, 0.f, 0.f);
    in.s = make_float2(0.f, 0.f);
    in.has_shape = false;
    return in;
}

__device__ __forceinline__ void load_surfel_shape(const SurfelPtrs& sp, long long i, SurfelIn& in) {
    if (in.has_shape) return;
    in.q = reinterpret_cast<const float4*>(sp.quat)[i];
    in.s = reinterpret_cast<const float2*>(sp.scale)[i];
    in.has_shape = true;
}

__device__ __forceinline__ bool project_surfel(const ViewParams& v, const Consts& k, const SurfelPtrs& sp,
                                               long long i, SurfelIn& in, ProjOut& o) {
    const float x = in.x, y = in.y, z = in.z;
    if (!box_keep(v, k, x, y)) return false;
    const float key = depth_key(v, x, y, z);
    if (v.kind == ROGS_PERSP && !(key > k.near_plane)) return false;
    const float alpha = in.alpha;
    if (!(alpha >= k.alpha_min)) return false;
    load_surfel_shape(sp, i, in);

    // camera-space centre p = R x + t, double-float (exact products)
    df p[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        df a = two_prod(v.R[3 * r], x);
        a = df_add(a, two_prod(v.R[3 * r + 1], y));
        a = df_add(a, two_prod(v.R[3 * r + 2], z));
        p[r] = df_add_f(a, v.t[r]);
    }
    const float px = __fadd_rn(p[0].hi, p[0].lo);
    const float py = __fadd_rn(p[1].hi, p[1].lo);
    const float pz = __fadd_rn(p[2].hi, p[2].lo);
    float J00, J02, J11, J12;
    if (v.kind == ROGS_PERSP) {
        if (!(pz > 0.0f)) return false;
        df ux = df_div(p[0], p[2]);
        df uy = df_div(p[1], p[2]);
        o.mx = df_add_f(df_mul_f(ux, v.fx), v.cx);
        o.my = df_add_f(df_mul_f(uy, v.fy), v.cy);
        const float inv = 1.0f / pz;
        const float uc = fminf(fmaxf(ux.hi, -v.lim_x), v.lim_x);
        const float vc = fminf(fmaxf(uy.hi, -v.lim_y), v.lim_y);
        J00 = v.fx * inv;
        J02 = -v.fx * uc * inv;
        J11 = v.fy * inv;
        J12 = -v.fy * vc * inv;
    } else {
        o.mx = df_add_f(df_mul_f(p[0], v.fx), v.cx);
        o.my = df_add_f(df_mul_f(p[1], v.fy), v.cy);
        J00 = v.fx; J02 = 0.0f; J11 = v.fy; J12 = 0.0f;
    }

    // surfel axes: first two columns of R(q), q normalised
    const float4 q = in.q;
    const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * qi, qx = q.y * qi, qy = q.z * qi, qz = q.w * qi;
    const float2 s = in.s;
    const float c0x = (1.0f - 2.0f * (qy * qy + qz * qz)) * s.x;
    const float c0y = (2.0f * (qx * qy + w * qz)) * s.x;
    const float c0z = (2.0f * (qx * qz - w * qy)) * s.x;
    const float c1x = (2.0f * (qx * qy - w * qz)) * s.y;
    const float c1y = (1.0f - 2.0f * (qx * qx + qz * qz)) * s.y;
    const float c1z = (2.0f * (qy * qz + w * qx)) * s.y;
    // V = W M (camera frame), T2 = J V
    const float v0x = v.R[0] * c0x + v.R[1] * c0y + v.R[2] * c0z;
    const float v0y = v.R[3] * c0x + v.R[4] * c0y + v.R[5] * c0z;
    const float v0z = v.R[6] * c0x + v.R[7] * c0y + v.R[8] * c0z;
    const float v1x = v.R[0] * c1x + v.R[1] * c1y + v.R[2] * c1z;
    const float v1y = v.R[3] * c1x + v.R[4] * c1y + v.R[5] * c1z;
    const float v1z = v.R[6] * c1x + v.R[7] * c1y + v.R[8] * c1z;
    const float t0x = J00 * v0x + J02 * v0z, t0y = J11 * v0y + J12 * v0z;
    const float t1x = J00 * v1x + J02 * v1z, t1y = J11 * v1y + J12 * v1z;
    const float s00 = t0x * t0x + t1x * t1x + k.eps;
    const float s01 = t0x * t0y + t1x * t1y;
    const float s11 = t0y * t0y + t1y * t1y + k.eps;
    const float det = s00 * s11 - s01 * s01;
    if (!(det > 0.0f)) return false;
    const float id = 1.0f / det;
    o.A = s11 * id;
    o.B = -s01 * id;
    o.C = s00 * id;

    // conservative footprint: a >= alpha_min  <=>  d^T Sigma'^-1 d <= 2 ln(alpha / alpha_min)
    const float kappa = 2.0f * logf(alpha / k.alpha_min);
    const float rx = sqrtf(fmaxf(kappa, 0.0f) * s00) * 1.001f + 1e-3f;
    const float ry = sqrtf(fmaxf(kappa, 0.0f) * s11) * 1.001f + 1e-3f;
    const float mxf = o.mx.hi, myf = o.my.hi;
    if (!(fabsf(mxf) < 4.0e6f && fabsf(myf) < 4.0e6f)) return false;
    if (mxf + rx < 0.0f || mxf - rx > (float)v.W || myf + ry < 0.0f || myf - ry > (float)v.H) return false;
    const float fx0 = floorf((mxf - rx - 0.5f) / (float)k.tile_w);
    const float fx1 = floorf((mxf + rx - 0.5f) / (float)k.tile_w);
    const float fy0 = floorf((myf - ry - 0.5f) / (float)k.tile_h);
    const float fy1 = floorf((myf + ry - 0.5f) / (float)k.tile_h);
    o.tx0 = (int)fminf(fmaxf(fx0, 0.0f), (float)(v.tiles_x - 1));
    o.tx1 = (int)fminf(fmaxf(fx1, 0.0f), (float)(v.tiles_x - 1));
    o.ty0 = (int)fminf(fmaxf(fy0, 0.0f), (float)(v.tiles_y - 1));
    o.ty1 = (int)fminf(fmaxf(fy1, 0.0f), (float)(v.tiles_y - 1));
    o.depth = pz;
    o.key = key;
    o.alpha = alpha;
    return true;
}

constexpr int kProjThreads = 256;

__global__ void __launch_bounds__(kProjThreads) cull_k(const ViewParams* __restrict__ views, int n_views, Consts k,
                                                        SurfelPtrs sp, uint32_t* __restrict__ bits, long long n_words) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    extern __shared__ ViewParams sv[];
    load_views_smem(sv, views, n_views);
    const int lane = threadIdx.x & 31;
    const long long warps_total = (long long)gridDim.x * (kProjThreads / 32);
    for (long long w = (long long)blockIdx.x * (kProjThreads / 32) + (threadIdx.x >> 5); w < n_words;
         w += warps_total) {
        const long long i = w * 32 + lane;
        for (int v = 0; v < n_views; ++v) {
            bool vis = false;
            if (i < sp.n) {
                SurfelIn in = load_surfel_pos(sp, i);
                ProjOut o;
                vis = project_surfel(sv[v], k, sp, i, in, o);
            }
            const unsigned b = __ballot_sync(kFull, vis);
            if (lane == 0) bits[(long long)v * n_words + w] = b;
        }
    }
}

__global__ void __launch_bounds__(kProjThreads) project_k(const ViewParams* __restrict__ views, int n_views, Consts k,
                                                           SurfelPtrs sp, const uint32_t* __restrict__ bits,
                                                           const uint32_t* __restrict__ word_off, long long n_words,
                                                           Record* __restrict__ recs, uint2* __restrict__ rects,
                                                           float* __restrict__ feat, int ncp,
                                                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                           unsigned long long rec_cap) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    extern __shared__ ViewParams sv[];
    load_views_smem(sv, views, n_views);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int C = k.C;
    const long long warps_total = (long long)gridDim.x * (kProjThreads / 32);
    for (long long w = (long long)blockIdx.x * (kProjThreads / 32) + wib; w < n_words; w += warps_total) {
        const long long i = w * 32 + lane;
        SurfelIn in{};
        bool loaded = false;
        for (int g = 0; g < n_views; g += 32) {
            // lane = view: the visibility word and first record position of (view, w)
            const int lv = g + lane;
            const long long qv = (long long)lv * n_words + w;
            const uint32_t bw = lv < n_views ? bits[qv] : 0u;
            const uint32_t ow = bw ? word_off[qv] : 0u;
            const unsigned anyv = __ballot_sync(kFull, bw != 0u);
            if (!anyv) continue;
            bool mine = false;   // some view of this group sees this lane's surfel
            for (unsigned m = anyv; m; m &= m - 1) mine |= (__shfl_sync(kFull, bw, __ffs(m) - 1) >> lane) & 1u;
            if (mine && !loaded) {   // the surfel's inputs, once for all its views
                in = load_surfel_pos(sp, i);
                load_surfel_shape(sp, i, in);
                loaded = true;
            }
            for (unsigned m = anyv; m; m &= m - 1) {
                const int vv = __ffs(m) - 1;
                const int v = g + vv;
                const uint32_t b = __shfl_sync(kFull, bw, vv);
                const uint32_t first = __shfl_sync(kFull, ow, vv);
                const bool vis = (b >> lane) & 1u;
                const uint32_t slot = __popc(b & lt);
                const unsigned long long pos = (unsigned long long)first + slot;
                if (vis && pos < rec_cap) {
                    ProjOut o;
                    o.tx0 = o.ty0 = 1;
                    o.tx1 = o.ty1 = 0;
                    if (!project_surfel(sv[v], k, sp, i, in, o)) {
                        // cannot happen with identical arithmetic; keep the record inert
                        o.tx0 = o.ty0 = 1;
                        o.tx1 = o.ty1 = 0;
                    }
                    Record r;
                    float mi = floorf(o.mx.hi), ni = floorf(o.my.hi);
                    float mf = __fadd_rn(__fsub_rn(o.mx.hi, mi), o.mx.lo);
                    float nf = __fadd_rn(__fsub_rn(o.my.hi, ni), o.my.lo);
                    if (mf < 0.0f) { mi -= 1.0f; mf += 1.0f; } else if (mf >= 1.0f) { mi += 1.0f; mf -= 1.0f; }
                    if (nf < 0.0f) { ni -= 1.0f; nf += 1.0f; } else if (nf >= 1.0f) { ni += 1.0f; nf -= 1.0f; }
                    r.mxi = mi; r.myi = ni; r.mxf = mf; r.myf = nf;
                    r.ca = o.A; r.cb = o.B; r.cc = o.C; r.opacity = o.alpha;
                    r.depth = o.depth; r.key = o.key;
                    r.surfel = (uint32_t)i;
                    r.view = (uint32_t)v;
                    float4* dst = reinterpret_cast<float4*>(recs + pos);
                    const float4* src = reinterpret_cast<const float4*>(&r);
                    dst[0] = src[0];
                    dst[1] = src[1];
                    dst[2] = src[2];
                    uint2 rc;
                    if (o.tx1 >= o.tx0 && o.ty1 >= o.ty0) {
                        rc.x = (uint32_t)o.tx0 | ((uint32_t)o.ty0 << 16);
                        rc.y = (uint32_t)o.tx1 | ((uint32_t)o.ty1 << 16);
                    } else {
                        rc.x = 1u | (1u << 16);  // empty: x1 < x0
                        rc.y = 0u;
                    }
                    rects[pos] = rc;
                    keys[pos] = float_sort_bits(o.key);
                    vals[pos] = (uint32_t)pos;
                    // feature row: rgb, the C logits, depth, zeros
                    const float* rgb = sp.rgb + 3ull * (unsigned long long)i;
                    const float* sem = sp.sem + (unsigned long long)C * (unsigned long long)i;
                    float4* fr = reinterpret_cast<float4*>(feat + pos * (unsigned long long)ncp);
                    for (int q4 = 0; q4 < ncp / 4; ++q4) {
                        float e[4];
#pragma unroll
                        for (int c4 = 0; c4 < 4; ++c4) {
                            const int ch = 4 * q4 + c4;
                            e[c4] = ch < 3 ? rgb[ch] : (ch - 3 < C ? sem[ch - 3] : (ch - 3 == C ? o.depth : 0.0f));
                        }
                        fr[q4] = make_float4(e[0], e[1], e[2], e[3]);
                    }
                }
            }
        }
    }
}

__global__ void upload_views_k(ViewsArg va, int n_views, ViewParams* dst, StateHeader* hdr) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    const int words = n_views * (int)(sizeof(ViewParams) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(va.v);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int t = threadIdx.x; t < words; t += blockDim.x) d[t] = src[t];
    if (threadIdx.x == 0 && hdr) {
        hdr->n_records = hdr->n_pairs = hdr->need_records = hdr->need_pairs = hdr->composited = 0ull;
        hdr->status = 0u;
        hdr->n_views = (unsigned)n_views;
    }
}

void upload_views(const ViewsArg& va, int n_views, ViewParams* dst, StateHeader* hdr, cudaStream_t s) {
    launch_pdl(upload_views_k, dim3(1), dim3(256), 0, s, va, n_views, dst, hdr);
    note_launches(1);
}

static int grid_for_words(long long n_words) {
    long long blocks = (n_words + (kProjThreads / 32) - 1) / (kProjThreads / 32);
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    return (int)blocks;
}

void cull_views(const ViewParams* views, int n_views, Consts k, SurfelPtrs sp, uint32_t* bits, long long n_words,
                cudaStream_t s) {
    size_t sm = sizeof(ViewParams) * (size_t)n_views;
    launch_pdl(cull_k, dim3(grid_for_words(n_words)), dim3(kProjThreads), sm, s, views, n_views, k, sp, bits, n_words);
    note_launches(1);
}

struct PopcF {
    const uint32_t* bits;
    __device__ uint32_t operator()(unsigned long long i) const { return (uint32_t)__popc(bits[i]); }
};

size_t scan_tile_sums_words(unsigned long long cap) { return (size_t)scan_tiles_for(cap) * 2 + 2; }

// The scan's one-block pass also leaves the record count: need_records, the
// count clamped to the capacity, and the overflow bit.
void scan_visible(const uint32_t* bits, long long n_words_total, uint32_t* word_off, uint32_t* tile_sums,
                  StateHeader* hdr, unsigned long long rec_cap, cudaStream_t s) {
    const ScanTotal total{&hdr->need_records, &hdr->n_records, rec_cap, &hdr->status, kStatusRecordOverflow};
    device_exclusive_scan<PopcF, uint32_t>(PopcF{bits}, nullptr, (unsigned long long)n_words_total, tile_sums,
                                           word_off, total, s);
}

void project_records(const ViewParams* views, int n_views, Consts k, SurfelPtrs sp, const uint32_t* bits,
                     const uint32_t* word_off, long long n_words, Record* recs, uint2* rects, float* feat,
                     uint32_t* keys, uint32_t* vals, unsigned long long rec_cap, cudaStream_t s) {
    size_t sm = sizeof(ViewParams) * (size_t)n_views;
    launch_pdl(project_k, dim3(grid_for_words(n_words)), dim3(kProjThreads), sm, s, views, n_views, k, sp, bits, word_off, n_words, recs,
                                                                rects, feat, padded_channels(k.C), keys, vals,
                                                                rec_cap);
    note_launches(1);
}

}  // namespace rogs
