// common.cuh -- device-side types and helpers shared by the librogs kernels.
//
// Numerics.  GB300 runs FP64 at a small fraction of its FP32 rate, so the
// few quantities that need more than binary32 (the camera-space centre and
// the projected mean of a surfel, which suffer cancellation when the map is
// hundreds of metres wide) are carried as unevaluated float pairs
// ("double-float": hi + lo, error-free transforms built from fused
// multiply-add, Dekker/Knuth two-sum and two-product).  The projected mean is
// then stored as an integer pixel part plus a fraction in [0, 1), so that the
// per-pixel offset (u + 0.5 - mean) is exact up to one rounding.
//
// Order decisions (binary32 depth sort key, near plane, perspective box cull)
// use a fixed sequence of IEEE binary32 operations written with __fmul_rn /
// __fadd_rn, which the compiler may not contract; the CPU oracle takes the
// same decisions with the same operations.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rogs.h"

namespace rogs {

// Programmatic dependent launch.  The library's kernels are launched with
// programmatic stream serialization: a kernel's blocks may be scheduled while
// the previous kernel of the stream drains its last blocks, and every kernel
// waits at its top (griddepcontrol.wait) until that previous kernel has
// completed and its memory is visible, so the overlap hides launch latency
// and changes no result.  Outside such a launch the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline void launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

constexpr int kMaxViews = ROGS_MAX_VIEWS;
constexpr unsigned kFull = 0xffffffffu;

// Per-view parameters, derived on the host from rogs_camera.
struct ViewParams {
    int kind, W, H, tiles_x, tiles_y, exp_idx, box, box_ok;
    long long tile_base;  // global id of this view's first tile
    long long pix_base;   // global index of this view's first pixel
    float fx, fy, cx, cy;
    float R[9], t[3];
    float ox, oy, xh0, xh1, zh0, zh1;  // box cull helpers (binary32, fixed order)
    float lim_x, lim_y;                // Jacobian clamp on x/z, y/z
};

struct ViewsArg {
    ViewParams v[kMaxViews];
};

struct Consts {
    float t_min, alpha_min, alpha_max, eps, near_plane, box_half_x, box_depth;
    int tile_w, tile_h, C;
    unsigned long long rec_cap, pair_cap;   // capacities of the state buffer (bounds checks)
};

// Bounds-checked build.  Compiled with -DROGS_CHECKED, every index the
// kernels take from device data (list entries, record ids, scatter
// positions) is tested before use; a failing test records its code in this
// translation unit's error word (the first code wins) and the access is
// skipped, so a bad index shows up as a status instead of a fault.  In the
// normal build rogs_ok() is `true` and the tests compile away.
#ifdef ROGS_CHECKED
static __device__ unsigned int g_rogs_check_word;
__device__ __forceinline__ bool rogs_ok(bool cond, unsigned code) {
    if (!cond) atomicCAS(&g_rogs_check_word, 0u, code);
    return cond;
}
// Host: read and clear this translation unit's error word.
static inline unsigned rogs_check_word_take() {
    unsigned v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_rogs_check_word, sizeof(v));
    cudaMemcpyToSymbol(g_rogs_check_word, &z, sizeof(z));
    return v;
}
#else
__device__ __forceinline__ bool rogs_ok(bool, unsigned) { return true; }
#endif

// 48-byte visible (view, surfel) record; layout documented in rogs.h.
struct __align__(16) Record {
    float mxi, myi, mxf, myf;
    float ca, cb, cc, opacity;
    float depth, key;
    uint32_t surfel, view;
};
static_assert(sizeof(Record) == 48, "record layout");

struct StateHeader {  // mirrors rogs_counts
    unsigned long long n_records, n_pairs, need_records, need_pairs, composited;
    unsigned int status, n_views;
};
static_assert(sizeof(StateHeader) == sizeof(rogs_counts), "header layout");

enum : unsigned { kStatusRecordOverflow = 1u, kStatusPairOverflow = 2u };

// ------------------------------------------------------------ double-float

struct df {
    float hi, lo;
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo);
    return quick_two_sum(s.hi, lo);
}

__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    return quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a / b for double-floats (one correction step, ~44 significant bits)
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df qb = df_mul_f(b, q1);
    df r = df_add(a, {-qb.hi, -qb.lo});
    float q2 = __fdiv_rn(r.hi, b.hi);
    return quick_two_sum(q1, q2);
}

// --------------------------------------------------------------- binary32

// ((r20 x + r21 y) + r22 z) + t2, rounded per operation; -0 -> +0.
__device__ __forceinline__ float depth_key(const ViewParams& v, float x, float y, float z) {
    float s = __fadd_rn(__fmul_rn(v.R[6], x), __fmul_rn(v.R[7], y));
    s = __fadd_rn(s, __fmul_rn(v.R[8], z));
    s = __fadd_rn(s, v.t[2]);
    return __fadd_rn(s, 0.0f);
}

// Supplementary "Perspective Rendering Acceleration": keep surfels inside the
// ground box +-box_half_x along the camera's ground-projected x axis and
// [0, box_depth] along its ground-projected z axis, from the camera centre.
__device__ __forceinline__ bool box_keep(const ViewParams& v, const Consts& k, float x, float y) {
    if (!v.box || v.kind != ROGS_PERSP || !v.box_ok) return true;
    float dx = __fsub_rn(x, v.ox);
    float dy = __fsub_rn(y, v.oy);
    float lat = __fadd_rn(__fmul_rn(dx, v.xh0), __fmul_rn(dy, v.xh1));
    float fwd = __fadd_rn(__fmul_rn(dx, v.zh0), __fmul_rn(dy, v.zh1));
    return (fabsf(lat) <= k.box_half_x) && (fwd >= 0.0f) && (fwd <= k.box_depth);
}

// Order-preserving map of a float to uint32 (ascending).
__device__ __forceinline__ uint32_t float_sort_bits(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Offset of a pixel centre from a split mean: ((u + 0.5) - mean_int) - mean_frac.
__device__ __forceinline__ float pix_offset(float pc, float mi, float mf) {
    return __fsub_rn(__fsub_rn(pc, mi), mf);
}

// Offsets from a pair's split mean m (mean_int, mean_frac) of the centre of
// pixel (x0, y0), staged once per entry and warp; pixel (x0 + lx, y0 + ly) is
// then at (dx0 + lx, dy0 + ly), one add per axis (both compositing kernels
// evaluate it this way).  The reference pixel is offset_origin(px, py): the
// same for every pixel of any warp block shape, so the rounding, and with it
// every output, does not depend on the tile shape.
__device__ __forceinline__ int2 offset_origin(int px, int py) { return make_int2(px & ~31, py & ~3); }
__device__ __forceinline__ float4 block_offsets(float4 m, int2 o) {
    return make_float4(pix_offset((float)o.x + 0.5f, m.x, m.z), pix_offset((float)o.y + 0.5f, m.y, m.w), 0.0f, 0.0f);
}

// Per-pixel opacity a = min(alpha_max, alpha * exp(power)) with
// power = -0.5 (A dx^2 + 2 B dx dy + C dy^2), evaluated as a base-2
// exponential of the same quadratic form with the conic pre-scaled once per
// pair (conic_to_exp2): A2 = -A/2 log2 e, B2 = -B log2 e, C2 = -C/2 log2 e,
// so exp(power) = 2^(A2 dx^2 + B2 dx dy + C2 dy^2) takes five multiplies and
// multiply-adds and one ex2.  Written with explicit rounding so that the forward and the
// backward kernels evaluate it bit-identically.  Returns a; g receives
// exp(power).
constexpr float kLog2e = 1.4426950408889634f;
__host__ __device__ __forceinline__ float4 conic_to_exp2(float4 c) {   // (A, B, C, alpha) -> (A2, B2, C2, alpha)
    return make_float4(c.x * (-0.5f * kLog2e), c.y * -kLog2e, c.z * (-0.5f * kLog2e), c.w);
}
__host__ __device__ __forceinline__ float4 conic_from_exp2(float4 c) {   // back to (A, B, C, alpha), up to rounding
    return make_float4(c.x * (-2.0f / kLog2e), c.y * (-1.0f / kLog2e), c.z * (-2.0f / kLog2e), c.w);
}
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float surfel_alpha(float dx, float dy, float A2, float B2, float C2, float alpha,
                                              float alpha_max, float& g) {
    // q = (A2 dx + B2 dy) dx + (C2 dy) dy
    const float q = __fmaf_rn(__fmaf_rn(A2, dx, __fmul_rn(B2, dy)), dx, __fmul_rn(__fmul_rn(C2, dy), dy));
    g = exp2_approx(q);
    return fminf(alpha_max, __fmul_rn(alpha, g));
}

// Supervision of the loss (Eqs. 8, 9), in the output's pixel order: colour
// planes [3][pixels] per view and one class label per pixel, either as FP32
// and int32 or as 8-bit camera data (colour = value / 255, label = class id);
// exactly one of rgb / rgb8 is set.  A label outside [0, C) drops the pixel's
// semantic term.
struct Targets {
    const float* rgb;
    const int32_t* label;
    const uint8_t* rgb8;
    const uint8_t* label8;
    const uint8_t* mask;   // 1 = the pixel is in M
};

// x / 255 rounded to the nearest float, for an integer x in [0, 255]: an
// 8-bit colour value as a fraction of full scale.  The product with the
// rounded reciprocal is corrected once by its residual x - 255 q, which one FMA
// gives exactly (Markstein's correction step); q + residual / 255 then rounds
// to the same float as the IEEE quotient for all 256 inputs (the plain product
// misses it for 126 of them).
__device__ __forceinline__ float unit_from_u8(uint32_t x) {
    const float xf = (float)x;
    constexpr float r = 1.0f / 255.0f;
    const float q = __fmul_rn(xf, r);
    const float e = __fmaf_rn(-q, 255.0f, xf);
    return __fmaf_rn(e, r, q);
}

// One pixel's supervision (Eqs. 8, 9) from either target format: the three
// colour values (colour planes start at rgb_base, `plane` pixels apart) and
// the class label (-1 when C = 0).
__device__ __forceinline__ void load_pixel_target(const Targets& tg, long long rgb_base, long long plane,
                                                  long long pix, int C, float& t0, float& t1, float& t2, int& lb) {
    if (tg.rgb8) {
        const uint8_t* t = tg.rgb8 + rgb_base;
        t0 = unit_from_u8(t[0]);
        t1 = unit_from_u8(t[plane]);
        t2 = unit_from_u8(t[2 * plane]);
        lb = C > 0 ? (int)tg.label8[pix] : -1;
    } else {
        const float* t = tg.rgb + rgb_base;
        t0 = t[0];
        t1 = t[plane];
        t2 = t[2 * plane];
        lb = C > 0 ? tg.label[pix] : -1;
    }
}

// Conservative test: can the entry reach a >= alpha_min at some pixel centre
// of the bw x bh block whose first pixel is (bx, by)?  Uses the bounding box of
// the ellipse d^T Q d <= 2 ln(alpha / alpha_min) (Q = conic), padded so that
// rounding never drops a pixel the exact per-pixel test would keep: the fast
// log, divisions and reciprocal square root used here are within a few ulp,
// far inside the 0.2 % + 0.01 px margin.
// Half-widths (rx, ry) of the padded bounding box; negative when the conic is
// degenerate (then every block is kept).
__device__ __forceinline__ float2 block_cull_radii(float4 c, float alpha_min) {
    const float det = c.x * c.z - c.y * c.y;
    if (!(det > 0.0f)) return make_float2(-1.0f, -1.0f);
    const float kap = __fdividef(fmaxf(2.0f * __logf(__fdividef(c.w, alpha_min)), 0.0f), det);
    const float qx = fmaxf(kap * c.z, 1e-30f), qy = fmaxf(kap * c.x, 1e-30f);
    return make_float2(qx * rsqrtf(qx) * 1.002f + 0.01f, qy * rsqrtf(qy) * 1.002f + 0.01f);
}

// Pixel block of one compositing warp (32 pixels, one per lane) inside a
// tile: bw x (32 / bw) pixels.  16x2 in 16x16 tiles: each output-plane access
// of a warp is two 64-byte row segments instead of four 32-byte ones (measured
// 8 % faster forward, 4 % faster backward on the scene than 8x4); 8x4 in the
// 8x8 and 32x8 tiles (32x1 rows in 32x8 tiles measured slower).
__host__ __device__ constexpr int block_w(int tw, int th) { return tw == 16 && th == 16 ? 16 : 8; }

__device__ __forceinline__ bool box_hits_block(float4 m, float2 r, float bx, float by, int bw, int bh) {
    if (r.x < 0.0f) return true;
    const float mx = m.x + m.z, my = m.y + m.w;
    return (mx + r.x >= bx + 0.5f) && (mx - r.x <= bx + (float)bw - 0.5f) && (my + r.y >= by + 0.5f) &&
           (my - r.y <= by + (float)bh - 0.5f);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp (among `valid`) whose digit d (bits under `mask`, at most
// 8) equals this lane's: one ballot per digit bit, so the cost does not depend
// on how many distinct digits the warp holds.  Every lane must call it.
__device__ __forceinline__ unsigned warp_digit_peers(uint32_t d, uint32_t mask, unsigned valid) {
    unsigned peers = valid;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if ((mask >> b) & 1u) {
            const unsigned m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
    }
    return peers;
}

// Copy the first n_views view parameter sets into shared memory (block-wide).
__device__ __forceinline__ void load_views_smem(ViewParams* sv, const ViewParams* views, int n_views) {
    const int words = n_views * (int)(sizeof(ViewParams) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(views);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sv);
    for (int t = threadIdx.x; t < words; t += blockDim.x) dst[t] = src[t];
    __syncthreads();
}

// Binary search of the view owning global tile t (tile_base ascending).
__device__ __forceinline__ int view_of_tile(const ViewParams* views, int n_views, long long t) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace rogs
