// api.cu -- the C-ABI of librogs (declared in include/rogs.h): argument
// checks, per-view parameter derivation, scratch management and the launch
// sequences of the forward, loss and backward passes.
//
// Host arithmetic that feeds an order decision (camera centre and ground
// axes of the perspective box cull) is done in binary32, one rounding per
// operation, in the same order as the oracle; this file is compiled with
// -ffp-contract=off so the host compiler cannot fuse it.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <string>
#include <vector>

#include "kernels.h"

using namespace rogs;

namespace rogs {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
// Test hook (rogs_debug_fail_alloc): while set, every scratch allocation of
// the library reports that the device is out of memory.
static std::atomic<int> g_fail_alloc{0};
bool debug_alloc_fails() { return g_fail_alloc.load() != 0; }
}  // namespace rogs

struct rogs_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct ProfEvent {
    int stage;
    cudaEvent_t a, b;
};

struct rogs_ctx {
    rogs_config cfg;
    int device = 0;
    std::string err;
    // capacity-sized scratch
    uint32_t *dk_a = nullptr, *dv_a = nullptr, *dk_b = nullptr, *dv_b = nullptr, *dk_c = nullptr, *dv_c = nullptr;
    uint32_t *pk_a = nullptr, *pv_a = nullptr, *pk_b = nullptr, *pk_c = nullptr, *pv_c = nullptr;
    uint32_t* hist = nullptr;
    unsigned long long *pair_off = nullptr, *pair_tiles = nullptr;
    float* rec_grad = nullptr;
    float* smooth_partials = nullptr;   // one per CTA of the smoothness-loss stencil
    float* smooth_val = nullptr;        // lambda_smooth L_smooth of the current training step
    float* elev_partials = nullptr;     // one per CTA of the LiDAR elevation loss
    cudaStream_t side = nullptr;        // runs the smoothness loss beside the backward compositing
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;   // the final loss sum beside the projection backward
    LidarScratch lidar{};               // point-cloud hash of rogs_elev_targets
    float* bev_out = nullptr;           // per-batch chunk outputs of rogs_bev_export
    uint8_t* bev_state = nullptr;
    size_t bev_out_cap = 0, bev_state_cap = 0;
    size_t lidar_cap = 0, lidar_hist_cap = 0, lidar_range_cap = 0;
    // grown on demand
    uint32_t *bits = nullptr, *word_off = nullptr, *bits_tiles = nullptr;
    size_t bits_cap = 0;  // words
    float* loss_partials = nullptr;
    unsigned long long* loss_counter = nullptr;
    size_t loss_cap = 0;  // blocks
    ViewParams* loss_views = nullptr;
    float* poses = nullptr;
    size_t poses_cap = 0;  // floats
    // per-stage timing
    bool prof = false;
    std::vector<ProfEvent> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[ROGS_N_STAGES] = {0};
    unsigned long long prof_calls[ROGS_N_STAGES] = {0};
    int prof_open = -1;
    cudaEvent_t prof_open_ev = nullptr;
    cudaStream_t prof_stream = nullptr;
};

namespace {

rogs_status fail(rogs_ctx* ctx, rogs_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

#define ROGS_CUDA(ctx, expr)                                                                        \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(ctx, ROGS_ERR_CUDA, std::string(#expr ": ") + cudaGetErrorString(e_));      \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

cudaEvent_t prof_event(rogs_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Close the open stage (if any) and open `stage` on stream s (-1: just close).
void prof_mark(rogs_ctx* ctx, int stage, cudaStream_t s) {
    if (!ctx->prof || capturing(s)) return;
    cudaEvent_t e = prof_event(ctx);
    cudaEventRecord(e, s);
    if (ctx->prof_open >= 0) ctx->prof_pending.push_back({ctx->prof_open, ctx->prof_open_ev, e});
    if (stage >= 0) {
        cudaEvent_t e2 = prof_event(ctx);
        cudaEventRecord(e2, s);
        ctx->prof_open = stage;
        ctx->prof_open_ev = e2;
    } else {
        ctx->prof_open = -1;
        ctx->prof_open_ev = nullptr;
    }
}

template <class T>
rogs_status grow(rogs_ctx* ctx, T*& ptr, size_t& cap, size_t need, cudaStream_t s, bool zero = false) {
    if (need <= cap && ptr) return ROGS_OK;
    if (capturing(s))
        return fail(ctx, ROGS_ERR_CAPACITY, "scratch must grow during stream capture; call rogs_reserve first");
    if (ptr) {
        cudaStreamSynchronize(s);
        cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
    }
    size_t n = need > 0 ? need : 1;
    cudaError_t e = debug_alloc_fails() ? cudaErrorMemoryAllocation : cudaMalloc((void**)&ptr, n * sizeof(T));
    if (e != cudaSuccess) {
        ptr = nullptr;
        return fail(ctx, ROGS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    // cleared on the stream of the call that grew it, so the clear is ordered
    // before that call's kernels
    if (zero && cudaMemsetAsync(ptr, 0, n * sizeof(T), s) != cudaSuccess)
        return fail(ctx, ROGS_ERR_CUDA, "cudaMemsetAsync of new scratch failed");
    cap = n;
    return ROGS_OK;
}

Consts make_consts(const rogs_config& c) {
    Consts k;
    k.t_min = c.t_min;
    k.alpha_min = c.alpha_min;
    k.alpha_max = c.alpha_max;
    k.eps = c.eps_dilate;
    k.near_plane = c.near_plane;
    k.box_half_x = c.box_half_x;
    k.box_depth = c.box_depth;
    k.tile_w = c.tile_w;
    k.tile_h = c.tile_h;
    k.C = c.num_classes;
    k.rec_cap = (unsigned long long)c.record_capacity;
    k.pair_cap = (unsigned long long)c.pair_capacity;
    return k;
}

// Derive device view parameters; returns false with a message on bad input.
bool make_views(const rogs_config& cfg, const rogs_camera* cams, int n, ViewsArg& va, long long& total_tiles,
                long long& total_pix, std::string& err) {
    total_tiles = 0;
    total_pix = 0;
    for (int i = 0; i < n; ++i) {
        const rogs_camera& c = cams[i];
        ViewParams& v = va.v[i];
        std::memset(&v, 0, sizeof(v));
        if (c.kind != ROGS_PERSP && c.kind != ROGS_ORTHO) { err = "camera kind must be ROGS_PERSP or ROGS_ORTHO"; return false; }
        if (c.width <= 0 || c.height <= 0) { err = "camera width and height must be positive"; return false; }
        if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !std::isfinite(c.fx) || !std::isfinite(c.fy)) {
            err = "camera focal lengths must be positive and finite";
            return false;
        }
        bool finite = std::isfinite(c.cx) && std::isfinite(c.cy);
        for (int k = 0; k < 9; ++k) finite = finite && std::isfinite(c.R_wc[k]);
        for (int k = 0; k < 3; ++k) finite = finite && std::isfinite(c.t_wc[k]);
        if (!finite) { err = "camera parameters must be finite"; return false; }
        v.kind = c.kind;
        v.W = c.width;
        v.H = c.height;
        v.tiles_x = (c.width + cfg.tile_w - 1) / cfg.tile_w;
        v.tiles_y = (c.height + cfg.tile_h - 1) / cfg.tile_h;
        if (v.tiles_x > 65535 || v.tiles_y > 65535) { err = "camera too large for 16-bit tile coordinates"; return false; }
        v.exp_idx = c.exposure_idx;
        v.box = c.use_box_cull ? 1 : 0;
        v.tile_base = total_tiles;
        v.pix_base = total_pix;
        total_tiles += (long long)v.tiles_x * v.tiles_y;
        total_pix += (long long)c.width * c.height;
        v.fx = c.fx; v.fy = c.fy; v.cx = c.cx; v.cy = c.cy;
        for (int k = 0; k < 9; ++k) v.R[k] = c.R_wc[k];
        for (int k = 0; k < 3; ++k) v.t[k] = c.t_wc[k];
        // camera centre o = -R^T t (binary32, fixed order)
        {
            float a = c.R_wc[0] * c.t_wc[0];
            float b = c.R_wc[3] * c.t_wc[1];
            float s = a + b;
            float d = c.R_wc[6] * c.t_wc[2];
            s = s + d;
            v.ox = -s;
            a = c.R_wc[1] * c.t_wc[0];
            b = c.R_wc[4] * c.t_wc[1];
            s = a + b;
            d = c.R_wc[7] * c.t_wc[2];
            s = s + d;
            v.oy = -s;
        }
        // ground-projected camera x and z axes, normalised (binary32)
        {
            float p = c.R_wc[0] * c.R_wc[0];
            float q = c.R_wc[1] * c.R_wc[1];
            float nx = std::sqrt(p + q);
            p = c.R_wc[6] * c.R_wc[6];
            q = c.R_wc[7] * c.R_wc[7];
            float nz = std::sqrt(p + q);
            v.box_ok = (nx >= 1e-6f && nz >= 1e-6f) ? 1 : 0;
            if (v.box_ok) {
                v.xh0 = c.R_wc[0] / nx; v.xh1 = c.R_wc[1] / nx;
                v.zh0 = c.R_wc[6] / nz; v.zh1 = c.R_wc[7] / nz;
            }
        }
        v.lim_x = (float)(cfg.jac_clamp * (0.5 * c.width / c.fx));
        v.lim_y = (float)(cfg.jac_clamp * (0.5 * c.height / c.fy));
    }
    if (total_tiles >= (1ll << 32)) { err = "too many tiles in one call"; return false; }
    return true;
}

struct Layout {
    rogs_state_layout l;
};

rogs_state_layout layout_for(const rogs_config& cfg, long long total_tiles, long long total_pix) {
    rogs_state_layout L;
    size_t off = 0;
    L.header = off; off = align256(off + sizeof(StateHeader));
    L.views = off; off = align256(off + sizeof(ViewParams) * kMaxViews);
    L.records = off; off = align256(off + sizeof(Record) * (size_t)cfg.record_capacity);
    L.rects = off; off = align256(off + 8 * (size_t)cfg.record_capacity);
    L.pair_rec = off; off = align256(off + 4 * (size_t)cfg.pair_capacity);
    L.tile_range = off; off = align256(off + 8 * (size_t)total_tiles);
    L.pix_T = off; off = align256(off + 4 * (size_t)total_pix);
    L.pix_last = off; off = align256(off + 4 * (size_t)total_pix);
    L.tile_order = off; off = align256(off + 4 * (size_t)total_tiles);
    L.rec_feat = off; off = align256(off + 4 * (size_t)padded_channels(cfg.num_classes) * (size_t)cfg.record_capacity);
    L.pair_mc = off; off = align256(off + 32 * (size_t)cfg.pair_capacity);
    L.pair_blk = off; off = align256(off + (size_t)cfg.pair_capacity);
    L.total_bytes = off;
    L.total_tiles = total_tiles;
    L.total_pixels = total_pix;
    return L;
}

int bits_for(long long n) {
    int b = 0;
    while (b < 32 && (1ll << b) < n) ++b;
    return b;
}

bool valid_config(const rogs_config& c, std::string& err) {
    const bool tile_ok = (c.tile_w == 16 && c.tile_h == 16) || (c.tile_w == 32 && c.tile_h == 8) ||
                         (c.tile_w == 8 && c.tile_h == 8);
    if (!tile_ok) { err = "tile must be 16x16, 32x8 or 8x8"; return false; }
    if (c.num_classes < 0 || c.num_classes > ROGS_MAX_CLASSES) { err = "num_classes out of range"; return false; }
    if (c.record_capacity < 1 || c.record_capacity > 0xffffffffll) { err = "record_capacity out of range"; return false; }
    if (c.pair_capacity < 1 || c.pair_capacity > 0xffffffffll) { err = "pair_capacity out of range"; return false; }
    if (!(c.alpha_min > 0.0f) || !(c.alpha_max > c.alpha_min) || !(c.alpha_max < 1.0f)) {
        err = "need 0 < alpha_min < alpha_max < 1";
        return false;
    }
    if (!(c.t_min > 0.0f) || !(c.t_min < 1.0f)) { err = "need 0 < t_min < 1"; return false; }
    if (!(c.eps_dilate >= 0.0f)) { err = "eps_dilate must be >= 0"; return false; }
    if (c.sort_tile != 1024 && c.sort_tile != 2048 && c.sort_tile != 4096 && c.sort_tile != 8192) {
        err = "sort_tile must be 1024, 2048, 4096 or 8192";
        return false;
    }
    return true;
}

bool check_surfels(const rogs_surfels* s, int C, std::string& err) {
    if (!s) { err = "surfels is NULL"; return false; }
    if (s->n < 0) { err = "negative surfel count"; return false; }
    if (s->n == 0) return true;
    if (!s->xyz || !s->scale || !s->quat || !s->opacity || !s->rgb || (C > 0 && !s->sem)) {
        err = "a surfel attribute pointer is NULL";
        return false;
    }
    if (((uintptr_t)s->quat & 15u) || ((uintptr_t)s->scale & 7u) || ((uintptr_t)s->xyz & 3u)) {
        err = "quat must be 16-byte and scale 8-byte aligned";
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

rogs_status rogs_default_config(int32_t num_classes, int64_t record_capacity, int64_t pair_capacity,
                                rogs_config* cfg) {
    if (!cfg) return ROGS_ERR_INVALID;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->num_classes = num_classes;
    cfg->t_min = 1e-4f;
    cfg->alpha_min = 1.0f / 255.0f;
    cfg->alpha_max = 0.99f;
    cfg->eps_dilate = 0.3f;
    cfg->near_plane = 0.2f;
    cfg->box_half_x = 20.0f;
    cfg->box_depth = 40.0f;
    cfg->jac_clamp = 1.3f;
    cfg->sort_tile = 4096;
    cfg->record_capacity = record_capacity;
    cfg->pair_capacity = pair_capacity;
    return ROGS_OK;
}

rogs_status rogs_create(const rogs_config* cfg, rogs_ctx** out) {
    if (!cfg || !out) return ROGS_ERR_INVALID;
    *out = nullptr;
    std::string err;
    if (!valid_config(*cfg, err)) return ROGS_ERR_INVALID;
    rogs_ctx* ctx = new rogs_ctx();
    ctx->cfg = *cfg;
    cudaGetDevice(&ctx->device);
    const size_t R = (size_t)cfg->record_capacity, P = (size_t)cfg->pair_capacity;
    const size_t big = R > P ? R : P;
    size_t c0 = 0;
    rogs_status st = ROGS_OK;
#define ROGS_ALLOC(ptr, count)                                                      \
    do {                                                                            \
        size_t cap_ = 0;                                                            \
        if (st == ROGS_OK) st = grow(ctx, ptr, cap_, (count), nullptr);             \
    } while (0)
    ROGS_ALLOC(ctx->dk_a, R); ROGS_ALLOC(ctx->dv_a, R); ROGS_ALLOC(ctx->dk_b, R);
    ROGS_ALLOC(ctx->dv_b, R); ROGS_ALLOC(ctx->dk_c, R); ROGS_ALLOC(ctx->dv_c, R);
    ROGS_ALLOC(ctx->pk_a, P); ROGS_ALLOC(ctx->pv_a, P); ROGS_ALLOC(ctx->pk_b, P);
    ROGS_ALLOC(ctx->pk_c, P); ROGS_ALLOC(ctx->pv_c, P);
    ROGS_ALLOC(ctx->hist, radix_hist_words(big));
    ROGS_ALLOC(ctx->pair_off, R + 1);
    ROGS_ALLOC(ctx->pair_tiles, scan_tile_sums_words(R));
    ROGS_ALLOC(ctx->loss_views, (size_t)kMaxViews);
    ROGS_ALLOC(ctx->smooth_partials, (size_t)smooth_blocks());
    ROGS_ALLOC(ctx->smooth_val, 1);
    ROGS_ALLOC(ctx->elev_partials, (size_t)elev_blocks());
    if (st == ROGS_OK && (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming) != cudaSuccess))
        st = ROGS_ERR_CUDA;
#undef ROGS_ALLOC
    (void)c0;
    if (st != ROGS_OK) {
        rogs_destroy(ctx);
        return st;
    }
    prepare_composite_fwd();
    prepare_composite_bwd();
    prepare_sort();
    cudaDeviceSynchronize();
    *out = ctx;
    return ROGS_OK;
}

void rogs_destroy(rogs_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    void* ptrs[] = {ctx->dk_a, ctx->dv_a, ctx->dk_b, ctx->dv_b, ctx->dk_c, ctx->dv_c, ctx->pk_a, ctx->pv_a,
                    ctx->pk_b, ctx->pk_c, ctx->pv_c, ctx->hist, ctx->pair_off, ctx->pair_tiles, ctx->rec_grad,
                    ctx->bits, ctx->word_off, ctx->bits_tiles, ctx->loss_partials, ctx->loss_counter,
                    ctx->loss_views, ctx->poses, ctx->smooth_partials, ctx->smooth_val, ctx->elev_partials,
                    ctx->lidar.keys, ctx->lidar.vals, ctx->lidar.skeys, ctx->lidar.svals, ctx->lidar.kalt,
                    ctx->lidar.valt, ctx->lidar.hist, ctx->lidar.ranges, ctx->lidar.sorted, ctx->bev_out,
                    ctx->bev_state};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
    if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (const ProfEvent& pe : ctx->prof_pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->prof_open_ev) cudaEventDestroy(ctx->prof_open_ev);
    delete ctx;
}

const char* rogs_last_error(const rogs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static rogs_status ensure_bits(rogs_ctx* ctx, long long n, int n_views, cudaStream_t s) {
    const long long n_words = (n + 31) / 32;
    const size_t need = (size_t)n_words * (size_t)n_views;
    size_t c1 = ctx->bits_cap, c2 = ctx->bits_cap;
    if (need <= ctx->bits_cap && ctx->bits) return ROGS_OK;
    size_t c3 = 0;
    rogs_status st = grow(ctx, ctx->bits, c1, need, s);
    if (st == ROGS_OK) st = grow(ctx, ctx->word_off, c2, need, s);
    if (st == ROGS_OK) {
        if (ctx->bits_tiles) { cudaFree(ctx->bits_tiles); ctx->bits_tiles = nullptr; }
        st = grow(ctx, ctx->bits_tiles, c3, scan_tile_sums_words(need), s);
    }
    if (st == ROGS_OK) ctx->bits_cap = c1 < c2 ? c1 : c2;
    return st;
}

// The per-record gradient rows are only needed by the backward: allocated
// (zeroed) on first use.
static rogs_status ensure_rec_grad(rogs_ctx* ctx, cudaStream_t s) {
    if (ctx->rec_grad) return ROGS_OK;
    size_t cap = 0;
    return grow(ctx, ctx->rec_grad, cap, (size_t)ctx->cfg.record_capacity * (size_t)grad_channels(ctx->cfg.num_classes), s, true);
}

static rogs_status ensure_loss(rogs_ctx* ctx, long long total_pix, cudaStream_t s, size_t min_partials = 0) {
    size_t nb = (size_t)loss_blocks(total_pix) + 1;
    if (min_partials + 1 > nb) nb = min_partials + 1;
    if (nb <= ctx->loss_cap && ctx->loss_partials) return ROGS_OK;
    size_t c = ctx->loss_cap, c2 = 0;
    rogs_status st = grow(ctx, ctx->loss_partials, c, nb, s);
    if (st == ROGS_OK && !ctx->loss_counter) st = grow(ctx, ctx->loss_counter, c2, 1, s);
    if (st == ROGS_OK) ctx->loss_cap = c;
    return st;
}

rogs_status rogs_reserve(rogs_ctx* ctx, int64_t n_surfels, const rogs_camera* cams, int32_t n_views,
                         int32_t training) {
    if (!ctx || n_surfels < 0 || n_views < 1 || n_views > kMaxViews) return fail(ctx, ROGS_ERR_INVALID, "bad reserve");
    rogs_status st = ensure_bits(ctx, n_surfels, n_views, nullptr);
    if (st == ROGS_OK && training) st = ensure_rec_grad(ctx, nullptr);
    if (st == ROGS_OK && training && cams) {
        static thread_local ViewsArg va;
        long long tt, tp;
        std::string err;
        if (!make_views(ctx->cfg, cams, n_views, va, tt, tp, err)) return fail(ctx, ROGS_ERR_INVALID, err);
        st = ensure_loss(ctx, tp, nullptr, (size_t)bwd_loss_partials(tt, ctx->cfg.tile_w, ctx->cfg.tile_h));
    }
    if (st == ROGS_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(ctx, ROGS_ERR_CUDA, "reserve: synchronise");
    return st;
}

void rogs_debug_fail_alloc(int32_t fail_all) { g_fail_alloc.store(fail_all ? 1 : 0); }

int32_t rogs_bounds_checked(uint32_t* code) {
#ifdef ROGS_CHECKED
    cudaDeviceSynchronize();
    const unsigned w[4] = {check_word_composite(), check_word_backward(), check_word_sort(), check_word_bin()};
    unsigned c = 0;
    for (unsigned x : w)
        if (!c) c = x;
    if (code) *code = c;
    return 1;
#else
    if (code) *code = 0;
    return 0;
#endif
}

rogs_status rogs_state_layout_of(const rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views,
                                 rogs_state_layout* layout, uint64_t* out_elems) {
    if (!ctx || !cams || !layout || n_views < 1 || n_views > kMaxViews) return ROGS_ERR_INVALID;
    static thread_local ViewsArg va;
    long long tt, tp;
    std::string err;
    if (!make_views(ctx->cfg, cams, n_views, va, tt, tp, err)) {
        const_cast<rogs_ctx*>(ctx)->err = err;
        return ROGS_ERR_INVALID;
    }
    *layout = layout_for(ctx->cfg, tt, tp);
    if (out_elems) *out_elems = (uint64_t)(3 + ctx->cfg.num_classes + 1) * (uint64_t)tp;
    return ROGS_OK;
}

rogs_status rogs_state_counts(rogs_ctx* ctx, const void* state, rogs_counts* counts, rogs_stream stream) {
    if (!ctx || !state || !counts) return fail(ctx, ROGS_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    ROGS_CUDA(ctx, cudaMemcpyAsync(counts, state, sizeof(rogs_counts), cudaMemcpyDeviceToHost, s));
    ROGS_CUDA(ctx, cudaStreamSynchronize(s));
    if (counts->status) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "capacity exceeded: need %llu records (cap %lld), %llu pairs (cap %lld)",
                      (unsigned long long)counts->need_records, (long long)ctx->cfg.record_capacity,
                      (unsigned long long)counts->need_pairs, (long long)ctx->cfg.pair_capacity);
        return fail(ctx, ROGS_ERR_CAPACITY, buf);
    }
    return ROGS_OK;
}

rogs_status rogs_init_from_poses(rogs_ctx* ctx, const float* grid_xy, int64_t n, const float* poses, int64_t n_poses,
                                 int32_t exact_plane, float* out_z, float* out_quat, int32_t* out_nearest,
                                 rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (n < 0 || n_poses < 1 || !poses) return fail(ctx, ROGS_ERR_INVALID, "need n >= 0 and at least one pose");
    if (n > 0 && (!grid_xy || !out_z || !out_quat)) return fail(ctx, ROGS_ERR_INVALID, "null device pointer");
    if (((uintptr_t)out_quat & 15u) || ((uintptr_t)grid_xy & 7u))
        return fail(ctx, ROGS_ERR_INVALID, "out_quat must be 16-byte and grid_xy 8-byte aligned");
    for (int64_t v = 0; v < n_poses; ++v) {
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(poses[12 * v + k])) return fail(ctx, ROGS_ERR_INVALID, "pose values must be finite");
        if (exact_plane && std::fabs(poses[12 * v + 3 + 8]) < 1e-6f)
            return fail(ctx, ROGS_ERR_INVALID, "pose with |n33| < 1e-6 (road normal parallel to the ground)");
    }
    cudaStream_t s = (cudaStream_t)stream;
    rogs_status st = grow(ctx, ctx->poses, ctx->poses_cap, (size_t)(12 * n_poses), s);
    if (st != ROGS_OK) return st;
    ROGS_CUDA(ctx, cudaMemcpyAsync(ctx->poses, poses, sizeof(float) * 12 * (size_t)n_poses, cudaMemcpyHostToDevice, s));
    init_from_poses(grid_xy, n, ctx->poses, n_poses, exact_plane, out_z, out_quat, out_nearest, s);
    ROGS_CUDA(ctx, cudaGetLastError());
    ROGS_CUDA(ctx, cudaStreamSynchronize(s));
    return ROGS_OK;
}

rogs_status rogs_render_fwd(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                            const float* exposure_ab, int32_t n_exposure, float* out, void* state,
                            rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    const rogs_config& cfg = ctx->cfg;
    std::string err;
    if (!cams || n_views < 1 || n_views > kMaxViews) return fail(ctx, ROGS_ERR_INVALID, "n_views out of range");
    if (!check_surfels(surfels, cfg.num_classes, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    if (!out || !state || !exposure_ab || n_exposure < 1) return fail(ctx, ROGS_ERR_INVALID, "null output/state/exposure");
    if ((uintptr_t)state & 255u) return fail(ctx, ROGS_ERR_INVALID, "state must be 256-byte aligned");
    if ((unsigned long long)surfels->n * (unsigned long long)n_views >= 0xffffffffull)
        return fail(ctx, ROGS_ERR_INVALID, "surfels x views must be < 2^32");
    static thread_local ViewsArg va;
    long long total_tiles, total_pix;
    if (!make_views(cfg, cams, n_views, va, total_tiles, total_pix, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    for (int i = 0; i < n_views; ++i)
        if (cams[i].exposure_idx < 0 || cams[i].exposure_idx >= n_exposure)
            return fail(ctx, ROGS_ERR_INVALID, "exposure_idx out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = surfels->n;
    const long long n_words = (n + 31) / 32;
    rogs_status st = ensure_bits(ctx, n, n_views, s);
    if (st != ROGS_OK) return st;

    const rogs_state_layout L = layout_for(cfg, total_tiles, total_pix);
    char* sb = (char*)state;
    StateHeader* hdr = (StateHeader*)(sb + L.header);
    ViewParams* views = (ViewParams*)(sb + L.views);
    Record* recs = (Record*)(sb + L.records);
    uint2* rects = (uint2*)(sb + L.rects);
    uint32_t* pair_rec = (uint32_t*)(sb + L.pair_rec);
    uint2* ranges = (uint2*)(sb + L.tile_range);
    float* pix_T = (float*)(sb + L.pix_T);
    uint32_t* pix_last = (uint32_t*)(sb + L.pix_last);
    uint32_t* tile_order = (uint32_t*)(sb + L.tile_order);
    const unsigned long long rcap = (unsigned long long)cfg.record_capacity;
    const unsigned long long pcap = (unsigned long long)cfg.pair_capacity;
    const Consts k = make_consts(cfg);
    const SurfelPtrs sp{surfels->xyz, surfels->scale, surfels->quat, surfels->opacity, surfels->rgb, surfels->sem, n};

    prof_mark(ctx, 0, s);
    upload_views(va, n_views, views, hdr, s);
    if (n > 0) {
        cull_views(views, n_views, k, sp, ctx->bits, n_words, s);
        scan_visible(ctx->bits, n_words * n_views, ctx->word_off, ctx->bits_tiles, hdr, rcap, s);
        project_records(views, n_views, k, sp, ctx->bits, ctx->word_off, n_words, recs, rects,
                        (float*)(sb + L.rec_feat), ctx->dk_a, ctx->dv_a,
                        rcap, s);
        // depth sort: stable on the binary32 depth key; ties keep (view, surfel) order.
        // The records are a few times fewer than the pairs: 1024 keys per CTA
        // give its four passes enough CTAs to fill the SMs at every sort_tile.
        prof_mark(ctx, 1, s);
        radix_sort_pairs(ctx->dk_a, ctx->dv_a, ctx->dk_b, ctx->dv_b, ctx->dk_c, ctx->dv_c, &hdr->n_records, rcap, 32,
                         ctx->hist, s, kRsMinTile);
        prof_mark(ctx, 2, s);
        scan_pairs(ctx->dv_b, rects, hdr, rcap, ctx->pair_off, ctx->pair_tiles, hdr, pcap, s);
        emit_pairs(views, n_views, ctx->dv_b, recs, rects, ctx->pair_off, hdr, rcap, ctx->pk_a, ctx->pv_a, pcap, s);
        // tile sort: stable on the global tile id; lists stay in depth order
        prof_mark(ctx, 3, s);
        radix_sort_pairs(ctx->pk_a, ctx->pv_a, ctx->pk_b, pair_rec, ctx->pk_c, ctx->pv_c, &hdr->n_pairs, pcap,
                         bits_for(total_tiles), ctx->hist, s, cfg.sort_tile);
    }
    ROGS_CUDA(ctx, cudaMemsetAsync(ranges, 0, 8 * (size_t)total_tiles, s));
    if (n > 0)
        tile_ranges(ctx->pk_b, pair_rec, recs, views, n_views, k, hdr, pcap, ranges, (float4*)(sb + L.pair_mc),
                    (uint8_t*)(sb + L.pair_blk), s);
    // longest lists first: the compositing kernels take their tiles in this order
    order_tiles(ranges, total_tiles, tile_order, (unsigned long long)total_tiles <= pcap, ctx->pk_a, ctx->pv_a,
                ctx->pk_c, ctx->pv_c, ctx->pk_b, ctx->hist, s, cfg.sort_tile);
    prof_mark(ctx, 4, s);
    composite_fwd(cfg.tile_w, cfg.tile_h, cfg.num_classes, views, n_views, total_tiles, k, sp, recs,
                  (const float*)(sb + L.rec_feat), (const float4*)(sb + L.pair_mc), (const uint8_t*)(sb + L.pair_blk),
                  pair_rec, ranges,
                  tile_order, exposure_ab, out, pix_T, pix_last, hdr, s);
    prof_mark(ctx, -1, s);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

}  // extern "C"

namespace {

// The targets of one call are complete: colour planes, mask, and the labels
// when the model has classes.
bool targets_complete(const Targets& tg, int C) {
    if (tg.rgb8) return tg.mask && (C == 0 || tg.label8);
    return tg.rgb && tg.mask && (C == 0 || tg.label);
}

rogs_status loss_impl(rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views, const float* out, const Targets& tg,
                      float lambda_c, float lambda_s, float* loss, float* grad_out, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (!cams || n_views < 1 || n_views > kMaxViews) return fail(ctx, ROGS_ERR_INVALID, "n_views out of range");
    if (!out || !targets_complete(tg, ctx->cfg.num_classes) || !loss || !grad_out)
        return fail(ctx, ROGS_ERR_INVALID, "null device pointer");
    static thread_local ViewsArg va;
    long long tt, tp;
    std::string err;
    if (!make_views(ctx->cfg, cams, n_views, va, tt, tp, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    cudaStream_t s = (cudaStream_t)stream;
    rogs_status st = ensure_loss(ctx, tp, s);
    if (st != ROGS_OK) return st;
    prof_mark(ctx, 5, s);
    upload_views(va, n_views, ctx->loss_views, nullptr, s);
    loss_fwd_bwd(ctx->loss_views, n_views, tp, ctx->cfg.num_classes, out, tg, lambda_c, lambda_s,
                 loss, grad_out, ctx->loss_counter, ctx->loss_partials, (int)ctx->loss_cap, s);
    prof_mark(ctx, -1, s);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

}  // namespace

extern "C" {

rogs_status rogs_loss(rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views, const float* out, const float* tgt_rgb,
                      const int32_t* label, const uint8_t* mask, float lambda_c, float lambda_s, float* loss,
                      float* grad_out, rogs_stream stream) {
    const Targets tg{tgt_rgb, label, nullptr, nullptr, mask};
    return loss_impl(ctx, cams, n_views, out, tg, lambda_c, lambda_s, loss, grad_out, stream);
}

rogs_status rogs_loss_u8(rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views, const float* out,
                         const uint8_t* tgt_rgb, const uint8_t* label, const uint8_t* mask, float lambda_c,
                         float lambda_s, float* loss, float* grad_out, rogs_stream stream) {
    const Targets tg{nullptr, nullptr, tgt_rgb, label, mask};
    if (!tgt_rgb) return ctx ? fail(ctx, ROGS_ERR_INVALID, "null device pointer") : ROGS_ERR_INVALID;
    return loss_impl(ctx, cams, n_views, out, tg, lambda_c, lambda_s, loss, grad_out, stream);
}

rogs_status rogs_render_bwd(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                            const float* exposure_ab, int32_t n_exposure, const void* state, const float* grad_out,
                            const rogs_grads* grads, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    const rogs_config& cfg = ctx->cfg;
    std::string err;
    if (!cams || n_views < 1 || n_views > kMaxViews) return fail(ctx, ROGS_ERR_INVALID, "n_views out of range");
    if (!check_surfels(surfels, cfg.num_classes, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    if (!state || !grad_out || !grads || !exposure_ab || n_exposure < 1)
        return fail(ctx, ROGS_ERR_INVALID, "null state/grad_out/grads/exposure");
    if ((uintptr_t)state & 255u) return fail(ctx, ROGS_ERR_INVALID, "state must be 256-byte aligned");
    static thread_local ViewsArg va;
    long long total_tiles, total_pix;
    if (!make_views(cfg, cams, n_views, va, total_tiles, total_pix, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    for (int i = 0; i < n_views; ++i)
        if (cams[i].exposure_idx < 0 || cams[i].exposure_idx >= n_exposure)
            return fail(ctx, ROGS_ERR_INVALID, "exposure_idx out of range");
    if (grads->quat && ((uintptr_t)grads->quat & 15u)) return fail(ctx, ROGS_ERR_INVALID, "grad quat alignment");
    cudaStream_t s = (cudaStream_t)stream;
    {
        rogs_status st = ensure_rec_grad(ctx, s);
        if (st != ROGS_OK) return st;
    }
    const rogs_state_layout L = layout_for(cfg, total_tiles, total_pix);
    const char* sb = (const char*)state;
    const StateHeader* hdr = (const StateHeader*)(sb + L.header);
    const ViewParams* views = (const ViewParams*)(sb + L.views);
    const Record* recs = (const Record*)(sb + L.records);
    const uint32_t* pair_rec = (const uint32_t*)(sb + L.pair_rec);
    const uint2* ranges = (const uint2*)(sb + L.tile_range);
    const float* pix_T = (const float*)(sb + L.pix_T);
    const uint32_t* pix_last = (const uint32_t*)(sb + L.pix_last);
    const uint32_t* tile_order = (const uint32_t*)(sb + L.tile_order);
    const Consts k = make_consts(cfg);
    const SurfelPtrs sp{surfels->xyz, surfels->scale, surfels->quat, surfels->opacity, surfels->rgb, surfels->sem,
                        surfels->n};
    const GradPtrs gp{grads->xyz, grads->scale, grads->quat, grads->opacity, grads->rgb, grads->sem, grads->exposure};
    BwdArgs a{};
    a.views = views; a.n_views = n_views; a.k = k; a.sp = sp; a.recs = recs; a.pair_rec = pair_rec; a.ranges = ranges;
    a.feat = (const float*)(sb + L.rec_feat);
    a.pair_mc = (const float4*)(sb + L.pair_mc);
    a.pair_blk = (const uint8_t*)(sb + L.pair_blk);
    a.tile_order = tile_order; a.exposure_ab = exposure_ab; a.pix_T = pix_T; a.pix_last = pix_last;
    a.grad_out = grad_out;
    a.rec_grad = ctx->rec_grad; a.d_exposure = grads->exposure;
    prof_mark(ctx, 6, s);
    composite_bwd(cfg.tile_w, cfg.tile_h, total_tiles, a, s);
    prof_mark(ctx, 7, s);
    project_bwd(views, sp, recs, hdr, (unsigned long long)cfg.record_capacity, ctx->rec_grad, cfg.num_classes, gp, s);
    prof_mark(ctx, -1, s);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

}  // extern "C"

namespace {

rogs_status train_step_impl(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                            const float* exposure_ab, int32_t n_exposure, float* out, void* state, const Targets& tg,
                            float lambda_c, float lambda_s, float lambda_smooth, float* loss, const rogs_grads* grads,
                            rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    const rogs_config& cfg = ctx->cfg;
    if (!targets_complete(tg, cfg.num_classes) || !loss || !grads)
        return fail(ctx, ROGS_ERR_INVALID, "null target/loss/grads pointer");
    if (lambda_smooth != 0.0f && (!surfels || !surfels->grid_index || surfels->grid_w <= 0 || surfels->grid_h <= 0))
        return fail(ctx, ROGS_ERR_INVALID, "smoothness loss needs the grid index map");
    if (grads->quat && ((uintptr_t)grads->quat & 15u)) return fail(ctx, ROGS_ERR_INVALID, "grad quat alignment");
    cudaStream_t s = (cudaStream_t)stream;
    static thread_local ViewsArg va;
    long long total_tiles, total_pix;
    std::string err;
    if (!cams || n_views < 1 || n_views > kMaxViews) return fail(ctx, ROGS_ERR_INVALID, "n_views out of range");
    if (!make_views(cfg, cams, n_views, va, total_tiles, total_pix, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    const int n_partials = bwd_loss_partials(total_tiles, cfg.tile_w, cfg.tile_h);
    rogs_status st = ensure_loss(ctx, total_pix, s, (size_t)n_partials);
    if (st == ROGS_OK) st = ensure_rec_grad(ctx, s);
    if (st != ROGS_OK) return st;
    // |M| (the mask count of Eqs. 8-9) and lambda_smooth L_smooth (dz into the
    // gradient, the loss into a scalar the final sum adds) depend only on the
    // inputs: they run on the side stream while the forward renders, and the
    // backward waits for them
    ROGS_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
    ROGS_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    mask_count(tg.mask, total_pix, ctx->loss_counter, ctx->side);
    if (lambda_smooth != 0.0f)
        smooth_loss(surfels->grid_index, surfels->grid_w, surfels->grid_h, surfels->xyz, lambda_smooth,
                    ctx->smooth_val, grads->xyz, ctx->smooth_partials, ctx->side);
    ROGS_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
    st = rogs_render_fwd(ctx, surfels, cams, n_views, exposure_ab, n_exposure, out, state, stream);
    ROGS_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));   // joined even if the forward was refused
    if (st != ROGS_OK) return st;
    const rogs_state_layout L = layout_for(cfg, total_tiles, total_pix);
    const char* sb = (const char*)state;
    const StateHeader* hdr = (const StateHeader*)(sb + L.header);
    const ViewParams* views = (const ViewParams*)(sb + L.views);
    const Record* recs = (const Record*)(sb + L.records);
    const Consts k = make_consts(cfg);
    const SurfelPtrs sp{surfels->xyz, surfels->scale, surfels->quat, surfels->opacity, surfels->rgb, surfels->sem,
                        surfels->n};
    const GradPtrs gp{grads->xyz, grads->scale, grads->quat, grads->opacity, grads->rgb, grads->sem, grads->exposure};
    BwdArgs a{};
    a.views = views; a.n_views = n_views; a.k = k; a.sp = sp; a.recs = recs;
    a.feat = (const float*)(sb + L.rec_feat);
    a.pair_mc = (const float4*)(sb + L.pair_mc);
    a.pair_blk = (const uint8_t*)(sb + L.pair_blk);
    a.pair_rec = (const uint32_t*)(sb + L.pair_rec);
    a.ranges = (const uint2*)(sb + L.tile_range);
    a.tile_order = (const uint32_t*)(sb + L.tile_order);
    a.exposure_ab = exposure_ab;
    a.pix_T = (const float*)(sb + L.pix_T);
    a.pix_last = (const uint32_t*)(sb + L.pix_last);
    a.grad_out = nullptr;
    a.out = out; a.tg = tg; a.mask_count = ctx->loss_counter;
    a.lambda_c = lambda_c; a.lambda_s = lambda_s; a.loss_partials = ctx->loss_partials;
    a.rec_grad = ctx->rec_grad; a.d_exposure = grads->exposure;
    prof_mark(ctx, 6, s);
    composite_bwd(cfg.tile_w, cfg.tile_h, total_tiles, a, s);
    // the final loss sum (its partials are complete) runs on the side stream
    // beside the projection backward; the call's stream waits for both
    ROGS_CUDA(ctx, cudaEventRecord(ctx->ev_fork2, s));
    ROGS_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork2, 0));
    loss_final(ctx->loss_partials, n_partials, ctx->loss_counter, lambda_smooth != 0.0f ? ctx->smooth_val : nullptr,
               loss, ctx->side);
    ROGS_CUDA(ctx, cudaEventRecord(ctx->ev_join2, ctx->side));
    prof_mark(ctx, 7, s);
    project_bwd(views, sp, recs, hdr, (unsigned long long)cfg.record_capacity, ctx->rec_grad, cfg.num_classes, gp, s);
    prof_mark(ctx, -1, s);
    ROGS_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join2, 0));
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

}  // namespace

extern "C" {

rogs_status rogs_train_step(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                            const float* exposure_ab, int32_t n_exposure, float* out, void* state,
                            const float* tgt_rgb, const int32_t* label, const uint8_t* mask, float lambda_c,
                            float lambda_s, float lambda_smooth, float* loss, const rogs_grads* grads,
                            rogs_stream stream) {
    const Targets tg{tgt_rgb, label, nullptr, nullptr, mask};
    return train_step_impl(ctx, surfels, cams, n_views, exposure_ab, n_exposure, out, state, tg, lambda_c, lambda_s,
                           lambda_smooth, loss, grads, stream);
}

rogs_status rogs_train_step_u8(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                               const float* exposure_ab, int32_t n_exposure, float* out, void* state,
                               const uint8_t* tgt_rgb, const uint8_t* label, const uint8_t* mask, float lambda_c,
                               float lambda_s, float lambda_smooth, float* loss, const rogs_grads* grads,
                               rogs_stream stream) {
    if (!tgt_rgb) return ctx ? fail(ctx, ROGS_ERR_INVALID, "null target/loss/grads pointer") : ROGS_ERR_INVALID;
    const Targets tg{nullptr, nullptr, tgt_rgb, label, mask};
    return train_step_impl(ctx, surfels, cams, n_views, exposure_ab, n_exposure, out, state, tg, lambda_c, lambda_s,
                           lambda_smooth, loss, grads, stream);
}

rogs_status rogs_smooth_loss(rogs_ctx* ctx, const rogs_surfels* surfels, float lambda_smooth, float* loss,
                             float* grad_xyz, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (!surfels || !loss || !surfels->xyz) return fail(ctx, ROGS_ERR_INVALID, "null surfels / loss pointer");
    if (!surfels->grid_index || surfels->grid_w <= 0 || surfels->grid_h <= 0)
        return fail(ctx, ROGS_ERR_INVALID, "smoothness loss needs the grid index map");
    cudaStream_t s = (cudaStream_t)stream;
    smooth_loss(surfels->grid_index, surfels->grid_w, surfels->grid_h, surfels->xyz, lambda_smooth, loss, grad_xyz,
                ctx->smooth_partials, s);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

rogs_status rogs_elev_targets(rogs_ctx* ctx, const rogs_surfels* surfels, const float* points, int64_t n_points,
                              float radius, float* z_target, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (!surfels || !z_target || (surfels->n > 0 && !surfels->xyz) || n_points < 0 || (n_points > 0 && !points))
        return fail(ctx, ROGS_ERR_INVALID, "null surfels / points / z_target");
    if (!(radius > 0.0f) || n_points >= (1ll << 31)) return fail(ctx, ROGS_ERR_INVALID, "radius <= 0 or too many points");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t m = (size_t)(n_points > 0 ? n_points : 1);
    const size_t nb = (size_t)1 << lidar_bucket_bits(n_points);
    LidarScratch& w = ctx->lidar;
    rogs_status st = ROGS_OK;
    if (m > ctx->lidar_cap) {
        size_t c[7] = {0, 0, 0, 0, 0, 0, 0};
        if (st == ROGS_OK) st = grow(ctx, w.keys, c[0], m, s);
        if (st == ROGS_OK) st = grow(ctx, w.vals, c[1], m, s);
        if (st == ROGS_OK) st = grow(ctx, w.skeys, c[2], m, s);
        if (st == ROGS_OK) st = grow(ctx, w.svals, c[3], m, s);
        if (st == ROGS_OK) st = grow(ctx, w.kalt, c[4], m, s);
        if (st == ROGS_OK) st = grow(ctx, w.valt, c[5], m, s);
        if (st == ROGS_OK) st = grow(ctx, w.sorted, c[6], m, s);
        if (st != ROGS_OK) return st;
        ctx->lidar_cap = m;
    }
    if (radix_hist_words(m) > ctx->lidar_hist_cap) {
        size_t c = 0;
        st = grow(ctx, w.hist, c, radix_hist_words(m), s);
        if (st != ROGS_OK) return st;
        ctx->lidar_hist_cap = radix_hist_words(m);
    }
    if (nb > ctx->lidar_range_cap) {
        size_t c = 0;
        st = grow(ctx, w.ranges, c, nb, s);
        if (st != ROGS_OK) return st;
        ctx->lidar_range_cap = nb;
    }
    lidar_targets(surfels->xyz, surfels->n, points, n_points, radius, w, z_target, s);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

rogs_status rogs_elev_loss(rogs_ctx* ctx, const rogs_surfels* surfels, const float* z_target, float lambda_z,
                           float* loss, float* grad_xyz, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (!surfels || !z_target || !loss || (surfels->n > 0 && !surfels->xyz))
        return fail(ctx, ROGS_ERR_INVALID, "null surfels / z_target / loss");
    elev_loss(surfels->xyz, surfels->n, z_target, lambda_z, loss, grad_xyz, ctx->elev_partials, (cudaStream_t)stream);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

rogs_status rogs_bev_export(rogs_ctx* ctx, const rogs_surfels* surfels, const float* exposure_ab, int32_t n_exposure,
                            int32_t exposure_idx, double x0, double y1, float res, float cam_z, int32_t width,
                            int32_t height, int32_t chunk, int32_t batch, float* image, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (!surfels || !exposure_ab || !image) return fail(ctx, ROGS_ERR_INVALID, "null surfels / exposure / image");
    if (width < 1 || height < 1 || chunk < 1 || !(res > 0.0f) || batch < 1 || batch > kMaxStitch || batch > kMaxViews)
        return fail(ctx, ROGS_ERR_INVALID, "bad export size, chunk, resolution or batch");
    if (exposure_idx < 0 || exposure_idx >= n_exposure) return fail(ctx, ROGS_ERR_INVALID, "exposure_idx out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const int nch = 3 + ctx->cfg.num_classes + 1;
    const int nx = (width + chunk - 1) / chunk, ny = (height + chunk - 1) / chunk;
    std::vector<rogs_camera> cams;
    std::vector<int> ox, oy;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int cw = std::min(chunk, width - i * chunk), chh = std::min(chunk, height - j * chunk);
            // straight down: image x along +x, image y along -y from the top edge y1
            const double cxw = x0 + ((double)i * chunk + 0.5 * cw) * res;
            const double cyw = y1 - ((double)j * chunk + 0.5 * chh) * res;
            rogs_camera c{};
            c.kind = ROGS_ORTHO;
            c.width = cw;
            c.height = chh;
            c.exposure_idx = exposure_idx;
            c.use_box_cull = 0;
            c.fx = c.fy = (float)(1.0 / res);
            c.cx = 0.5f * (float)cw;
            c.cy = 0.5f * (float)chh;
            const double Rm[9] = {1, 0, 0, 0, -1, 0, 0, 0, -1};
            const double cen[3] = {cxw, cyw, (double)cam_z};
            for (int r = 0; r < 9; ++r) c.R_wc[r] = (float)Rm[r];
            for (int r = 0; r < 3; ++r)
                c.t_wc[r] = (float)-(Rm[3 * r] * cen[0] + Rm[3 * r + 1] * cen[1] + Rm[3 * r + 2] * cen[2]);
            cams.push_back(c);
            ox.push_back(i * chunk);
            oy.push_back(j * chunk);
        }
    // scratch for one batch of full-size chunks
    std::vector<rogs_camera> full(batch, cams[0]);
    for (auto& c : full) { c.width = std::min(chunk, width); c.height = std::min(chunk, height); }
    rogs_state_layout L;
    uint64_t elems = 0;
    rogs_status st = rogs_state_layout_of(ctx, full.data(), batch, &L, &elems);
    if (st != ROGS_OK) return st;
    st = grow(ctx, ctx->bev_out, ctx->bev_out_cap, (size_t)elems, s);
    if (st == ROGS_OK) st = grow(ctx, ctx->bev_state, ctx->bev_state_cap, (size_t)L.total_bytes, s);
    if (st != ROGS_OK) return st;
    for (size_t b0 = 0; b0 < cams.size(); b0 += (size_t)batch) {
        const int nb = (int)std::min<size_t>((size_t)batch, cams.size() - b0);
        st = rogs_render_fwd(ctx, surfels, cams.data() + b0, nb, exposure_ab, n_exposure, ctx->bev_out,
                             ctx->bev_state, stream);
        if (st != ROGS_OK) return st;
        rogs_counts cnt;
        st = rogs_state_counts(ctx, ctx->bev_state, &cnt, stream);   // overflow check (synchronises)
        if (st != ROGS_OK) return st;
        StitchViews sv{};
        long long acc = 0;
        for (int v = 0; v < nb; ++v) {
            const rogs_camera& c = cams[b0 + v];
            acc += (long long)c.width * c.height;
            sv.pix_end[v] = acc;
            sv.w[v] = c.width;
            sv.h[v] = c.height;
            sv.x0[v] = ox[b0 + v];
            sv.y0[v] = oy[b0 + v];
        }
        stitch_views(sv, nb, nch, ctx->bev_out, image, width, height, s);
    }
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

rogs_status rogs_adam_step(rogs_ctx* ctx, const rogs_adam_group* groups, int32_t n_groups, int32_t step, float beta1,
                           float beta2, float eps, int32_t zero_grad, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (!groups || n_groups < 1 || n_groups > ROGS_MAX_ADAM_GROUPS)
        return fail(ctx, ROGS_ERR_INVALID, "n_groups outside [1, ROGS_MAX_ADAM_GROUPS]");
    if (step < 1) return fail(ctx, ROGS_ERR_INVALID, "step must be >= 1");
    for (int i = 0; i < n_groups; ++i) {
        const rogs_adam_group& g = groups[i];
        if (g.n < 0 || g.stride < 1) return fail(ctx, ROGS_ERR_INVALID, "group with n < 0 or stride < 1");
        if (g.zero_lead < 0 || g.zero_lead >= g.stride)
            return fail(ctx, ROGS_ERR_INVALID, "group with zero_lead outside [0, stride)");
        if (g.decay_steps < 0 || (g.decay_steps > 0 && !(g.lr > 0.0f && g.lr_end > 0.0f)))
            return fail(ctx, ROGS_ERR_INVALID, "group with decay_steps < 0, or a decay without positive lr and lr_end");
        if (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v)) return fail(ctx, ROGS_ERR_INVALID, "null group pointer");
    }
    adam_step(groups, n_groups, step, beta1, beta2, eps, zero_grad != 0, (cudaStream_t)stream);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

rogs_status rogs_sort_pairs(rogs_ctx* ctx, const uint32_t* keys_in, const uint32_t* vals_in, int64_t n,
                            int32_t key_bits, uint32_t* keys_out, uint32_t* vals_out, rogs_stream stream) {
    if (!ctx) return ROGS_ERR_INVALID;
    if (n < 0 || n > ctx->cfg.pair_capacity) return fail(ctx, ROGS_ERR_INVALID, "n outside [0, pair_capacity]");
    if (key_bits < 0 || key_bits > 32) return fail(ctx, ROGS_ERR_INVALID, "key_bits outside [0, 32]");
    if (n == 0) return ROGS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return fail(ctx, ROGS_ERR_INVALID, "null device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, ctx->pk_c, ctx->pv_c, nullptr, (unsigned long long)n,
                     key_bits, ctx->hist, s, ctx->cfg.sort_tile);
    ROGS_CUDA(ctx, cudaGetLastError());
    return ROGS_OK;
}

static rogs_status finish_capture(rogs_ctx* ctx, cudaStream_t s, rogs_status st, rogs_graph** out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != ROGS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || !g) return fail(ctx, ROGS_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ctx, ROGS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    rogs_graph* gr = new rogs_graph();
    gr->graph = g;
    gr->exec = exec;
    *out = gr;
    return ROGS_OK;
}

static rogs_status begin_capture(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                                 cudaStream_t s, bool with_loss) {
    if (!s) return fail(ctx, ROGS_ERR_INVALID, "graph capture needs a non-default stream");
    if (!surfels || !cams || n_views < 1 || n_views > kMaxViews) return fail(ctx, ROGS_ERR_INVALID, "bad arguments");
    static thread_local ViewsArg va;
    long long tt, tp;
    std::string err;
    if (!make_views(ctx->cfg, cams, n_views, va, tt, tp, err)) return fail(ctx, ROGS_ERR_INVALID, err);
    rogs_status st = ensure_bits(ctx, surfels->n, n_views, s);   // size scratch before capturing
    if (st == ROGS_OK && with_loss)
        st = ensure_loss(ctx, tp, s, (size_t)bwd_loss_partials(tt, ctx->cfg.tile_w, ctx->cfg.tile_h));
    if (st == ROGS_OK && with_loss) st = ensure_rec_grad(ctx, s);
    if (st != ROGS_OK) return st;
    ROGS_CUDA(ctx, cudaStreamSynchronize(s));
    ROGS_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    return ROGS_OK;
}

rogs_status rogs_train_graph_create(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                                    int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                                    void* state, const float* tgt_rgb, const int32_t* label, const uint8_t* mask,
                                    float lambda_c, float lambda_s, float lambda_smooth, float* loss,
                                    const rogs_grads* grads,
                                    rogs_stream stream, rogs_graph** gout) {
    if (!ctx || !gout) return ROGS_ERR_INVALID;
    *gout = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rogs_status st = begin_capture(ctx, surfels, cams, n_views, s, true);
    if (st != ROGS_OK) return st;
    st = rogs_train_step(ctx, surfels, cams, n_views, exposure_ab, n_exposure, out, state, tgt_rgb, label, mask,
                         lambda_c, lambda_s, lambda_smooth, loss, grads, stream);
    return finish_capture(ctx, s, st, gout);
}

rogs_status rogs_train_graph_create_u8(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                                       int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                                       void* state, const uint8_t* tgt_rgb, const uint8_t* label, const uint8_t* mask,
                                       float lambda_c, float lambda_s, float lambda_smooth, float* loss,
                                       const rogs_grads* grads, rogs_stream stream, rogs_graph** gout) {
    if (!ctx || !gout) return ROGS_ERR_INVALID;
    *gout = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rogs_status st = begin_capture(ctx, surfels, cams, n_views, s, true);
    if (st != ROGS_OK) return st;
    st = rogs_train_step_u8(ctx, surfels, cams, n_views, exposure_ab, n_exposure, out, state, tgt_rgb, label, mask,
                            lambda_c, lambda_s, lambda_smooth, loss, grads, stream);
    return finish_capture(ctx, s, st, gout);
}

rogs_status rogs_render_graph_create(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                                     int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                                     void* state, rogs_stream stream, rogs_graph** gout) {
    if (!ctx || !gout) return ROGS_ERR_INVALID;
    *gout = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rogs_status st = begin_capture(ctx, surfels, cams, n_views, s, false);
    if (st != ROGS_OK) return st;
    st = rogs_render_fwd(ctx, surfels, cams, n_views, exposure_ab, n_exposure, out, state, stream);
    return finish_capture(ctx, s, st, gout);
}

rogs_status rogs_graph_launch(rogs_graph* graph, rogs_stream stream) {
    if (!graph || !graph->exec) return ROGS_ERR_INVALID;
    if (cudaGraphLaunch(graph->exec, (cudaStream_t)stream) != cudaSuccess) return ROGS_ERR_CUDA;
    return ROGS_OK;
}

void rogs_graph_destroy(rogs_graph* graph) {
    if (!graph) return;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
}

rogs_status rogs_profile_enable(rogs_ctx* ctx, int32_t enable) {
    if (!ctx) return ROGS_ERR_INVALID;
    rogs_profile tmp;
    rogs_status st = rogs_profile_read(ctx, &tmp);  // drain pending events
    ctx->prof = enable != 0;
    for (int i = 0; i < ROGS_N_STAGES; ++i) {
        ctx->prof_ms[i] = 0.0;
        ctx->prof_calls[i] = 0;
    }
    return st;
}

rogs_status rogs_profile_read(rogs_ctx* ctx, rogs_profile* out) {
    if (!ctx || !out) return ROGS_ERR_INVALID;
    for (const ProfEvent& pe : ctx->prof_pending) {
        cudaError_t e = cudaEventSynchronize(pe.b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pe.a, pe.b);
        if (e == cudaSuccess) {
            ctx->prof_ms[pe.stage] += ms;
            ctx->prof_calls[pe.stage] += 1;
        }
        ctx->prof_pool.push_back(pe.a);
        ctx->prof_pool.push_back(pe.b);
    }
    ctx->prof_pending.clear();
    for (int i = 0; i < ROGS_N_STAGES; ++i) {
        out->ms[i] = ctx->prof_ms[i];
        out->calls[i] = ctx->prof_calls[i];
    }
    return ROGS_OK;
}

uint64_t rogs_launch_count(void) { return (uint64_t)g_launches.load(); }

}  // extern "C"
