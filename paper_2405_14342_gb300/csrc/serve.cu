// serve.cu -- continuous-batching request loop over a resident surfel map.
//
// The worker thread owns max_inflight (context, stream) slots and a device
// pool of memory_budget bytes.  It forms batches from the pending FIFO
// (admission: a batch grows while the next request fits the free pool and the
// free pinned staging), renders each batch with one rogs_render_fwd call over
// all its views, packs every request's channels (serve_pack_k) and copies
// them to pinned host memory, then records an event.  Completion is detected
// by polling the events; a finished batch returns its device memory at once,
// and the next batch can start while others are still on the GPU.  Host-side
// waits are bounded by timeout_s; no kernel here waits on anything.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"

namespace rogs {

struct PackReq {
    long long pix_base;
    unsigned long long dst_off;   // byte offset of the request's packed result
    int W, H, channels, kind;
    float cam_z;
    int pad;
};

struct PackArg {
    PackReq r[kMaxViews];
};

// Pack the requested channels of every request of a batch:
// RGB float [3][H][W], ELEV float [H][W], SEM uint8 [H][W] (argmax).
__global__ void __launch_bounds__(256) serve_pack_k(PackArg pa, int n_req, long long total_pix, int C,
                                                    const float* __restrict__ out, const float* __restrict__ pix_T,
                                                    unsigned char* __restrict__ packed) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total_pix;
         p += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_req - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pa.r[mid].pix_base <= p) lo = mid; else hi = mid - 1;
        }
        const PackReq& r = pa.r[lo];
        const long long q = p - r.pix_base;
        const long long plane = (long long)r.W * r.H;
        const int nch = 3 + C + 1;
        const float* o = out + (long long)nch * r.pix_base + q;
        unsigned char* dst = packed + r.dst_off;
        long long off = 0;
        if (r.channels & ROGS_CH_RGB) {
            float* d = reinterpret_cast<float*>(dst);
            d[q] = o[0];
            d[plane + q] = o[plane];
            d[2 * plane + q] = o[2 * plane];
            off += 12 * plane;
        }
        if (r.channels & ROGS_CH_ELEV) {
            const float cov = 1.0f - pix_T[p];
            const float D = o[(3 + C) * plane];
            float e = __int_as_float(0x7fc00000);   // NaN where the surface is not covered
            if (cov >= 0.5f) e = (r.kind == ROGS_ORTHO) ? r.cam_z - D / cov : D / cov;
            reinterpret_cast<float*>(dst + off)[q] = e;
            off += 4 * plane;
        }
        if (r.channels & ROGS_CH_SEM) {
            int best = 0;
            float bv = C > 0 ? o[3 * plane] : 0.0f;
            for (int c = 1; c < C; ++c) {
                const float x = o[(3 + c) * plane];
                if (x > bv) { bv = x; best = c; }
            }
            dst[off + q] = (unsigned char)best;
        }
    }
}

// First-fit allocator over [0, size) with coalescing (host bookkeeping only).
class Arena {
public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (!bytes) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (!bytes) bytes = 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }
    size_t size() const { return size_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

}  // namespace rogs

using namespace rogs;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kStPending = 0, kStInflight = 1, kStDone = 2, kStFailed = 3;

struct Request {
    uint64_t id;
    rogs_camera cam;
    int channels;
    size_t result_bytes;
    size_t pinned_off = 0;
    bool has_pinned = false;
    int state = kStPending;
    rogs_status err = ROGS_OK;
};

struct Batch {
    int slot;
    std::vector<uint64_t> ids;
    std::vector<std::pair<size_t, size_t>> pinned_hold;   // results of timed-out requests, freed at completion
    size_t dev_off = 0, dev_bytes = 0;
    size_t hdr_pinned_off = 0;
    cudaEvent_t done = nullptr;
    Clock::time_point launched;
};

size_t request_result_bytes(const rogs_camera& c, int channels) {
    const size_t P = (size_t)c.width * (size_t)c.height;
    size_t b = 0;
    if (channels & ROGS_CH_RGB) b += 12 * P;
    if (channels & ROGS_CH_ELEV) b += 4 * P;
    if (channels & ROGS_CH_SEM) b += P;
    return b;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct rogs_server {
    rogs_serve_config cfg;
    rogs_config rcfg;
    rogs_surfels map;
    const float* exposure = nullptr;
    int n_exposure = 0;
    int device = 0;
    int C = 0;
    std::vector<rogs_ctx*> ctxs;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    unsigned char* pool = nullptr;
    unsigned char* pinned = nullptr;
    Arena dev_arena, pin_arena;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::list<Batch> inflight;
    rogs_serve_stats stats{};

    // device bytes of a batch with these cameras: outputs + state + packed results
    bool batch_bytes(const std::vector<rogs_camera>& cams, const std::vector<int>& chans, size_t* out_bytes,
                     size_t* state_bytes, size_t* packed_bytes) {
        rogs_state_layout L;
        uint64_t elems = 0;
        if (rogs_state_layout_of(ctxs[0], cams.data(), (int)cams.size(), &L, &elems) != ROGS_OK) return false;
        *out_bytes = al256(4 * (size_t)elems);
        *state_bytes = al256((size_t)L.total_bytes);
        size_t pk = 0;
        for (size_t i = 0; i < cams.size(); ++i) pk += al256(request_result_bytes(cams[i], chans[i]));
        *packed_bytes = pk;
        return true;
    }

    void finish(Batch& b, rogs_status st) {
        const rogs_counts* hdr = reinterpret_cast<const rogs_counts*>(pinned + b.hdr_pinned_off);
        if (st == ROGS_OK && hdr->status) st = ROGS_ERR_CAPACITY;
        for (uint64_t id : b.ids) {
            auto it = reqs.find(id);
            if (it == reqs.end()) continue;
            Request& r = it->second;
            if (st == ROGS_OK) {
                r.state = kStDone;
                stats.completed++;
            } else {
                r.state = kStFailed;
                r.err = st;
                stats.failed++;
                if (r.has_pinned) {
                    pin_arena.release(r.pinned_off, r.result_bytes);
                    r.has_pinned = false;
                }
            }
        }
        for (auto& h : b.pinned_hold) pin_arena.release(h.first, h.second);
        b.pinned_hold.clear();
        pin_arena.release(b.hdr_pinned_off, sizeof(rogs_counts));
        dev_arena.release(b.dev_off, b.dev_bytes);
        slot_busy[b.slot] = false;
        stats.inflight--;
    }

    // Try to start one batch; returns true if one was launched.
    bool admit() {
        int slot = -1;
        for (size_t i = 0; i < slot_busy.size(); ++i)
            if (!slot_busy[i]) { slot = (int)i; break; }
        if (slot < 0 || pending.empty()) return false;
        std::vector<rogs_camera> cams;
        std::vector<int> chans;
        std::vector<uint64_t> ids;
        size_t ob = 0, sb = 0, pb = 0, pin_need = 0;
        const size_t dev_free = dev_arena.largest();
        const size_t pin_free = pin_arena.largest();
        for (uint64_t id : pending) {
            if ((int)cams.size() >= cfg.max_batch_views) break;
            const Request& r = reqs[id];
            cams.push_back(r.cam);
            chans.push_back(r.channels);
            size_t o2, s2, p2;
            if (!batch_bytes(cams, chans, &o2, &s2, &p2) || o2 + s2 + p2 > dev_free ||
                pin_need + al256(r.result_bytes) + 256 > pin_free) {
                cams.pop_back();
                chans.pop_back();
                break;
            }
            ob = o2; sb = s2; pb = p2;
            pin_need += al256(r.result_bytes);
            ids.push_back(id);
        }
        if (ids.empty()) return false;   // the head request waits for memory
        Batch b;
        b.slot = slot;
        b.ids = ids;
        b.dev_bytes = ob + sb + pb;
        if (!dev_arena.alloc(b.dev_bytes, &b.dev_off)) return false;
        if (!pin_arena.alloc(sizeof(rogs_counts), &b.hdr_pinned_off)) {
            dev_arena.release(b.dev_off, b.dev_bytes);
            return false;
        }
        for (uint64_t id : ids) {
            Request& r = reqs[id];
            if (!pin_arena.alloc(r.result_bytes, &r.pinned_off)) {   // cannot happen: checked above
                r.has_pinned = false;
            } else {
                r.has_pinned = true;
            }
        }
        for (size_t i = 0; i < ids.size(); ++i) pending.pop_front();
        float* out = reinterpret_cast<float*>(pool + b.dev_off);
        void* state = pool + b.dev_off + ob;
        unsigned char* packed = pool + b.dev_off + ob + sb;
        cudaStream_t s = streams[slot];
        rogs_status st = rogs_render_fwd(ctxs[slot], &map, cams.data(), (int)cams.size(), exposure, n_exposure, out,
                                         state, s);
        rogs_state_layout L;
        uint64_t elems = 0;
        rogs_state_layout_of(ctxs[slot], cams.data(), (int)cams.size(), &L, &elems);
        if (st == ROGS_OK) {
            static thread_local PackArg pa;
            long long pix = 0;
            size_t doff = 0;
            for (size_t i = 0; i < cams.size(); ++i) {
                PackReq& q = pa.r[i];
                q.pix_base = pix;
                q.dst_off = doff;
                q.W = cams[i].width;
                q.H = cams[i].height;
                q.channels = chans[i];
                q.kind = cams[i].kind;
                const float* R = cams[i].R_wc;
                const float* t = cams[i].t_wc;
                q.cam_z = (float)(-((double)R[2] * t[0] + (double)R[5] * t[1] + (double)R[8] * t[2]));
                q.pad = 0;
                pix += (long long)cams[i].width * cams[i].height;
                doff += al256(request_result_bytes(cams[i], chans[i]));
            }
            long long blocks = (pix + 255) / 256;
            if (blocks > 152 * 8) blocks = 152 * 8;
            launch_pdl(serve_pack_k, dim3((int)(blocks > 0 ? blocks : 1)), dim3(256), 0, s,
                pa, (int)cams.size(), pix, C, out, reinterpret_cast<const float*>((char*)state + L.pix_T), packed);
            note_launches(1);
            doff = 0;
            for (size_t i = 0; i < ids.size(); ++i) {
                Request& r = reqs[ids[i]];
                if (r.has_pinned && r.result_bytes)
                    cudaMemcpyAsync(pinned + r.pinned_off, packed + doff, r.result_bytes, cudaMemcpyDeviceToHost, s);
                doff += al256(r.result_bytes);
            }
            cudaMemcpyAsync(pinned + b.hdr_pinned_off, state, sizeof(rogs_counts), cudaMemcpyDeviceToHost, s);
            if (cudaGetLastError() != cudaSuccess) st = ROGS_ERR_CUDA;
        }
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
        cudaEventRecord(b.done, s);
        b.launched = Clock::now();
        slot_busy[slot] = true;
        stats.inflight++;
        stats.batches++;
        stats.views_rendered += cams.size();
        for (auto& c : cams) stats.pixels_rendered += (uint64_t)c.width * c.height;
        for (uint64_t id : ids) reqs[id].state = kStInflight;
        stats.pending = (uint32_t)pending.size();
        if (st != ROGS_OK) {
            cudaEventSynchronize(b.done);
            cudaEventDestroy(b.done);
            reinterpret_cast<rogs_counts*>(pinned + b.hdr_pinned_off)->status = 0;
            finish(b, st);
            return true;
        }
        inflight.push_back(b);
        return true;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progress = false;
            for (auto it = inflight.begin(); it != inflight.end();) {
                const cudaError_t q = cudaEventQuery(it->done);
                const double age = std::chrono::duration<double>(Clock::now() - it->launched).count();
                if (q == cudaSuccess || (q != cudaErrorNotReady)) {
                    finish(*it, q == cudaSuccess ? ROGS_OK : ROGS_ERR_CUDA);
                    cudaEventDestroy(it->done);
                    it = inflight.erase(it);
                    progress = true;
                } else if (age > cfg.timeout_s) {
                    // give up on the requests; the memory stays held until the GPU is done with it
                    for (uint64_t id : it->ids) {
                        auto r = reqs.find(id);
                        if (r != reqs.end() && r->second.state == kStInflight) {
                            r->second.state = kStFailed;
                            r->second.err = ROGS_ERR_TIMEOUT;
                            if (r->second.has_pinned) {   // the copy may still land there
                                it->pinned_hold.emplace_back(r->second.pinned_off, r->second.result_bytes);
                                r->second.has_pinned = false;
                            }
                            stats.failed++;
                        }
                    }
                    it->ids.clear();
                    it->launched = Clock::now() + std::chrono::hours(24 * 365);
                    ++it;
                } else {
                    ++it;
                }
            }
            if (stop) {
                if (inflight.empty()) break;
            } else {
                while (admit()) progress = true;
            }
            stats.pending = (uint32_t)pending.size();
            if (!progress) cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
};

extern "C" {

rogs_status rogs_serve_result_bytes(const rogs_camera* cam, int32_t channels, int32_t num_classes, uint64_t* bytes) {
    (void)num_classes;
    if (!cam || !bytes || channels <= 0 || channels > 7 || cam->width <= 0 || cam->height <= 0)
        return ROGS_ERR_INVALID;
    *bytes = request_result_bytes(*cam, channels);
    return ROGS_OK;
}

rogs_status rogs_serve_open(const rogs_config* cfg_render, const rogs_surfels* map, const float* exposure_ab,
                            int32_t n_exposure, const rogs_serve_config* cfg, rogs_server** out) {
    if (!cfg_render || !map || !exposure_ab || n_exposure < 1 || !cfg || !out) return ROGS_ERR_INVALID;
    *out = nullptr;
    if (cfg->max_batch_views < 1 || cfg->max_batch_views > ROGS_MAX_VIEWS || cfg->max_inflight < 1 ||
        cfg->max_inflight > 16 || cfg->max_queue < 1 || cfg->memory_budget < (1ull << 20) || !(cfg->timeout_s > 0))
        return ROGS_ERR_INVALID;
    rogs_server* srv = new rogs_server();
    srv->cfg = *cfg;
    srv->rcfg = *cfg_render;
    srv->rcfg.record_capacity = cfg->record_capacity;
    srv->rcfg.pair_capacity = cfg->pair_capacity;
    srv->map = *map;
    srv->exposure = exposure_ab;
    srv->n_exposure = n_exposure;
    srv->C = cfg_render->num_classes;
    cudaGetDevice(&srv->device);
    rogs_status st = ROGS_OK;
    for (int i = 0; i < cfg->max_inflight && st == ROGS_OK; ++i) {
        rogs_ctx* c = nullptr;
        st = rogs_create(&srv->rcfg, &c);
        if (st == ROGS_OK) {
            srv->ctxs.push_back(c);
            st = rogs_reserve(c, map->n, nullptr, cfg->max_batch_views, 0);
        }
        cudaStream_t s = nullptr;
        if (st == ROGS_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = ROGS_ERR_CUDA;
        if (st == ROGS_OK) {
            srv->streams.push_back(s);
            srv->slot_busy.push_back(false);
        }
    }
    if (st == ROGS_OK && (rogs::debug_alloc_fails() || cudaMalloc((void**)&srv->pool, cfg->memory_budget) != cudaSuccess))
        st = ROGS_ERR_OOM;
    const size_t pin_size = cfg->memory_budget / 4 + (1u << 20);
    if (st == ROGS_OK && cudaHostAlloc((void**)&srv->pinned, pin_size, cudaHostAllocDefault) != cudaSuccess)
        st = ROGS_ERR_OOM;
    if (st != ROGS_OK) {
        for (auto c : srv->ctxs) rogs_destroy(c);
        for (auto s : srv->streams) cudaStreamDestroy(s);
        if (srv->pool) cudaFree(srv->pool);
        if (srv->pinned) cudaFreeHost(srv->pinned);
        delete srv;
        return st;
    }
    srv->dev_arena.reset(cfg->memory_budget);
    srv->pin_arena.reset(pin_size);
    srv->worker = std::thread([srv] { srv->run(); });
    *out = srv;
    return ROGS_OK;
}

rogs_status rogs_serve_submit(rogs_server* srv, const rogs_camera* cam, int32_t channels, uint64_t* ticket) {
    if (!srv || !cam || !ticket || channels <= 0 || channels > 7) return ROGS_ERR_INVALID;
    std::vector<rogs_camera> one{*cam};
    std::vector<int> ch{channels};
    std::lock_guard<std::mutex> lk(srv->mu);
    if (cam->exposure_idx < 0 || cam->exposure_idx >= srv->n_exposure) return ROGS_ERR_INVALID;
    size_t ob, sb, pb;
    if (!srv->batch_bytes(one, ch, &ob, &sb, &pb)) return ROGS_ERR_INVALID;
    if (ob + sb + pb > srv->dev_arena.size() || al256(request_result_bytes(*cam, channels)) + 512 > srv->pin_arena.size())
        return ROGS_ERR_OOM;
    if ((int)srv->pending.size() >= srv->cfg.max_queue) return ROGS_ERR_BUSY;
    Request r;
    r.id = srv->next_id++;
    r.cam = *cam;
    r.channels = channels;
    r.result_bytes = request_result_bytes(*cam, channels);
    srv->reqs.emplace(r.id, r);
    srv->pending.push_back(r.id);
    srv->stats.submitted++;
    srv->stats.pending = (uint32_t)srv->pending.size();
    *ticket = r.id;
    srv->cv.notify_one();
    return ROGS_OK;
}

rogs_status rogs_serve_poll(rogs_server* srv, uint64_t ticket, void* host_out, int32_t* done) {
    if (!srv || !done) return ROGS_ERR_INVALID;
    *done = 0;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return ROGS_ERR_INVALID;
    Request& r = it->second;
    if (r.state == kStFailed) {
        const rogs_status e = r.err;
        srv->reqs.erase(it);
        return e;
    }
    if (r.state != kStDone) return ROGS_ERR_NOT_READY;
    if (r.result_bytes && !host_out) return ROGS_ERR_INVALID;
    if (r.result_bytes) std::memcpy(host_out, srv->pinned + r.pinned_off, r.result_bytes);
    if (r.has_pinned) srv->pin_arena.release(r.pinned_off, r.result_bytes);
    srv->reqs.erase(it);
    *done = 1;
    return ROGS_OK;
}

rogs_status rogs_serve_get_stats(rogs_server* srv, rogs_serve_stats* out) {
    if (!srv || !out) return ROGS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    return ROGS_OK;
}

rogs_status rogs_serve_set_timeout(rogs_server* srv, double timeout_s) {
    if (!srv || !(timeout_s > 0)) return ROGS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->cfg.timeout_s = timeout_s;
    return ROGS_OK;
}

void rogs_serve_close(rogs_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->pending.clear();
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (auto c : srv->ctxs) rogs_destroy(c);
    for (auto s : srv->streams) cudaStreamDestroy(s);
    if (srv->pool) cudaFree(srv->pool);
    if (srv->pinned) cudaFreeHost(srv->pinned);
    delete srv;
}

}  // extern "C"
