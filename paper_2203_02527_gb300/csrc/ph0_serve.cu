// ph0_serve.cu -- serving context of the C ABI (ph0_ctx_*, ph0_submit,
// ph0_poll, ph0_release): a request loop that admits point clouds of any
// N and d as they arrive, by device-memory budget, and keeps several on the
// GPU at once.  The paper has no counterpart (its experiments run one cloud
// at a time, Sec. 3.1, Sec. 4.1); the per-cloud computation is the same path
// and gives the same bits alone and in the mix.
//
//  * One device arena and one pinned host pool are allocated at creation;
//    every request's device buffers (points, bars, workspace) and host copies
//    come from them (first-fit, coalescing).  A request is admitted when its
//    buffers fit: memory frees as earlier requests complete.
//  * Large clouds run the multi-kernel path on one of `streams` CUDA streams,
//    so that several overlap on the device.
//  * Small clouds (n <= small_max_n) are grouped into batches computed by the
//    fused one-CTA-per-cloud kernel in a single launch, replayed from a
//    captured CUDA graph (the task count is read on the device).
//  * A worker thread completes requests (event queries), frees their memory
//    and admits the next ones; ph0_poll returns finished results, whose bars
//    stay in the pinned pool until ph0_release.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ph0_common.cuh"

namespace ph0 {

cudaError_t prepare_small_kernel();
cudaError_t launch_small(const SmallTask *tasks, const int32_t *ntasks_dev, uint32_t *counter, int grid,
                         cudaStream_t s);
int small_max_n();
int small_max_d();
int sm_count();
int barcodes_whole(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                   ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream, const ph0_tuning *tuning,
                   bool fallback);

namespace {

// First-fit allocator over [0, size) with coalescing; offsets 256-aligned.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t bytes, size_t &off) {
        bytes = align_up(bytes ? bytes : 1, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes ? bytes : 1, 256);
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

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

struct Request {
    uint64_t tag = 0;
    int32_t n = 0, d = 0;
    int32_t status = PH0_OK;
    int32_t inf_vertex = 0;
    bool small = false;
    bool full = false;  // run with the complete sort's fallback (after its flag was seen)
    // pinned host: [points | bars | status words: status, infinite bar's vertex, fallback flag]
    size_t h_off = 0, h_bytes = 0;
    // device: [points | bars | workspace or fixed-point scratch | status]
    size_t d_off = 0, d_bytes = 0;
    size_t ws_bytes = 0;
    int slot = -1;
    double t_submit = 0, t_done = 0;
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace ph0

using namespace ph0;

struct ph0_ctx {
    ph0_options opt{};
    int device = 0;
    char *dev = nullptr;        // device arena
    char *host = nullptr;       // pinned host pool
    Arena dev_arena, host_arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<Request *> slot_req;   // large request per stream slot
    // small batches
    cudaStream_t small_stream = nullptr;
    cudaEvent_t small_event = nullptr;
    SmallTask *d_tasks = nullptr;      // device task table [batch_max]
    SmallTask *h_tasks = nullptr;      // pinned staging of the table
    int32_t *d_ntasks = nullptr, *h_ntasks = nullptr;
    uint32_t *d_counter = nullptr;
    cudaGraphExec_t small_graph = nullptr;
    std::vector<Request *> small_batch;  // in flight
    // requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> by_tag;
    std::deque<Request *> finished;      // not yet returned by poll
    bool stop = false;
    std::thread worker;
    cudaError_t error = cudaSuccess;

    ph0_bar *bars_host(Request *r) {
        return reinterpret_cast<ph0_bar *>(host + r->h_off + align_up(size_t(r->n) * r->d * 4, 256));
    }
    float *pts_host(Request *r) { return reinterpret_cast<float *>(host + r->h_off); }
    int32_t *status_host(Request *r) {
        return reinterpret_cast<int32_t *>(host + r->h_off + align_up(size_t(r->n) * r->d * 4, 256) +
                                           align_up(size_t(r->n > 1 ? r->n - 1 : 1) * sizeof(ph0_bar), 256));
    }

    static size_t host_bytes(int64_t n, int32_t d) {
        return align_up(size_t(n) * d * 4, 256) + align_up(size_t(n > 1 ? n - 1 : 1) * sizeof(ph0_bar), 256) + 256;
    }
    size_t dev_bytes(const Request &r) const {
        const size_t pts = align_up(size_t(r.n) * r.d * 4, 256);
        const size_t bars = align_up(size_t(r.n > 1 ? r.n - 1 : 1) * sizeof(ph0_bar), 256);
        const size_t work = r.small ? align_up(size_t(r.n) * r.d * 8, 256) : r.ws_bytes;
        return pts + bars + work + 256;
    }

    // a request whose device work finished: its status and the vertex of its
    // infinite bar, both written by the device into the pinned pool
    void complete_ok(Request *r) {
        r->inf_vertex = status_host(r)[1];
        complete(r, status_host(r)[0]);
    }

    void complete(Request *r, int32_t status) {
        r->status = status;
        r->t_done = now_s();
        dev_arena.release(r->d_off, r->d_bytes);
        finished.push_back(r);
    }

    // Launch one large request on stream slot `k`.  The first launch leaves
    // out the whole path's gated fallback (about 14 launches that return at
    // once on almost every cloud) and copies the fix-up's fallback flag back
    // with the status; a request whose flag is set runs again in full
    // before it completes, so every result is still exact.
    cudaError_t launch_large(Request *r, int k) {
        cudaStream_t s = streams[k];
        char *base = dev + r->d_off;
        float *d_pts = reinterpret_cast<float *>(base);
        ph0_bar *d_bars = reinterpret_cast<ph0_bar *>(base + align_up(size_t(r->n) * r->d * 4, 256));
        void *ws = base + align_up(size_t(r->n) * r->d * 4, 256) +
                   align_up(size_t(r->n > 1 ? r->n - 1 : 1) * sizeof(ph0_bar), 256);
        cudaError_t e = cudaMemcpyAsync(d_pts, pts_host(r), size_t(r->n) * r->d * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        const int rc = barcodes_whole(d_pts, r->n, r->d, r->d, d_bars, nullptr, ws, r->ws_bytes, s, nullptr, r->full);
        if (rc != PH0_OK) return cudaErrorUnknown;
        if (r->n > 1)
            e = cudaMemcpyAsync(bars_host(r), d_bars, size_t(r->n - 1) * sizeof(ph0_bar), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(status_host(r), ws, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                s);  // header: status, vertex of the infinite bar
        status_host(r)[2] = 0;
        if (e == cudaSuccess && !r->full)
            e = cudaMemcpyAsync(status_host(r) + 2, &at<Header>(ws, Layout(r->n, r->d).hdr)->fixup_fallback,
                                sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(events[k], s);
        return e;
    }

    // Launch the current small batch (graph replay).
    cudaError_t launch_small_batch() {
        const int nt = int(small_batch.size());
        for (int i = 0; i < nt; ++i) {
            Request *r = small_batch[i];
            char *base = dev + r->d_off;
            SmallTask &t = h_tasks[i];
            t.pts = reinterpret_cast<const float *>(base);
            t.bars = reinterpret_cast<ph0_bar *>(base + align_up(size_t(r->n) * r->d * 4, 256));
            t.fixed = reinterpret_cast<int64_t *>(base + align_up(size_t(r->n) * r->d * 4, 256) +
                                                  align_up(size_t(r->n > 1 ? r->n - 1 : 1) * sizeof(ph0_bar), 256));
            t.status = reinterpret_cast<int32_t *>(base + r->d_bytes - 256);
            t.n = r->n;
            t.d = r->d;
            t.ld = r->d;
            t.pad = 0;
            cudaError_t e = cudaMemcpyAsync(const_cast<float *>(t.pts), pts_host(r), size_t(r->n) * r->d * 4,
                                            cudaMemcpyHostToDevice, small_stream);
            if (e != cudaSuccess) return e;
        }
        *h_ntasks = nt;
        cudaError_t e = cudaMemcpyAsync(d_tasks, h_tasks, sizeof(SmallTask) * nt, cudaMemcpyHostToDevice, small_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_ntasks, h_ntasks, sizeof(int32_t), cudaMemcpyHostToDevice, small_stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(small_graph, small_stream);
        for (int i = 0; i < nt && e == cudaSuccess; ++i) {
            Request *r = small_batch[i];
            if (r->n > 1)
                e = cudaMemcpyAsync(bars_host(r), h_tasks[i].bars, size_t(r->n - 1) * sizeof(ph0_bar),
                                    cudaMemcpyDeviceToHost, small_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(status_host(r), h_tasks[i].status, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    small_stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(small_event, small_stream);
        return e;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            bool busy = false;
            // ---- completions ----
            for (size_t k = 0; k < streams.size(); ++k) {
                Request *r = slot_req[k];
                if (!r) continue;
                busy = true;
                const cudaError_t q = cudaEventQuery(events[k]);
                if (q == cudaErrorNotReady) continue;
                if (q == cudaSuccess && !r->full && status_host(r)[0] == PH0_OK && status_host(r)[2] != 0) {
                    r->full = true;  // crowded distances: the complete sort, on the same slot
                    const cudaError_t e = launch_large(r, int(k));
                    if (e == cudaSuccess) continue;
                    error = e;
                    complete(r, PH0_ECUDA);
                } else if (q == cudaSuccess) {
                    complete_ok(r);
                } else {
                    complete(r, PH0_ECUDA);
                }
                slot_req[k] = nullptr;
                cv_done.notify_all();
            }
            if (!small_batch.empty()) {
                busy = true;
                const cudaError_t q = cudaEventQuery(small_event);
                if (q != cudaErrorNotReady) {
                    for (Request *r : small_batch) {
                        if (q == cudaSuccess) complete_ok(r);
                        else complete(r, PH0_ECUDA);
                    }
                    small_batch.clear();
                    cv_done.notify_all();
                }
            }
            // ---- admissions, in arrival order ----
            if (small_batch.empty()) {
                for (auto it = pending.begin(); it != pending.end() && int(small_batch.size()) < opt.batch_max;) {
                    Request *r = *it;
                    if (!r->small) { ++it; continue; }
                    r->d_bytes = dev_bytes(*r);
                    if (!dev_arena.alloc(r->d_bytes, r->d_off)) break;
                    small_batch.push_back(r);
                    it = pending.erase(it);
                }
                if (!small_batch.empty()) {
                    busy = true;
                    cudaError_t e = launch_small_batch();
                    if (e != cudaSuccess) {
                        error = e;
                        cudaStreamSynchronize(small_stream);
                        for (Request *r : small_batch) complete(r, PH0_ECUDA);
                        small_batch.clear();
                        cv_done.notify_all();
                    }
                }
            }
            for (size_t k = 0; k < streams.size(); ++k) {
                if (slot_req[k]) continue;
                auto it = pending.begin();
                while (it != pending.end() && (*it)->small) ++it;
                if (it == pending.end()) break;
                Request *r = *it;
                r->d_bytes = dev_bytes(*r);
                if (!dev_arena.alloc(r->d_bytes, r->d_off)) break;  // wait for memory
                pending.erase(it);
                slot_req[k] = r;
                r->slot = int(k);
                busy = true;
                cudaError_t e = launch_large(r, int(k));
                if (e != cudaSuccess) {
                    error = e;
                    complete(r, PH0_ECUDA);
                    slot_req[k] = nullptr;
                    cv_done.notify_all();
                }
            }
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
};

extern "C" {

int ph0_ctx_create(const ph0_options *opt, ph0_ctx **out) {
    if (!opt || !out || opt->mem_budget < (size_t(1) << 20) || opt->host_budget < (size_t(1) << 20))
        return PH0_EINVAL;
    ph0_ctx *c = new ph0_ctx();
    c->opt = *opt;
    if (c->opt.streams < 1) c->opt.streams = 1;
    if (c->opt.streams > 64) c->opt.streams = 64;
    if (c->opt.small_max_n < 0 || c->opt.small_max_n > small_max_n()) c->opt.small_max_n = small_max_n();
    if (c->opt.batch_max < 1) c->opt.batch_max = 1;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->dev, opt->mem_budget);
    if (e == cudaSuccess) e = cudaHostAlloc(&c->host, opt->host_budget, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tasks, sizeof(SmallTask) * size_t(c->opt.batch_max));
    if (e == cudaSuccess) e = cudaHostAlloc(&c->h_tasks, sizeof(SmallTask) * size_t(c->opt.batch_max), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ntasks, sizeof(int32_t) + sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaHostAlloc(&c->h_ntasks, sizeof(int32_t), cudaHostAllocDefault);
    if (e == cudaSuccess) {
        c->d_counter = reinterpret_cast<uint32_t *>(c->d_ntasks + 1);
        c->dev_arena.reset(opt->mem_budget);
        c->host_arena.reset(opt->host_budget);
        c->streams.resize(size_t(c->opt.streams));
        c->events.resize(size_t(c->opt.streams));
        c->slot_req.assign(size_t(c->opt.streams), nullptr);
        for (int k = 0; k < c->opt.streams && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&c->streams[size_t(k)], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->events[size_t(k)], cudaEventDisableTiming);
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->small_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->small_event, cudaEventDisableTiming);
    // capture the fused batch launch once; replays read the task count on the device
    if (e == cudaSuccess) {
        const int grid = sm_count();
        cudaGraph_t g = nullptr;
        e = prepare_small_kernel();
        if (e == cudaSuccess) e = cudaStreamBeginCapture(c->small_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = launch_small(c->d_tasks, c->d_ntasks, c->d_counter, grid, c->small_stream);
            e = cudaStreamEndCapture(c->small_stream, &g);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->small_graph, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
        ph0_ctx_destroy(c);
        cudaGetLastError();  // a failed allocation is not sticky: clear it for the caller's next check
        return PH0_ECUDA;
    }
    c->worker = std::thread([c] { c->run(); });
    *out = c;
    return PH0_OK;
}

int ph0_submit(ph0_ctx *c, const float *pts_host, int64_t n, int32_t d, uint64_t tag) {
    if (!c || (!pts_host && n > 0)) return PH0_EINVAL;
    if (n < 1 || d < 1) return PH0_EINVAL;
    if (n > kMaxNWide || d > kMaxD) return PH0_ETOOBIG;
    Request *r = new Request();
    r->tag = tag;
    r->n = int32_t(n);
    r->d = d;
    r->small = n <= c->opt.small_max_n && d <= small_max_d();
    r->ws_bytes = r->small ? 0 : ph0_workspace_bytes(n, d);
    r->h_bytes = ph0_ctx::host_bytes(n, d);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->by_tag.count(tag)) {
            delete r;
            return PH0_EINVAL;  // tag still in use
        }
        if (c->dev_bytes(*r) > c->opt.mem_budget) {
            delete r;
            return PH0_ENOMEM;  // can never be admitted
        }
        if (!c->host_arena.alloc(r->h_bytes, r->h_off)) {
            delete r;
            return PH0_EBUSY;  // pinned pool full: poll and release first
        }
        c->by_tag[tag] = r;
    }
    std::memcpy(c->pts_host(r), pts_host, size_t(n) * d * sizeof(float));
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->pending.push_back(r);
    }
    c->cv_work.notify_one();
    return PH0_OK;
}

int ph0_poll(ph0_ctx *c, ph0_result *out, int32_t max, int32_t *got, int32_t wait_ms) {
    if (!c || !got || (max > 0 && !out)) return PH0_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    if (c->finished.empty() && wait_ms > 0)
        c->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [c] { return !c->finished.empty(); });
    int k = 0;
    while (k < max && !c->finished.empty()) {
        Request *r = c->finished.front();
        c->finished.pop_front();
        ph0_result &o = out[k++];
        o.tag = r->tag;
        o.status = r->status;
        o.n = r->n;
        o.d = r->d;
        o.inf_vertex = r->inf_vertex;
        o.n_bars = r->n - 1;
        o.bars = c->bars_host(r);
        o.submit_time = r->t_submit;
        o.done_time = r->t_done;
    }
    *got = k;
    return c->error == cudaSuccess ? PH0_OK : PH0_ECUDA;
}

int ph0_release(ph0_ctx *c, uint64_t tag) {
    if (!c) return PH0_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->by_tag.find(tag);
    if (it == c->by_tag.end()) return PH0_EINVAL;
    Request *r = it->second;
    for (Request *f : c->finished)
        if (f == r) return PH0_EBUSY;  // finished but not yet returned by ph0_poll
    if (r->t_done == 0) return PH0_EBUSY;  // still queued or running
    c->host_arena.release(r->h_off, r->h_bytes);
    c->by_tag.erase(it);
    delete r;
    return PH0_OK;
}

int ph0_ctx_destroy(ph0_ctx *c) {
    if (!c) return PH0_EINVAL;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->cv_work.notify_all();
    if (c->worker.joinable()) c->worker.join();
    cudaDeviceSynchronize();
    for (auto &kv : c->by_tag) delete kv.second;
    for (auto s : c->streams) if (s) cudaStreamDestroy(s);
    for (auto ev : c->events) if (ev) cudaEventDestroy(ev);
    if (c->small_graph) cudaGraphExecDestroy(c->small_graph);
    if (c->small_stream) cudaStreamDestroy(c->small_stream);
    if (c->small_event) cudaEventDestroy(c->small_event);
    cudaFree(c->dev);
    cudaFree(c->d_tasks);
    cudaFree(c->d_ntasks);
    cudaFreeHost(c->host);
    cudaFreeHost(c->h_tasks);
    cudaFreeHost(c->h_ntasks);
    delete c;
    return PH0_OK;
}

}  // extern "C"
