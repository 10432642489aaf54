// Serving loop of libsivf (sivf_server_*): request queue, continuous
// batching, admission by free slabs, and overlapped batches in flight.
//
// One worker thread owns the index.  Requests arrive from any thread into a
// FIFO.  The worker repeatedly (1) completes batches whose last copy has
// landed (results to the callers' host arrays, statuses, free-slab count),
// and (2) when a slot is free, takes the run of same-kind requests at the
// head of the FIFO (up to the kind's batch limit and, for inserts, while the
// worst-case slab demand fits the free slabs known on the host), stages
// their inputs in the slot's pinned buffer, and enqueues on the slot's
// stream: copy in, the index call(s), copy out.  Cross-slot order on the
// device: a query batch waits for the last mutation batch's kernels; a
// mutation batch waits for the kernels of every batch still in flight.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"

using namespace sivf;

namespace {

// host memory the DMA engines can read directly (cudaMallocHost /
// cudaHostRegister); pageable memory is staged through the slot's buffer
bool page_locked(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

int64_t steady_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    int kind = 0;
    int64_t n = 0, n_evict = 0;
    const int64_t *ids = nullptr, *evict = nullptr;
    const float *x = nullptr;
    float *dist = nullptr;
    int64_t *labels = nullptr;
    bool pin_ids = false, pin_x = false, pin_ev = false;  // page-locked host arrays
    int64_t t_arr = 0, t_launch = 0, t_done = 0;
    int32_t status = 0;
    int64_t count = 0, batch = -1;
    bool done = false;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t computed = nullptr;  // the batch's kernels are done
    cudaEvent_t finished = nullptr;  // its outputs and status are on the host
    char *h_in = nullptr, *d_in = nullptr;
    char *h_out = nullptr, *d_out = nullptr;
    Ctl *h_ctl = nullptr;            // pinned [2]: after the evictions, after the call
    int32_t *h_word = nullptr;       // pinned [2]: free slabs, error word
    bool busy = false;
    int kind = 0;
    int64_t seq = 0, n = 0, n_evict = 0, demand = 0;
    int32_t host_status = 0;         // a call that failed on the host
    std::vector<int64_t> reqs;       // request ids, in batch order
    std::vector<Req> rq;             // their copies (read without the lock)
};

}  // namespace

struct sivf_server {
    sivf_index *ix = nullptr;
    sivf_server_config cfg{};
    std::vector<Slot> slots;
    cudaEvent_t mut_done = nullptr;  // kernels of the last mutation batch
    bool any_mut = false;

    // shared with submitters (guarded by mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> reqs;            // every request, index = id
    std::deque<int64_t> pending;     // ids not yet in a batch
    int64_t completed = 0;
    bool stop = false;
    int32_t fatal = 0;               // sticky SIVF_E_* seen by the worker
    sivf_server_stats_t st{};

    // worker only
    int64_t free_known = 0, free_seq = -1, reserved = 0, seq = 0;
    int64_t last_deferred = -1;      // request at the head when an insert last waited
    int in_flight = 0, mut_in_flight = 0;
    bool compact_dirty = true;       // the index may have changed since the last pass
                                     // that moved nothing (true at start)
    std::thread worker;

    void run();
    void idle_compact();
    bool reap();
    bool launch();
    void finish(Slot &sl, int32_t status);
    int64_t worst_demand(int64_t n) const
    {
        return (n + ix->C - 1) / ix->C + std::min<int64_t>(n, ix->nlist);
    }
};

void sivf_server::finish(Slot &sl, int32_t status)
{
    const int64_t t = steady_ns();
    std::lock_guard<std::mutex> lk(mu);
    for (int64_t r : sl.reqs) {
        Req &q = reqs[r];
        q.status = status;
        q.count = status == SIVF_OK ? q.n : 0;
        q.batch = sl.seq;
        q.t_done = t;
        q.done = true;
        st.requests[q.kind] += 1;
        if (status) st.rejected += 1;
    }
    st.batches[sl.kind] += 1;
    st.items[sl.kind] += sl.n;
    completed += (int64_t)sl.reqs.size();
    sl.busy = false;
    sl.reqs.clear();
    sl.rq.clear();
    --in_flight;
    if (sl.kind != SIVF_OP_SEARCH) --mut_in_flight;
    cv_done.notify_all();
}

bool sivf_server::reap()
{
    bool prog = false;
    for (Slot &sl : slots) {
        if (!sl.busy) continue;
        cudaError_t e = cudaEventQuery(sl.finished);
        if (e == cudaErrorNotReady) continue;
        prog = true;
        int32_t status = sl.host_status;
        if (e != cudaSuccess) {
            status = SIVF_E_CUDA;
        } else if (sl.kind == SIVF_OP_SEARCH) {
            // rows of each request, in batch order
            const int k = cfg.k;
            const float *hd = reinterpret_cast<const float *>(sl.h_out);
            const int64_t *hl =
                reinterpret_cast<const int64_t *>(sl.h_out + (size_t)cfg.max_query_batch * k * 4);
            int64_t row = 0;
            for (const Req &q : sl.rq) {
                memcpy(q.dist, hd + row * k, sizeof(float) * q.n * k);
                memcpy(q.labels, hl + row * k, sizeof(int64_t) * q.n * k);
                row += q.n;
            }
        } else if (!status) {
            auto ctl_status = [](const Ctl &c) {
                return (c.flags & FLAG_BAD_ID) ? (int32_t)SIVF_E_ARG : c.status;
            };
            if (sl.n_evict) status = ctl_status(sl.h_ctl[0]);
            if (!status && sl.n) status = ctl_status(sl.h_ctl[1]);
            if (sl.seq > free_seq) {
                free_known = sl.h_word[0];
                free_seq = sl.seq;
            }
            if (sl.h_word[1]) {
                mark_corrupt(ix);
                status = (sl.h_word[1] & 8u) ? SIVF_E_TIMEOUT : SIVF_E_CORRUPT;
                std::lock_guard<std::mutex> lk(mu);
                fatal = status;
            }
            reserved -= sl.demand;
        }
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            fatal = SIVF_E_CUDA;
        }
        finish(sl, status);
    }
    return prog;
}

bool sivf_server::launch()
{
    Slot *sl = nullptr;
    for (Slot &s : slots)
        if (!s.busy) {
            sl = &s;
            break;
        }
    if (!sl) return false;
    std::vector<int64_t> take;
    int kind;
    int64_t n = 0, ne = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (pending.empty()) return false;
        kind = reqs[pending.front()].kind;
        for (int64_t id : pending) {
            const Req &q = reqs[id];
            if (q.kind != kind) break;
            if (kind == SIVF_OP_SEARCH) {
                if (n + q.n > cfg.max_query_batch) break;
            } else if (kind == SIVF_OP_REMOVE) {
                if (n + q.n > cfg.max_delete_batch) break;
            } else {
                if (n + q.n > cfg.max_insert_batch || ne + q.n_evict > cfg.max_delete_batch)
                    break;
                const int64_t avail = free_known - reserved;
                if (worst_demand(n + q.n) > avail) {
                    if (!take.empty()) break;      // serve what fits
                    if (mut_in_flight) {           // frees may be on the way
                        if (last_deferred != id) st.deferred += 1;
                        last_deferred = id;
                        return false;
                    }
                    // alone; the device's exact admission decides
                }
            }
            take.push_back(id);
            n += q.n;
            ne += q.n_evict;
            if (kind == SIVF_OP_ADD && worst_demand(n) > free_known - reserved) break;
        }
        for (size_t i = 0; i < take.size(); ++i) pending.pop_front();
        const int64_t t = steady_ns();
        sl->rq.clear();
        for (int64_t id : take) {
            reqs[id].t_launch = t;
            sl->rq.push_back(reqs[id]);
        }
        if (in_flight + 1 > st.max_in_flight) st.max_in_flight = in_flight + 1;
    }
    Slot &s = *sl;
    s.busy = true;
    s.kind = kind;
    s.seq = seq++;
    s.n = n;
    s.n_evict = ne;
    s.demand = kind == SIVF_OP_ADD ? worst_demand(n) : 0;
    s.host_status = 0;
    s.reqs.swap(take);
    ++in_flight;
    if (kind != SIVF_OP_SEARCH) {
        ++mut_in_flight;
        compact_dirty = true;
    }
    reserved += s.demand;

    const int d = ix->d;
    sivf_index *x = ix;
    sivf_status rc = SIVF_OK;
    cudaError_t ce = cudaSuccess;
    size_t off = 0;
    // append `bytes` of `src` to the slot's device input: page-locked arrays
    // by DMA from where they are, the rest through the pinned staging buffer
    auto put = [&](const void *src, size_t bytes, bool pinned) {
        if (!bytes || ce != cudaSuccess) return;
        if (pinned) {
            ce = cudaMemcpyAsync(s.d_in + off, src, bytes, cudaMemcpyHostToDevice, s.s);
        } else {
            memcpy(s.h_in + off, src, bytes);
            ce = cudaMemcpyAsync(s.d_in + off, s.h_in + off, bytes, cudaMemcpyHostToDevice, s.s);
        }
        off += bytes;
    };
    if (kind == SIVF_OP_SEARCH) {
        for (const Req &q : s.rq) put(q.x, sizeof(float) * q.n * d, q.pin_x);
        if (any_mut && ce == cudaSuccess) ce = cudaStreamWaitEvent(s.s, mut_done, 0);
        float *dd = reinterpret_cast<float *>(s.d_out);
        int64_t *dl = reinterpret_cast<int64_t *>(s.d_out + (size_t)cfg.max_query_batch * cfg.k * 4);
        if (ce == cudaSuccess)
            rc = sivf_search(x, reinterpret_cast<const float *>(s.d_in), n, cfg.k, cfg.nprobe,
                             (sivf_scan_dtype)cfg.dtype, dd, dl, s.s);
        if (ce == cudaSuccess && !rc) ce = cudaEventRecord(s.computed, s.s);
        if (ce == cudaSuccess && !rc) {
            ce = cudaMemcpyAsync(s.h_out, dd, sizeof(float) * n * cfg.k, cudaMemcpyDeviceToHost,
                                 s.s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(s.h_out + (size_t)cfg.max_query_batch * cfg.k * 4, dl,
                                     sizeof(int64_t) * n * cfg.k, cudaMemcpyDeviceToHost, s.s);
        }
    } else {
        // layout of the staged inputs: evictions, ids, vectors
        size_t o_ev = 0, o_id, o_x;
        for (const Req &q : s.rq) put(q.evict, sizeof(int64_t) * q.n_evict, q.pin_ev);
        off = (off + 255) & ~(size_t)255;
        o_id = off;
        for (const Req &q : s.rq) put(q.ids, sizeof(int64_t) * q.n, q.pin_ids);
        off = (off + 255) & ~(size_t)255;
        o_x = off;
        if (kind == SIVF_OP_ADD)
            for (const Req &q : s.rq) put(q.x, sizeof(float) * q.n * d, q.pin_x);
        // after every batch still in flight
        for (Slot &o : slots)
            if (&o != &s && o.busy && ce == cudaSuccess) ce = cudaStreamWaitEvent(s.s, o.computed, 0);
        const int64_t *d_ev = reinterpret_cast<const int64_t *>(s.d_in + o_ev);
        const int64_t *d_id = reinterpret_cast<const int64_t *>(s.d_in + o_id);
        const float *d_x = reinterpret_cast<const float *>(s.d_in + o_x);
        if (ce == cudaSuccess && kind == SIVF_OP_ADD && ne) {
            rc = sivf_remove(x, d_ev, ne, s.s, nullptr);
            if (!rc) ce = cudaMemcpyAsync(&s.h_ctl[0], stream_ctl(x, s.s), sizeof(Ctl),
                                          cudaMemcpyDeviceToHost, s.s);
        }
        if (ce == cudaSuccess && !rc) {
            rc = kind == SIVF_OP_ADD ? sivf_add(x, d_id, d_x, n, s.s, nullptr)
                                     : sivf_remove(x, d_id, n, s.s, nullptr);
            if (!rc) ce = cudaMemcpyAsync(&s.h_ctl[1], stream_ctl(x, s.s), sizeof(Ctl),
                                          cudaMemcpyDeviceToHost, s.s);
        }
        if (ce == cudaSuccess && !rc) {
            ce = cudaEventRecord(s.computed, s.s);
            if (ce == cudaSuccess) ce = cudaEventRecord(mut_done, s.s);
            any_mut = true;
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(&s.h_word[0], x->free_top, 4, cudaMemcpyDeviceToHost, s.s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(&s.h_word[1], x->err, 4, cudaMemcpyDeviceToHost, s.s);
        }
    }
    if (ce != cudaSuccess) rc = SIVF_E_CUDA;
    if (rc) {
        // nothing (more) was enqueued for this batch: complete it with the error
        s.host_status = rc;
        if (kind == SIVF_OP_ADD) reserved -= s.demand;
        s.demand = 0;
        cudaStreamSynchronize(s.s);
        finish(s, rc);
        return true;
    }
    cudaEventRecord(s.finished, s.s);
    return true;
}

// Background compaction: with nothing pending and nothing in flight, one
// bounded pass on the first slot's stream (the call syncs it), so a
// request that arrives meanwhile waits for at most one pass.  Passes repeat
// while they move members and stop until the next mutation batch.
void sivf_server::idle_compact()
{
    int64_t fr = 0, mv = 0;
    const sivf_status rc = sivf_compact(ix, cfg.compact_min_free, cfg.max_insert_batch,
                                        slots[0].s, &fr, &mv);
    std::lock_guard<std::mutex> lk(mu);
    if (rc) {
        fatal = rc;
        compact_dirty = false;
        return;
    }
    if (mv == 0) {
        compact_dirty = false;
        return;
    }
    free_known += fr;
    st.compact_passes += 1;
    st.compact_freed += fr;
    st.compact_moved += mv;
}

void sivf_server::run()
{
    cudaSetDevice(ix->device);
    for (;;) {
        bool prog = reap();
        prog = launch() || prog;
        if (prog) continue;
        std::unique_lock<std::mutex> lk(mu);
        if (stop && pending.empty() && in_flight == 0) break;
        if (in_flight == 0 && pending.empty() && cfg.compact_min_free > 0 && compact_dirty &&
            !fatal) {
            lk.unlock();
            idle_compact();
            continue;
        }
        if (in_flight == 0 && pending.empty())
            cv_work.wait_for(lk, std::chrono::milliseconds(2));
        else {
            lk.unlock();
            std::this_thread::yield();
        }
    }
}

static void server_free(sivf_server *sv)
{
    for (Slot &s : sv->slots) {
        if (s.s) {
            cudaStreamSynchronize(s.s);
            release_stream(sv->ix, s.s);
            cudaStreamDestroy(s.s);
        }
        if (s.computed) cudaEventDestroy(s.computed);
        if (s.finished) cudaEventDestroy(s.finished);
        if (s.h_in) cudaFreeHost(s.h_in);
        if (s.h_out) cudaFreeHost(s.h_out);
        if (s.h_ctl) cudaFreeHost(s.h_ctl);
        if (s.h_word) cudaFreeHost(s.h_word);
        if (s.d_in) cudaFree(s.d_in);
        if (s.d_out) cudaFree(s.d_out);
    }
    if (sv->mut_done) cudaEventDestroy(sv->mut_done);
    delete sv;
}

extern "C" {

int64_t sivf_server_now_ns(void) { return steady_ns(); }

sivf_status sivf_server_create(sivf_index *ix, const sivf_server_config *cfg, sivf_server **out)
{
    if (!ix || !cfg || !out) return SIVF_E_ARG;
    *out = nullptr;
    const sivf_server_config &c = *cfg;
    if (c.depth < 1 || c.depth > 8 || c.k < 1 || c.k > kMaxK || c.nprobe < 1 ||
        c.nprobe > ix->nlist || c.dtype < SIVF_FP32 || c.dtype > SIVF_FP8E4M3 ||
        c.max_query_batch < 1 || c.max_insert_batch < 1 || c.max_delete_batch < 1 ||
        c.compact_min_free < 0)
        return set_error(ix, SIVF_E_ARG, "bad server config");
    if (!ix->have_centroids) return set_error(ix, SIVF_E_STATE, "set_centroids first");
    if (sivf_status hs = index_health(ix)) return hs;
    sivf_server *sv = new (std::nothrow) sivf_server();
    if (!sv) return SIVF_E_NOMEM;
    sv->ix = ix;
    sv->cfg = c;
    sv->slots.resize(c.depth);
    const size_t d = ix->d;
    const size_t in_b = std::max({(size_t)c.max_query_batch * d * 4,
                                  (size_t)c.max_delete_batch * 8 + (size_t)c.max_insert_batch * 8 +
                                      (size_t)c.max_insert_batch * d * 4 + 1024});
    const size_t out_b = (size_t)c.max_query_batch * c.k * 12;
    auto bad = [&](sivf_status st, const char *what) {
        server_free(sv);
        return set_error(ix, st, what);
    };
    if (cudaEventCreateWithFlags(&sv->mut_done, cudaEventDisableTiming) != cudaSuccess)
        return bad(SIVF_E_CUDA, "server events");
    for (Slot &s : sv->slots) {
        if (cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.computed, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.finished, cudaEventDisableTiming) != cudaSuccess)
            return bad(SIVF_E_CUDA, "server streams");
        if (cudaMallocHost(&s.h_in, in_b) != cudaSuccess ||
            cudaMallocHost(&s.h_out, out_b) != cudaSuccess ||
            cudaMallocHost(&s.h_ctl, 2 * sizeof(Ctl)) != cudaSuccess ||
            cudaMallocHost(&s.h_word, 8) != cudaSuccess ||
            cudaMalloc(&s.d_in, in_b) != cudaSuccess || cudaMalloc(&s.d_out, out_b) != cudaSuccess)
            return bad(SIVF_E_NOMEM, "server slot buffers");
        memset(s.h_ctl, 0, 2 * sizeof(Ctl));
        memset(s.h_word, 0, 8);
        sivf_status st = sivf_reserve(ix, c.max_insert_batch, c.max_delete_batch,
                                      c.max_query_batch, c.k, c.nprobe, s.s);
        if (st) {
            server_free(sv);
            return st;
        }
    }
    sivf_stats_t stt;
    sivf_status st = sivf_stats(ix, nullptr, &stt);
    if (st) {
        server_free(sv);
        return st;
    }
    if (stt.error_bits) return bad(SIVF_E_CORRUPT, "index has a device error");
    sv->free_known = stt.free_slabs;
    if (cudaDeviceSynchronize() != cudaSuccess) return bad(SIVF_E_CUDA, "server setup");
    try {
        sv->worker = std::thread([sv]() { sv->run(); });
    } catch (...) {
        return bad(SIVF_E_NOMEM, "server thread");
    }
    *out = sv;
    return SIVF_OK;
}

sivf_status sivf_server_submit(sivf_server *sv, int kind, int64_t n, const int64_t *ids,
                               const float *x, int64_t n_evict, const int64_t *evict,
                               float *dist, int64_t *labels, int64_t arrival_ns, int64_t *req)
{
    if (!sv || !req) return SIVF_E_ARG;
    sivf_index *ix = sv->ix;
    const sivf_server_config &c = sv->cfg;
    const char *why = nullptr;
    if (kind < SIVF_OP_ADD || kind > SIVF_OP_SEARCH) why = "unknown request kind";
    else if (n < 1) why = "empty request";
    else if (kind == SIVF_OP_SEARCH && (n > c.max_query_batch || !x || !dist || !labels))
        why = "bad query request";
    else if (kind == SIVF_OP_REMOVE && (n > c.max_delete_batch || !ids)) why = "bad delete request";
    else if (kind == SIVF_OP_ADD &&
             (n > c.max_insert_batch || !ids || !x || n_evict < 0 ||
              n_evict > c.max_delete_batch || (n_evict && !evict)))
        why = "bad insert request";
    if (why) return set_error(ix, SIVF_E_ARG, why);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal) return (sivf_status)sv->fatal;
    if (sv->stop) return set_error(ix, SIVF_E_STATE, "server stopping");
    Req q;
    q.kind = kind;
    q.n = n;
    q.ids = ids;
    q.x = x;
    q.n_evict = kind == SIVF_OP_ADD ? n_evict : 0;
    q.evict = evict;
    q.dist = dist;
    q.labels = labels;
    q.t_arr = arrival_ns ? arrival_ns : steady_ns();
    q.pin_ids = page_locked(ids);
    q.pin_x = page_locked(x);
    q.pin_ev = page_locked(q.n_evict ? evict : nullptr);
    *req = (int64_t)sv->reqs.size();
    sv->reqs.push_back(q);
    sv->pending.push_back(*req);
    sv->cv_work.notify_one();
    return SIVF_OK;
}

sivf_status sivf_server_wait(sivf_server *sv, int64_t req, int64_t timeout_us,
                             sivf_request_info *info)
{
    if (!sv) return SIVF_E_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (req < 0 || req >= (int64_t)sv->reqs.size())
        return set_error(sv->ix, SIVF_E_ARG, "unknown request");
    auto done = [&]() { return sv->reqs[req].done; };
    if (timeout_us < 0) sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done))
        return SIVF_E_TIMEOUT;
    const Req &q = sv->reqs[req];
    if (info) {
        info->kind = q.kind;
        info->status = q.status;
        info->count = q.count;
        info->batch = q.batch;
        info->latency_ms = (double)(q.t_done - q.t_arr) * 1e-6;
        info->queue_ms = (double)(q.t_launch - q.t_arr) * 1e-6;
    }
    return sv->fatal ? (sivf_status)sv->fatal : SIVF_OK;
}

sivf_status sivf_server_drain(sivf_server *sv, int64_t timeout_us)
{
    if (!sv) return SIVF_E_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto done = [&]() { return sv->completed == (int64_t)sv->reqs.size(); };
    if (timeout_us < 0) sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done))
        return SIVF_E_TIMEOUT;
    return sv->fatal ? (sivf_status)sv->fatal : SIVF_OK;
}

sivf_status sivf_server_stats(sivf_server *sv, sivf_server_stats_t *out)
{
    if (!sv || !out) return SIVF_E_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->st;
    return SIVF_OK;
}

sivf_status sivf_server_destroy(sivf_server *sv)
{
    if (!sv) return SIVF_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    const int32_t fatal = sv->fatal;
    server_free(sv);
    return (sivf_status)fatal;
}

}  // extern "C"
