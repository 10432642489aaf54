// Mixed-batch executor (sivf_exec_*) and scan-tile tuning (sivf_set_tile,
// sivf_get_tile, sivf_autotune).
//
// The executor records a queue of uneven add / remove / search batches into
// one CUDA graph on a private stream, whose scratch arena is reserved for
// the largest batch before recording starts, so nothing inside the graph
// allocates or waits on the host.  The probe selection of every search batch
// reads only its queries and the centroids, not the lists, so it is recorded
// on a second stream forked at the start of the queue: it runs under the
// batches before it, and each search waits only for its own probes.  After every batch a one-thread kernel
// copies the batch's status and count out of the stream's control block
// together with a %globaltimer stamp.  The autotuner times searches of one
// batch shape over a set of tiles by coordinate descent and installs the
// fastest in the index's tile table.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"

using namespace sivf;

// set while this thread records an executor's queue (ordinary kernel edges)
thread_local bool sivf::tl_recording = false;

namespace {

struct OpRecord {        // device, one per batch
    int32_t status;
    int32_t flags;
    int64_t count;
    uint64_t t_ns;       // %globaltimer when the batch's work was done
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_stamp(uint64_t *t)
{
    pdl_begin();
    *t = global_ns();
}

// the batch just finished on this stream: its status and count
__global__ void k_op_record(const Ctl *ctl, OpRecord *r, int is_search, int64_t nq)
{
    pdl_begin();
    OpRecord o;
    int st = is_search ? (int)SIVF_OK : ctl->status;
    if (!is_search && (ctl->flags & FLAG_BAD_ID)) st = SIVF_E_ARG;
    o.status = st;
    o.flags = is_search ? 0 : ctl->flags;
    o.count = is_search ? nq : (st == SIVF_OK ? ctl->count : 0);
    o.t_ns = global_ns();
    *r = o;
}

}  // namespace

struct sivf_exec {
    sivf_index *ix = nullptr;
    std::vector<sivf_op> ops;
    cudaStream_t cap = nullptr;      // private stream: keys the executor's scratch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    OpRecord *rec = nullptr;         // device [nops]
    uint64_t *t0 = nullptr;          // device, queue start stamp
    OpRecord *host = nullptr;        // pinned [nops + 1]
    int64_t kernels = 0;
    cudaStream_t side = nullptr;     // probe selection of the search batches
    std::vector<int32_t *> probes;   // device, per op (search batches only)
    float *cbuf = nullptr;           // device, the coarse selection's scratch
    std::vector<cudaEvent_t> evs;    // fork, per search, join
};

static void exec_free(sivf_exec *e)
{
    if (!e) return;
    if (e->cap) cudaStreamSynchronize(e->cap);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->ix && e->cap) release_stream(e->ix, e->cap);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->rec) cudaFree(e->rec);
    if (e->t0) cudaFree(e->t0);
    if (e->side) cudaStreamDestroy(e->side);
    for (int32_t *p : e->probes)
        if (p) cudaFree(p);
    if (e->cbuf) cudaFree(e->cbuf);
    for (cudaEvent_t ev : e->evs) cudaEventDestroy(ev);
    if (e->host) cudaFreeHost(e->host);
    delete e;
}

static sivf_status check_op(sivf_index *ix, const sivf_op &op, int i)
{
    char b[160];
    const char *why = nullptr;
    if (op.kind < SIVF_OP_ADD || op.kind > SIVF_OP_COMPACT) why = "unknown kind";
    else if (op.n < 1 || op.n > INT32_MAX) why = "n must be in [1, 2^31)";
    else if (op.kind == SIVF_OP_COMPACT) {
        if (op.k < 1) why = "compact: min_free (k) must be >= 1";
    }
    else if (!op.x && op.kind != SIVF_OP_REMOVE) why = "null x";
    else if (!op.ids && op.kind != SIVF_OP_SEARCH) why = "null ids";
    else if (op.kind == SIVF_OP_SEARCH) {
        if (!op.dist || !op.labels) why = "null dist / labels";
        else if (op.k < 1 || op.nprobe < 1 || op.nprobe > ix->nlist) why = "bad k / nprobe";
        else if (op.dtype < SIVF_FP32 || op.dtype > SIVF_FP8E4M3) why = "unknown dtype";
    }
    if (!why) return SIVF_OK;
    snprintf(b, sizeof b, "queued batch %d: %s", i, why);
    return set_error(ix, SIVF_E_ARG, b);
}

#define EXEC_TRY(call)                                                           \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            char b_[200];                                                        \
            snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));    \
            exec_free(e);                                                        \
            return set_error(ix, SIVF_E_CUDA, b_);                               \
        }                                                                        \
    } while (0)

extern "C" {

sivf_status sivf_exec_create(sivf_index *ix, const sivf_op *ops, int nops, sivf_exec **out)
{
    if (!ix || !out) return SIVF_E_ARG;
    *out = nullptr;
    if (nops < 1 || !ops) return set_error(ix, SIVF_E_ARG, "empty queue");
    if (!ix->have_centroids) return set_error(ix, SIVF_E_STATE, "set_centroids first");
    if (sivf_status hs = index_health(ix)) return hs;
    size_t need = 0;
    int64_t max_add = 1;
    for (int i = 0; i < nops; ++i) {
        sivf_status st = check_op(ix, ops[i], i);
        if (st) return st;
        need = std::max(need, op_need(ix, ops[i]));
        if (ops[i].kind == SIVF_OP_ADD) max_add = std::max(max_add, ops[i].n);
    }
    sivf_exec *e = new (std::nothrow) sivf_exec();
    if (!e) return SIVF_E_NOMEM;
    e->ix = ix;
    e->ops.assign(ops, ops + nops);
    EXEC_TRY(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking));
    EXEC_TRY(cudaMalloc(&e->rec, sizeof(OpRecord) * nops));
    EXEC_TRY(cudaMalloc(&e->t0, sizeof(uint64_t)));
    EXEC_TRY(cudaMallocHost(&e->host, sizeof(OpRecord) * (nops + 1)));
    EXEC_TRY(cudaMemset(e->rec, 0, sizeof(OpRecord) * nops));
    sivf_status st = reserve_stream(ix, e->cap, need, max_add);
    if (st) {
        exec_free(e);
        return st;
    }
    Ctl *ctl = stream_ctl(ix, e->cap);
    if (!ctl) {
        exec_free(e);
        return set_error(ix, SIVF_E_CUDA, "executor scratch missing");
    }
    // probe buffers of the search batches and the coarse selection's scratch
    e->probes.assign(nops, nullptr);
    size_t cneed = 0;
    int nsearch = 0;
    for (int i = 0; i < nops; ++i)
        if (ops[i].kind == SIVF_OP_SEARCH) {
            EXEC_TRY(cudaMalloc(&e->probes[i], sizeof(int32_t) * ops[i].n * ops[i].nprobe));
            cneed = std::max(cneed, coarse_bytes(ix, ops[i].n));
            ++nsearch;
        }
    if (nsearch) {
        EXEC_TRY(cudaMalloc(&e->cbuf, cneed));
        EXEC_TRY(cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking));
        e->evs.assign(nops + 2, nullptr);
        for (auto &ev : e->evs) EXEC_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    EXEC_TRY(cudaStreamSynchronize(e->cap));
    EXEC_TRY(cudaDeviceSynchronize());

    // record the queue
    const int64_t launches0 = ix->launches;
    ix->capturing = true;
    tl_recording = true;
    cudaError_t ce = cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        ix->capturing = false;
        tl_recording = false;
        EXEC_TRY(ce);
    }
    launch_pdl(k_stamp, 1, 1, 0, e->cap, e->t0);
    if (nsearch) {
        // fork: the probe selection of every search batch, in queue order
        cudaEventRecord(e->evs[nops], e->cap);
        cudaStreamWaitEvent(e->side, e->evs[nops], 0);
        for (int i = 0; i < nops; ++i) {
            const sivf_op &op = e->ops[i];
            if (op.kind != SIVF_OP_SEARCH) continue;
            coarse_topP(ix, op.x, op.n, op.nprobe, e->probes[i], e->cbuf, coarse_rows(ix, op.n),
                        e->side);
            cudaEventRecord(e->evs[i], e->side);
        }
        cudaEventRecord(e->evs[nops + 1], e->side);
    }
    sivf_status bad = SIVF_OK;
    int bad_i = -1;
    for (int i = 0; i < nops && !bad; ++i) {
        const sivf_op &op = e->ops[i];
        sivf_status s2;
        if (op.kind == SIVF_OP_ADD)
            s2 = sivf_add(ix, op.ids, op.x, op.n, e->cap, nullptr);
        else if (op.kind == SIVF_OP_REMOVE)
            s2 = sivf_remove(ix, op.ids, op.n, e->cap, nullptr);
        else if (op.kind == SIVF_OP_COMPACT)
            s2 = sivf_compact(ix, op.k, op.n, e->cap, nullptr, nullptr);
        else {
            cudaStreamWaitEvent(e->cap, e->evs[i], 0);  // this batch's probes
            s2 = search_probed(ix, op.x, op.n, op.k, op.nprobe, e->probes[i],
                               (sivf_scan_dtype)op.dtype, op.dist, op.labels, e->cap);
        }
        if (s2) {
            bad = s2;
            bad_i = i;
            break;
        }
        // the op's kernels ran on the executor's stream: its control block
        if (stream_ctl(ix, e->cap) != ctl) {
            bad = SIVF_E_CUDA;
            bad_i = i;
            break;
        }
        launch_pdl(k_op_record, 1, 1, 0, e->cap, ctl, e->rec + i, op.kind == SIVF_OP_SEARCH, op.n);
    }
    if (nsearch) cudaStreamWaitEvent(e->cap, e->evs[nops + 1], 0);  // join the side stream
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(e->cap, &g);
    ix->capturing = false;
    tl_recording = false;
    ix->launches = launches0;  // recorded, not run
    if (bad) {
        if (g) cudaGraphDestroy(g);
        std::string why = "queued batch " + std::to_string(bad_i) + ": " + ix->last_error;
        exec_free(e);
        return set_error(ix, bad, why.c_str());
    }
    e->graph = g;
    EXEC_TRY(ce);
    EXEC_TRY(cudaGraphInstantiate(&e->gexec, e->graph, 0));
    size_t nn = 0;
    EXEC_TRY(cudaGraphGetNodes(e->graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    EXEC_TRY(cudaGraphGetNodes(e->graph, nodes.data(), &nn));
    for (auto n : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++e->kernels;
    }
    EXEC_TRY(cudaGraphUpload(e->gexec, e->cap));
    EXEC_TRY(cudaStreamSynchronize(e->cap));
    *out = e;
    return SIVF_OK;
}

sivf_status sivf_exec_launch(sivf_exec *e, void *stream)
{
    if (!e) return SIVF_E_ARG;
    sivf_index *ix = e->ix;
    if (sivf_status hs = index_health(ix)) return hs;
    cudaError_t ce = cudaGraphLaunch(e->gexec, (cudaStream_t)stream);
    if (ce != cudaSuccess) return set_error(ix, SIVF_E_CUDA, cudaGetErrorString(ce));
    ix->launches += e->kernels;
    return SIVF_OK;
}

sivf_status sivf_exec_results(sivf_exec *e, void *stream, sivf_op_result *res)
{
    if (!e || !res) return SIVF_E_ARG;
    sivf_index *ix = e->ix;
    const int n = (int)e->ops.size();
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t err = 0;
    if (cudaMemcpyAsync(e->host, e->rec, sizeof(OpRecord) * n, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&e->host[n].t_ns, e->t0, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&e->host[n].flags, ix->err, 4, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_error(ix, SIVF_E_CUDA, "reading executor results");
    err = (uint32_t)e->host[n].flags;
    uint64_t prev = e->host[n].t_ns;
    for (int i = 0; i < n; ++i) {
        res[i].status = e->host[i].status;
        res[i].pad = 0;
        res[i].count = e->host[i].count;
        const uint64_t t = e->host[i].t_ns;
        res[i].device_ms = t >= prev ? (double)(t - prev) * 1e-6 : 0.0;
        prev = t;
    }
    if (err) {
        mark_corrupt(ix);
        char b[96];
        snprintf(b, sizeof b, "device error bits 0x%x", err);
        set_error(ix, SIVF_E_CORRUPT, b);
        return (err & ERR_TIMEOUT) ? SIVF_E_TIMEOUT : SIVF_E_CORRUPT;
    }
    return SIVF_OK;
}

int64_t sivf_exec_kernels(const sivf_exec *e) { return e ? e->kernels : 0; }

sivf_status sivf_exec_destroy(sivf_exec *e)
{
    exec_free(e);
    return SIVF_OK;
}

// ---------------------------------------------------------------- tiles
static int kept_per_pair(int dtype, int k) { return dtype == SIVF_FP32 ? k : 4 * k; }

static sivf_status tile_args(sivf_index *ix, sivf_scan_dtype dtype, int64_t nq, int k,
                             int nprobe)
{
    if (!ix) return SIVF_E_ARG;
    if (dtype < SIVF_FP32 || dtype > SIVF_FP8E4M3 || nq < 1 || k < 1 || k > kMaxK ||
        nprobe < 1 || nprobe > ix->nlist)
        return set_error(ix, SIVF_E_ARG, "bad tile bucket arguments");
    return SIVF_OK;
}

sivf_status sivf_set_tile(sivf_index *ix, sivf_scan_dtype dtype, int64_t nq, int k,
                          int nprobe, const sivf_tile *tile)
{
    sivf_status st = tile_args(ix, dtype, nq, k, nprobe);
    if (st) return st;
    const int K = kept_per_pair(dtype, k);
    TileChoice &c = ix->tune[dtype][tune_bucket(ix, nq, nprobe)][tune_kbucket(K)];
    if (!tile) {
        c.set = 0;
        return SIVF_OK;
    }
    if (!tile_valid(ix, dtype, *tile, K))
        return set_error(ix, SIVF_E_ARG, "tile out of range or over shared memory");
    c.t = *tile;
    c.set = 1;
    return SIVF_OK;
}

sivf_status sivf_get_tile(sivf_index *ix, sivf_scan_dtype dtype, int64_t nq, int k,
                          int nprobe, sivf_tile *out)
{
    sivf_status st = tile_args(ix, dtype, nq, k, nprobe);
    if (st) return st;
    if (!out) return set_error(ix, SIVF_E_ARG, "null out");
    *out = current_tile(ix, dtype, nq, nprobe, kept_per_pair(dtype, k));
    return SIVF_OK;
}

sivf_status sivf_autotune(sivf_index *ix, const float *q, int64_t nq, int k, int nprobe,
                          sivf_scan_dtype dtype, int reps, void *stream, sivf_tile *best,
                          double *best_ms)
{
    sivf_status st = tile_args(ix, dtype, nq, k, nprobe);
    if (st) return st;
    if (!q || !best || reps < 1) return set_error(ix, SIVF_E_ARG, "bad autotune arguments");
    const int K = kept_per_pair(dtype, k);
    TileChoice &slot = ix->tune[dtype][tune_bucket(ix, nq, nprobe)][tune_kbucket(K)];
    const TileChoice saved = slot;
    cudaStream_t s = (cudaStream_t)stream;
    float *dist = nullptr;
    int64_t *lab = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (dist) cudaFree(dist);
        if (lab) cudaFree(lab);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&dist, sizeof(float) * nq * k) != cudaSuccess ||
        cudaMalloc(&lab, sizeof(int64_t) * nq * k) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return set_error(ix, SIVF_E_NOMEM, "autotune buffers");
    }
    // mean ms per search with tile t installed (negative: the search failed)
    auto time_tile = [&](const sivf_tile &t) -> double {
        slot.t = t;
        slot.set = 1;
        if (sivf_search(ix, q, nq, k, nprobe, dtype, dist, lab, stream)) return -1.0;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r)
            if (sivf_search(ix, q, nq, k, nprobe, dtype, dist, lab, stream)) return -1.0;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    sivf_tile cur = current_tile(ix, dtype, nq, nprobe, K);
    double cur_ms = time_tile(cur);
    if (cur_ms < 0) {
        slot = saved;
        cleanup();
        return set_error(ix, SIVF_E_ARG, ("autotune: search failed: " + ix->last_error).c_str());
    }
    static const int tq_v[] = {8, 16, 32, 64};
    static const int spc_v[] = {1, 2, 4, 8};
    static const int ips_v[] = {1, 2, 4, 8, 16};
    static const int sel_v[] = {0, 1, 2, 4};
    static const int nf_v[] = {0, 1};
    static const int tsel_v[] = {0, 1, 2};
    static const int tqr_v[] = {64, 128};
    struct Knob {
        int32_t sivf_tile::*field;
        const int *v;
        int n;
    };
    std::vector<Knob> knobs;
    if (dtype == SIVF_FP32) {
        knobs.push_back({&sivf_tile::queries_per_tile, tq_v, 4});
        knobs.push_back({&sivf_tile::select_slabs, sel_v, 4});
    } else {
        knobs.push_back({&sivf_tile::queries_per_tile, tqr_v, 2});
        knobs.push_back({&sivf_tile::nearest_first, nf_v, 2});
        knobs.push_back({&sivf_tile::select_slabs, tsel_v, 3});
    }
    knobs.push_back({&sivf_tile::slabs_per_chunk, spc_v, 4});
    knobs.push_back({&sivf_tile::items_per_sm, ips_v, 5});
    for (int pass = 0; pass < 2; ++pass) {
        bool moved = false;
        for (const Knob &kb : knobs)
            for (int j = 0; j < kb.n; ++j) {
                if (cur.*(kb.field) == kb.v[j]) continue;
                sivf_tile t = cur;
                t.*(kb.field) = kb.v[j];
                if (!tile_valid(ix, dtype, t, K)) continue;
                const double ms = time_tile(t);
                if (ms >= 0 && ms < cur_ms * 0.98) {
                    cur = t;
                    cur_ms = ms;
                    moved = true;
                }
            }
        if (!moved) break;
    }
    slot.t = cur;
    slot.set = 1;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    cleanup();
    return SIVF_OK;
}

}  // extern "C"
