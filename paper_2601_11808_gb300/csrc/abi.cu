// The C ABI of libsivf (include/sivf.h): argument checks, device state
// allocation, per-stream scratch, and the order in which each call enqueues
// the kernels of the hot path.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

using namespace sivf;

namespace {

// per-stream call context: control block, scratch arena, pinned mirror
struct Ctx {
    Ctl *ctl = nullptr;
    char *scratch = nullptr;
    size_t bytes = 0;
    Ctl *host = nullptr;
};

struct Extra {
    std::unordered_map<void *, Ctx> ctx;
    bool corrupt = false;
    int32_t last_status = 0;
    int64_t last_count = 0;
};

Extra &ex(sivf_index *ix) { return *reinterpret_cast<Extra *>(ix->extra); }

sivf_status fail(sivf_index *ix, sivf_status st, const char *what)
{
    if (ix) ix->last_error = what;
    return st;
}

#define CUDA_TRY(ix, call)                                                        \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            char b_[256];                                                         \
            snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));     \
            return fail(ix, e_ == cudaErrorMemoryAllocation ? SIVF_E_NOMEM        \
                                                            : SIVF_E_CUDA, b_);   \
        }                                                                         \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

__global__ void k_init_pool(int32_t *free_list, SlabMeta *meta, int64_t S)
{
    pdl_begin();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        free_list[s] = (int32_t)(S - 1 - s);  // slab 0 on top
        meta[s].list = -1;
        meta[s].fill = 0;
        meta[s].live = 0;
        meta[s].pad = 0;
    }
}

// bump allocator over a context's arena
struct Bump {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += n * sizeof(T);
        return p;
    }
};

sivf_status get_ctx(sivf_index *ix, void *stream, size_t need, Ctx **out)
{
    Ctx &c = ex(ix).ctx[stream];
    if (!c.ctl) {
        CUDA_TRY(ix, cudaMalloc(&c.ctl, sizeof(Ctl)));
        CUDA_TRY(ix, cudaMemset(c.ctl, 0, sizeof(Ctl)));
        CUDA_TRY(ix, cudaMallocHost(&c.host, sizeof(Ctl)));
    }
    if (need > c.bytes) {
        CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
        if (c.scratch) CUDA_TRY(ix, cudaFree(c.scratch));
        c.scratch = nullptr;
        c.bytes = 0;
        size_t nb = std::max(need + need / 4, (size_t)1 << 20);
        CUDA_TRY(ix, cudaMalloc(&c.scratch, nb));
        c.bytes = nb;
    }
    ix->ctl = c.ctl;
    *out = &c;
    return SIVF_OK;
}

sivf_status grow_rank_rows(sivf_index *ix, int64_t n, void *stream)
{
    int need = (int)((n + kRankTile - 1) / kRankTile);
    if (need <= ix->nblk_max) return SIVF_OK;
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    CUDA_TRY(ix, cudaDeviceSynchronize());
    int nb = std::max(need, 2 * ix->nblk_max);
    int32_t *rc = nullptr;
    CUDA_TRY(ix, dalloc(&rc, (size_t)ix->nlist * nb));
    CUDA_TRY(ix, cudaMemset(rc, 0, sizeof(int32_t) * (size_t)ix->nlist * nb));
    CUDA_TRY(ix, cudaFree(ix->runcnt));
    ix->runcnt = rc;
    ix->nblk_max = nb;
    return SIVF_OK;
}

sivf_status check_health(sivf_index *ix)
{
    if (ex(ix).corrupt) return fail(ix, SIVF_E_CORRUPT, "index marked corrupt");
    return SIVF_OK;
}

sivf_status read_status(sivf_index *ix, void *stream, int64_t *count)
{
    Ctx &c = ex(ix).ctx[stream];
    if (!c.ctl) {
        if (count) *count = 0;
        return SIVF_OK;
    }
    uint32_t err = 0;
    CUDA_TRY(ix, cudaMemcpyAsync(c.host, c.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
    CUDA_TRY(ix, cudaMemcpyAsync(&c.host->pad[0], ix->err, sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    err = (uint32_t)c.host->pad[0];
    int st = c.host->status;
    if (c.host->flags & FLAG_BAD_ID) st = SIVF_E_ARG;
    ex(ix).last_status = st;
    ex(ix).last_count = st == SIVF_OK ? c.host->count : 0;
    if (count) *count = ex(ix).last_count;
    if (err) {
        ex(ix).corrupt = true;
        char b[96];
        snprintf(b, sizeof b, "device error bits 0x%x", err);
        ix->last_error = b;
        return (err & ERR_TIMEOUT) ? SIVF_E_TIMEOUT : SIVF_E_CORRUPT;
    }
    if (st == SIVF_E_NOMEM) ix->last_error = "slab pool or list directory exhausted";
    if (st == SIVF_E_ARG) ix->last_error = "id outside [0, n_max)";
    return (sivf_status)st;
}

}  // namespace

namespace sivf {

int64_t coarse_rows(const sivf_index *ix, int64_t n)
{
    // approximate-distance rows per chunk: at most 64 MB of scratch
    int64_t r = ((int64_t)64 << 20) / (4 * (int64_t)ix->nlist);
    return std::max<int64_t>(1, std::min<int64_t>(n, std::max<int64_t>(r, 128)));
}

size_t coarse_bytes(const sivf_index *ix, int64_t n)
{
    return (size_t)coarse_rows(ix, n) * ix->nlist * 4 + 256;
}

int prof_begin(sivf_index *ix, int k, int n, cudaStream_t st)
{
    ix->launches += n;
    if (!ix->prof_on || ix->capturing) return -1;
    ProfEvent e;
    e.kind = k;
    e.launches = n;
    if (cudaEventCreate(&e.start) != cudaSuccess) return -1;
    if (cudaEventCreate(&e.stop) != cudaSuccess) {
        cudaEventDestroy(e.start);
        return -1;
    }
    cudaEventRecord(e.start, st);
    ix->prof.push_back(e);
    return (int)ix->prof.size() - 1;
}

void prof_end(sivf_index *ix, int tok, cudaStream_t st)
{
    if (tok >= 0 && tok < (int)ix->prof.size()) cudaEventRecord(ix->prof[tok].stop, st);
}
}  // namespace sivf

static void prof_clear(sivf_index *ix)
{
    for (auto &e : ix->prof) {
        cudaEventDestroy(e.start);
        cudaEventDestroy(e.stop);
    }
    ix->prof.clear();
}

extern "C" {

const char *sivf_version(void) { return "sivf-gb300 0.1 (sm_103a)"; }

const char *sivf_last_error(const sivf_index *index)
{
    return index ? index->last_error.c_str() : "null index";
}

sivf_status sivf_create(const sivf_config *cfg, sivf_index **out)
{
    if (!cfg || !out) return SIVF_E_ARG;
    *out = nullptr;
    const int d = cfg->d, L = cfg->nlist, C = cfg->slab_size;
    if (d < 4 || d > kMaxD || d % 4 || L < 1 || L > 65536 ||
        !(C == 32 || C == 64 || C == 128) || cfg->n_max < 1 || cfg->n_max > ((int64_t)1 << 40) ||
        cfg->n_slabs < 1 || cfg->n_slabs > INT32_MAX || cfg->dir_cap < 0 ||
        (cfg->scan_dtypes & ~((1u << SIVF_BF16) | (1u << SIVF_FP8E4M3))) ||
        (size_t)2 * C * d * 4 > kMaxStageBytes ||
        (cfg->scan_dtypes && d % 16))
        return SIVF_E_ARG;
    sivf_index *ix = new (std::nothrow) sivf_index();
    if (!ix) return SIVF_E_NOMEM;
    ix->extra = new Extra();
    ix->d = d;
    ix->nlist = L;
    ix->C = C;
    ix->W = C / 32;
    ix->n_max = cfg->n_max;
    ix->n_slabs = cfg->n_slabs;
    ix->dir_cap = cfg->dir_cap ? std::min(cfg->dir_cap, cfg->n_slabs) : cfg->n_slabs;
    ix->dtypes = cfg->scan_dtypes;
    ix->wait_ns = kWaitNs;
    cudaGetDevice(&ix->device);
    ix->nblk_max = 64;
    const size_t S = (size_t)ix->n_slabs, rows = S * C;
    auto bad = [&](sivf_status st) {
        sivf_destroy(ix);
        return st;
    };
#define ALLOC(p, n) \
    if (dalloc(&(p), (n)) != cudaSuccess) return bad(SIVF_E_NOMEM);
    ALLOC(ix->cent, (size_t)L * d);
    ALLOC(ix->cnorm, (size_t)L);
    ALLOC(ix->cnrm_up, (size_t)L);
    // BF16 copy of the centroids for the tensor-core first stage of the
    // coarse selection (d % 16 == 0)
    if (d % 16 == 0 && d <= kMaxD) ALLOC(ix->cent_bf16, (size_t)L * d);
    if (d % 16 == 0 && d <= 128) ALLOC(ix->cent_lo, (size_t)L * d);
    ALLOC(ix->x32, rows * d);
    if (ix->dtypes & (1u << SIVF_BF16)) ALLOC(ix->xb16, rows * d);
    if (ix->dtypes & (1u << SIVF_FP8E4M3)) ALLOC(ix->x8, rows * d);
    if (ix->dtypes & (1u << SIVF_FP8E4M3)) ALLOC(ix->rnorm, rows);
    ALLOC(ix->inv_scale8, (size_t)L);
    ALLOC(ix->xnorm, rows);
    ALLOC(ix->ids, rows);
    ALLOC(ix->bits, S * ix->W);
    ALLOC(ix->meta, S);
    ALLOC(ix->free_list, S);
    ALLOC(ix->free_top, 1);
    ALLOC(ix->head, (size_t)L);
    ALLOC(ix->nslabs, (size_t)L);
    ALLOC(ix->list_live, (size_t)L);
    ALLOC(ix->dir, (size_t)L * ix->dir_cap);
    ALLOC(ix->att, (size_t)ix->n_max);
    ALLOC(ix->claim, (size_t)ix->n_max);
    ALLOC(ix->list_flag, (size_t)L);
    ALLOC(ix->aff_flag, (size_t)L);
    ALLOC(ix->runcnt, (size_t)L * ix->nblk_max);
    ALLOC(ix->err, 1);
    ALLOC(ix->stat, 4);
#undef ALLOC
    int32_t top = (int32_t)S;
    if (cudaMemset(ix->bits, 0, S * ix->W * 4) != cudaSuccess ||
        cudaMemset(ix->head, 0xff, (size_t)L * 4) != cudaSuccess ||
        cudaMemset(ix->nslabs, 0, (size_t)L * 4) != cudaSuccess ||
        cudaMemset(ix->list_live, 0, (size_t)L * 4) != cudaSuccess ||
        cudaMemset(ix->att, 0xff, (size_t)ix->n_max * 8) != cudaSuccess ||
        cudaMemset(ix->claim, 0xff, (size_t)ix->n_max * 4) != cudaSuccess ||
        cudaMemset(ix->list_flag, 0, (size_t)L * 4) != cudaSuccess ||
        cudaMemset(ix->aff_flag, 0, (size_t)L * 4) != cudaSuccess ||
        cudaMemset(ix->runcnt, 0, (size_t)L * ix->nblk_max * 4) != cudaSuccess ||
        cudaMemset(ix->err, 0, 4) != cudaSuccess ||
        cudaMemset(ix->stat, 0, 32) != cudaSuccess ||
        cudaMemcpy(ix->free_top, &top, 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return bad(SIVF_E_CUDA);
    k_init_pool<<<(unsigned)std::min<size_t>((S + 255) / 256, 152 * 64), 256>>>(
        ix->free_list, ix->meta, (int64_t)S);
    if (cudaDeviceSynchronize() != cudaSuccess) return bad(SIVF_E_CUDA);
    if ((ix->xb16 || ix->x8) && !tc_make_maps(ix)) return bad(SIVF_E_CUDA);
    ix->tmap_cent_ok = coarse_make_map(ix);
    ix->tmaps_ready = true;
    *out = ix;
    return SIVF_OK;
}

sivf_status sivf_destroy(sivf_index *ix)
{
    if (!ix) return SIVF_OK;
    cudaDeviceSynchronize();
    void *ptrs[] = {ix->cent, ix->cnorm, ix->cnrm_up, ix->cent_bf16, ix->cent_lo, ix->x32, ix->xb16,
                    ix->x8, ix->rnorm, ix->inv_scale8, ix->xnorm, ix->ids, ix->bits, ix->meta,
                    ix->free_list, ix->free_top, ix->head, ix->nslabs, ix->list_live, ix->dir, ix->att,
                    ix->claim, ix->list_flag, ix->aff_flag, ix->runcnt, ix->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    prof_clear(ix);
    if (ix->stat) cudaFree(ix->stat);
    if (ix->extra) {
        Extra &e = ex(ix);
        for (auto &kv : e.ctx) {
            if (kv.second.ctl) cudaFree(kv.second.ctl);
            if (kv.second.scratch) cudaFree(kv.second.scratch);
            if (kv.second.host) cudaFreeHost(kv.second.host);
        }
        delete &e;
    }
    delete ix;
    return SIVF_OK;
}

static sivf_status live_count(sivf_index *ix, int64_t *n)
{
    CUDA_TRY(ix, cudaMemcpy(n, ix->stat, 8, cudaMemcpyDeviceToHost));
    return SIVF_OK;
}

sivf_status sivf_set_centroids(sivf_index *ix, const float *c, void *stream)
{
    if (!ix || !c) return fail(ix, SIVF_E_ARG, "null argument");
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    int64_t live = 0;
    sivf_status st = live_count(ix, &live);
    if (st) return st;
    if (live) return fail(ix, SIVF_E_STATE, "set_centroids on a non-empty index");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(ix, cudaMemcpyAsync(ix->cent, c, sizeof(float) * ix->nlist * ix->d,
                                 cudaMemcpyDeviceToDevice, s));
    centroid_prep(ix, s);
    CUDA_TRY(ix, cudaGetLastError());
    CUDA_TRY(ix, assign_stage_choose(ix, s));
    ix->have_centroids = true;
    return SIVF_OK;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the state advances by the
// golden-ratio increment; the output is that state through two
// xor-shift-multiply rounds and a final xor-shift
static uint64_t splitmix64_next(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

sivf_status sivf_train(sivf_index *ix, const float *x, int64_t n, int iters, uint64_t seed,
                       void *stream)
{
    if (!ix) return SIVF_E_ARG;
    if (!x || n < ix->nlist || n > INT32_MAX || iters < 0)
        return fail(ix, SIVF_E_ARG, "bad train arguments (need nlist <= n, iters >= 0)");
    sivf_status st = check_health(ix);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(ix, cudaStreamSynchronize(s));
    int64_t live = 0;
    if ((st = live_count(ix, &live))) return st;
    if (live) return fail(ix, SIVF_E_STATE, "train on a non-empty index");
    const int L = ix->nlist, d = ix->d;
    // initial centroids: SplitMix64 outputs mod n in draw order, repeats skipped
    std::vector<int64_t> rows;
    rows.reserve(L);
    {
        std::vector<unsigned char> taken((size_t)n, 0);
        uint64_t state = seed;
        while ((int)rows.size() < L) {
            const int64_t r = (int64_t)(splitmix64_next(state) % (uint64_t)n);
            if (taken[(size_t)r]) continue;
            taken[(size_t)r] = 1;
            rows.push_back(r);
        }
    }
    const int64_t crows = coarse_rows(ix, n);
    const size_t need = coarse_bytes(ix, n) + (size_t)n * 4 + (size_t)L * d * 8 + (size_t)L * 4 +
                        (size_t)L * 8 + 5 * 256;
    Ctx *c;
    if ((st = get_ctx(ix, stream, need, &c))) return st;
    Bump b{c->scratch};
    int32_t *lab = b.take<int32_t>((size_t)n);
    float *Dbuf = b.take<float>((size_t)crows * L);
    double *sum = b.take<double>((size_t)L * d);
    int32_t *cnt = b.take<int32_t>((size_t)L);
    int64_t *rows_dev = b.take<int64_t>((size_t)L);
    CUDA_TRY(ix, cudaMemcpy(rows_dev, rows.data(), sizeof(int64_t) * L, cudaMemcpyHostToDevice));
    CUDA_TRY(ix, cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s));
    train_gather(ix, x, rows_dev, s);
    centroid_prep(ix, s);
    // the assignment's first stage is chosen on the initial centroids and
    // again on the trained ones
    CUDA_TRY(ix, assign_stage_choose(ix, s));
    for (int it = 0; it < iters; ++it) {
        coarse_topP(ix, x, n, 1, lab, Dbuf, crows, s);
        train_step(ix, x, n, lab, sum, cnt, s);
        centroid_prep(ix, s);
    }
    CUDA_TRY(ix, cudaGetLastError());
    CUDA_TRY(ix, assign_stage_choose(ix, s));
    ix->have_centroids = true;
    return SIVF_OK;
}

int32_t sivf_assign_stage(const sivf_index *ix)
{
    if (!ix || !ix->have_centroids) return -1;
    return first_stage_split(ix, 1);
}

sivf_status sivf_get_centroids(sivf_index *ix, float *c, void *stream)
{
    if (!ix || !c) return fail(ix, SIVF_E_ARG, "null argument");
    if (!ix->have_centroids) return fail(ix, SIVF_E_STATE, "no centroids yet");
    CUDA_TRY(ix, cudaMemcpyAsync(c, ix->cent, sizeof(float) * ix->nlist * ix->d,
                                 cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SIVF_OK;
}

sivf_status sivf_set_list_scales(sivf_index *ix, const float *inv_scale, void *stream)
{
    if (!ix || !inv_scale) return fail(ix, SIVF_E_ARG, "null argument");
    int64_t live = 0;
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    sivf_status st = live_count(ix, &live);
    if (st) return st;
    if (live) return fail(ix, SIVF_E_STATE, "set_list_scales on a non-empty index");
    CUDA_TRY(ix, cudaMemcpyAsync(ix->inv_scale8, inv_scale, sizeof(float) * ix->nlist,
                                 cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SIVF_OK;
}

static size_t add_bytes(const sivf_index *ix, int64_t n)
{
    const int L = ix->nlist;
    return coarse_bytes(ix, n) + (size_t)n * 8 + (size_t)L * (4 + 4 + 16 + 4) + 8 * 256;
}

static size_t search_bytes(const sivf_index *ix, int64_t nq, int k, int P, SearchPlan *plo)
{
    const int L = ix->nlist;
    SearchPlan pl = plan_search(ix, nq, P, k);
    if (plo) *plo = pl;
    size_t parts = (size_t)pl.run_cap * pl.K;
    return coarse_bytes(ix, nq) + (size_t)nq * P * 4 * 4 + (size_t)(L + 1) * 4 * 4 +
           parts * 12 + (size_t)nq * 4 * 3 + (size_t)nq * 16 + (size_t)nq * pl.K * 12 +
           (size_t)pl.item_cap * 8 + 19 * 256;
}

// plan of the reduced-precision scan for K' candidates (the batch's tile)
static SearchPlan plan_tc(const sivf_index *ix, int dtype, int64_t nq, int P, int Kc)
{
    return plan_from_tile(ix, dtype, nq, P, Kc, current_tile(ix, dtype, nq, P, Kc));
}

// scratch of one query chunk of m queries, and its scan plan
static size_t chunk_need(const sivf_index *ix, int64_t m, int P, int Kc, int dtype,
                         SearchPlan *plo)
{
    if (dtype == SIVF_FP32) return search_bytes(ix, m, Kc, P, plo);
    const int L = ix->nlist;
    SearchPlan pl = plan_tc(ix, dtype, m, P, Kc);
    *plo = pl;
    return coarse_bytes(ix, m) + (size_t)m * P * 4 * 4 + (size_t)(L + 1) * 4 * 4 +
           (size_t)pl.run_cap * (pl.RK * 12 + 4) + (size_t)m * 4 * 3 + (size_t)m * 16 +
           (size_t)m * pl.K * 12 + (size_t)pl.item_cap * 8 + (size_t)m * ix->d * 2 +
           (dtype == SIVF_FP8E4M3 ? (size_t)m * P * (ix->d + 8) : 0) + 23 * 256;
}

// Queries per chunk of a search of nq queries: all of them (at most 65536)
// when their scratch fits kChunkBytes, else the most (at least 256) that
// fit.  Each chunk streams the lists its queries probe, so fewer, larger
// chunks read each list fewer times.
constexpr size_t kChunkBytes = (size_t)6 << 30;
static int64_t query_chunk(const sivf_index *ix, int64_t nq, int P, int Kc, int dtype)
{
    SearchPlan pl;
    const size_t budget = ix->chunk_bytes > 0 ? (size_t)ix->chunk_bytes : kChunkBytes;
    const int64_t top = std::min<int64_t>(std::max<int64_t>(nq, 1), 65536);
    if (top <= 256 || chunk_need(ix, top, P, Kc, dtype, &pl) <= budget) return top;
    int64_t lo = 256, hi = top;  // need(lo) is taken to fit, need(hi) does not
    while (hi - lo > 64) {
        const int64_t mid = (lo + hi) / 2;
        if (chunk_need(ix, mid, P, Kc, dtype, &pl) <= budget) lo = mid;
        else hi = mid;
    }
    return lo;
}

// reduced-precision candidates: the re-rank depth K' = 4k
static int rerank_depth(int k) { return 4 * k; }

// scratch a search of exactly nq queries asks its stream for (the largest
// of its query chunks)
static size_t search_need(const sivf_index *ix, int64_t nq, int k, int P, int dtype)
{
    if (nq <= 0) return 0;
    const int Kc = dtype == SIVF_FP32 ? k : rerank_depth(k);
    const int64_t qc = query_chunk(ix, nq, P, Kc, dtype);
    SearchPlan pl;
    size_t need = chunk_need(ix, std::min(qc, nq), P, Kc, dtype, &pl);
    if (nq > qc && nq % qc) need = std::max(need, chunk_need(ix, nq % qc, P, Kc, dtype, &pl));
    return need;
}

static size_t remove_need(const sivf_index *ix) { return (size_t)ix->nlist * 4 + 512; }

// compaction: staged rows for at most max_moves members (never more than
// n_max), the selected lists' offsets and the slab bases
static int64_t compact_rows(const sivf_index *ix, int64_t max_moves)
{
    return std::max<int64_t>(1, std::min<int64_t>(max_moves, ix->n_max));
}

static size_t compact_need(const sivf_index *ix, int64_t max_moves)
{
    const size_t d = ix->d, L = ix->nlist;
    const size_t row = d * 4 + (ix->xb16 ? d * 2 : 0) + (ix->x8 ? d : 0) + 4 +
                       (ix->rnorm ? 4 : 0) + 8;
    return L * 4 + (L + 1) * 16 + (size_t)ix->n_slabs * 4 +
           (size_t)compact_rows(ix, max_moves) * row + 10 * 256;
}

sivf_status sivf_reserve(sivf_index *ix, int64_t max_add, int64_t max_remove,
                         int64_t max_queries, int max_k, int max_nprobe, void *stream)
{
    if (!ix || max_add < 0 || max_remove < 0 || max_queries < 0 || max_k < 0 ||
        max_nprobe < 0)
        return fail(ix, SIVF_E_ARG, "negative reserve");
    size_t need = add_bytes(ix, std::max<int64_t>(max_add, 1));
    need = std::max(need, remove_need(ix));
    if (max_queries && max_k && max_nprobe) {
        const int P = std::min(max_nprobe, ix->nlist);
        // every batch size up to max_queries: the chunk plans differ by size
        for (int dt = 0; dt < 3; ++dt) {
            if ((dt == SIVF_BF16 && !ix->xb16) || (dt == SIVF_FP8E4M3 && !ix->x8)) continue;
            for (int64_t m = max_queries; m >= 1; m = m > 64 ? m * 3 / 4 : m - 1)
                need = std::max(need, search_need(ix, m, max_k, P, dt));
        }
    }
    sivf_status st = grow_rank_rows(ix, max_add, stream);
    if (st) return st;
    Ctx *c;
    return get_ctx(ix, stream, need, &c);
}

sivf_status sivf_add(sivf_index *ix, const int64_t *ids, const float *x, int64_t n,
                     void *stream, int64_t *n_added)
{
    if (n_added) *n_added = 0;
    if (!ix) return SIVF_E_ARG;
    if (n < 0 || n > INT32_MAX || (n > 0 && (!ids || !x)))
        return fail(ix, SIVF_E_ARG, "bad add arguments");
    if (!ix->have_centroids) return fail(ix, SIVF_E_STATE, "set_centroids first");
    sivf_status st = check_health(ix);
    if (st) return st;
    if (n == 0) return SIVF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = grow_rank_rows(ix, n, stream))) return st;
    Ctx *c;
    if ((st = get_ctx(ix, stream, add_bytes(ix, n), &c))) return st;
    Bump b{c->scratch};
    InsertScratch sc;
    const int L = ix->nlist;
    sc.lab = b.take<int32_t>(n);
    sc.rloc = b.take<int32_t>(n);
    sc.touched = b.take<int32_t>(L);
    sc.bcnt = b.take<int32_t>(L);
    sc.plan = b.take<PlanEntry>(L);
    sc.affected = b.take<int32_t>(L);
    const int64_t rows = coarse_rows(ix, n);
    float *Dbuf = b.take<float>((size_t)rows * L);
    CUDA_TRY(ix, cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s));
    coarse_topP(ix, x, n, 1, sc.lab, Dbuf, rows, s);
    insert_batch(ix, ids, x, n, sc, s);
    CUDA_TRY(ix, cudaGetLastError());
    if (n_added) return read_status(ix, stream, n_added);
    return SIVF_OK;
}

sivf_status sivf_remove(sivf_index *ix, const int64_t *ids, int64_t n, void *stream,
                        int64_t *n_removed)
{
    if (n_removed) *n_removed = 0;
    if (!ix) return SIVF_E_ARG;
    if (n < 0 || (n > 0 && !ids)) return fail(ix, SIVF_E_ARG, "bad remove arguments");
    sivf_status st = check_health(ix);
    if (st) return st;
    if (n == 0) return SIVF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx *c;
    if ((st = get_ctx(ix, stream, (size_t)ix->nlist * 4 + 512, &c))) return st;
    Bump b{c->scratch};
    int32_t *affected = b.take<int32_t>(ix->nlist);
    CUDA_TRY(ix, cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s));
    remove_batch(ix, ids, n, affected, s);
    CUDA_TRY(ix, cudaGetLastError());
    if (n_removed) return read_status(ix, stream, n_removed);
    return SIVF_OK;
}

sivf_status sivf_compact(sivf_index *ix, int32_t min_free, int64_t max_moves, void *stream,
                         int64_t *n_freed, int64_t *n_moved)
{
    if (n_freed) *n_freed = 0;
    if (n_moved) *n_moved = 0;
    if (!ix) return SIVF_E_ARG;
    if (min_free < 1 || max_moves < 1) return fail(ix, SIVF_E_ARG, "bad compact arguments");
    sivf_status st = check_health(ix);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = ix->nlist, d = ix->d;
    const int64_t R = compact_rows(ix, max_moves);
    const size_t need = compact_need(ix, max_moves);
    Ctx *c;
    if ((st = get_ctx(ix, stream, need, &c))) return st;
    Bump b{c->scratch};
    CompactArgs a;
    a.L = L;
    a.C = ix->C;
    a.W = ix->W;
    a.d = d;
    a.n_slabs = ix->n_slabs;
    a.dir_cap = ix->dir_cap;
    a.n_max = ix->n_max;
    a.list_live = ix->list_live;
    a.nslabs = ix->nslabs;
    a.dir = ix->dir;
    a.head = ix->head;
    a.free_list = ix->free_list;
    a.free_top = ix->free_top;
    a.bits = ix->bits;
    a.meta = ix->meta;
    a.x32 = ix->x32;
    a.xnorm = ix->xnorm;
    a.rnorm = ix->rnorm;
    a.xb16 = ix->xb16;
    a.x8 = ix->x8;
    a.ids = ix->ids;
    a.att = ix->att;
    a.sel = b.take<int32_t>(L);
    a.voff = b.take<int64_t>(L + 1);
    a.soff = b.take<int64_t>(L + 1);
    a.sb = b.take<int32_t>(ix->n_slabs);
    a.t32 = b.take<float>((size_t)R * d);
    a.t16 = ix->xb16 ? b.take<__nv_bfloat16>((size_t)R * d) : nullptr;
    a.t8 = ix->x8 ? b.take<uint8_t>((size_t)R * d) : nullptr;
    a.tn = b.take<float>(R);
    a.tr = ix->rnorm ? b.take<float>(R) : nullptr;
    a.ti = b.take<int64_t>(R);
    a.ctl = c->ctl;
    a.err = ix->err;
    CUDA_TRY(ix, cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s));
    compact_pass(ix, a, min_free, std::min<int64_t>(max_moves, R), s);
    CUDA_TRY(ix, cudaGetLastError());
    if (n_freed || n_moved) {
        st = read_status(ix, stream, nullptr);
        if (st) return st;
        if (n_freed) *n_freed = c->host->demand;
        if (n_moved) *n_moved = c->host->count;
    }
    return SIVF_OK;
}

}  // extern "C"

namespace sivf {
size_t op_need(const sivf_index *ix, const sivf_op &op)
{
    switch (op.kind) {
    case SIVF_OP_ADD: return add_bytes(ix, std::max<int64_t>(op.n, 1));
    case SIVF_OP_REMOVE: return remove_need(ix);
    case SIVF_OP_COMPACT: return compact_need(ix, op.n);
    default: return search_need(ix, op.n, op.k, op.nprobe, op.dtype);
    }
}

sivf_status reserve_stream(sivf_index *ix, void *stream, size_t need, int64_t max_add)
{
    sivf_status st = grow_rank_rows(ix, max_add, stream);
    if (st) return st;
    Ctx *c;
    return get_ctx(ix, stream, need, &c);
}

Ctl *stream_ctl(sivf_index *ix, void *stream)
{
    auto it = ex(ix).ctx.find(stream);
    return it == ex(ix).ctx.end() ? nullptr : it->second.ctl;
}

void release_stream(sivf_index *ix, void *stream)
{
    auto it = ex(ix).ctx.find(stream);
    if (it == ex(ix).ctx.end()) return;
    if (it->second.ctl) cudaFree(it->second.ctl);
    if (it->second.scratch) cudaFree(it->second.scratch);
    if (it->second.host) cudaFreeHost(it->second.host);
    ex(ix).ctx.erase(it);
}

sivf_status set_error(sivf_index *ix, sivf_status st, const char *what)
{
    return fail(ix, st, what);
}

void mark_corrupt(sivf_index *ix) { ex(ix).corrupt = true; }

sivf_status index_health(sivf_index *ix) { return check_health(ix); }
}  // namespace sivf

extern "C" {

static sivf_status search_impl(sivf_index *ix, const float *q, int64_t nq, int k, int nprobe,
                               const int32_t *probes_in, sivf_scan_dtype dtype, float *dist,
                               int64_t *labels, void *stream, int cand_only = 0,
                               bool probes_unique = false)
{
    if (!ix) return SIVF_E_ARG;
    if (nq < 0 || k < 1 || k > kMaxK || nprobe < 1 ||
        (!probes_in && (nprobe > ix->nlist || nprobe > kMaxK)) ||
        (probes_in && nprobe > kMaxK) || (nq > 0 && (!q || !dist || !labels)))
        return fail(ix, SIVF_E_ARG, "bad search arguments");
    if (dtype != SIVF_FP32 && dtype != SIVF_BF16 && dtype != SIVF_FP8E4M3)
        return fail(ix, SIVF_E_ARG, "unknown scan dtype");
    const bool tc = dtype != SIVF_FP32;
    if (tc && ((dtype == SIVF_BF16 && !ix->xb16) || (dtype == SIVF_FP8E4M3 && !ix->x8)))
        return fail(ix, SIVF_E_ARG, "that reduced-precision copy was not enabled at create");
    const int Kc = tc ? (cand_only ? k : rerank_depth(k)) : k;
    if (tc && (4 * k > 512 && !cand_only)) return fail(ix, SIVF_E_ARG, "k > 128 for a reduced-precision scan");
    if (tc && (Kc > 512 || !tc_fits(ix, Kc)))
        return fail(ix, SIVF_E_ARG, "k too large for the reduced-precision scan");
    if (!probes_in && !ix->have_centroids) return fail(ix, SIVF_E_STATE, "set_centroids first");
    sivf_status st = check_health(ix);
    if (st) return st;
    if (nq == 0) return SIVF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int P = nprobe, L = ix->nlist;
    if (!tc && !scan_fits(ix, k)) return fail(ix, SIVF_E_ARG, "k too large for this slab shape");
    const int64_t qc = query_chunk(ix, nq, P, Kc, dtype);
    for (int64_t q0 = 0; q0 < nq; q0 += qc) {
        const int64_t m = std::min(qc, nq - q0);
        SearchPlan pl;
        const size_t need = chunk_need(ix, m, P, Kc, dtype, &pl);
        Ctx *c;
        if ((st = get_ctx(ix, stream, need, &c))) return st;
        Bump b{c->scratch};
        SearchScratch sc{};
        int32_t *probes = b.take<int32_t>((size_t)m * P);
        sc.lcnt = b.take<int32_t>(L);
        sc.loff = b.take<int32_t>(L + 1);
        sc.ibase = b.take<int32_t>(L + 1);
        sc.nch = b.take<int32_t>(L);
        sc.prank = b.take<int32_t>((size_t)m * P);
        sc.qlist = b.take<int32_t>((size_t)m * P);
        sc.prun = b.take<int32_t>((size_t)m * P);
        sc.qrun = b.take<int2>((size_t)2 * m);
        sc.part_d = b.take<float>((size_t)pl.run_cap * pl.RK);
        sc.part_i = b.take<int64_t>((size_t)pl.run_cap * pl.RK);
        sc.part_n = tc ? b.take<int32_t>((size_t)pl.run_cap) : nullptr;
        sc.thr = b.take<float>((size_t)m);
        sc.items = b.take<int2>((size_t)pl.item_cap);
        sc.qn = b.take<float>((size_t)m);
        sc.qsc = b.take<float>((size_t)m);
        const bool fp8 = dtype == SIVF_FP8E4M3;
        sc.qcast = tc ? b.take<unsigned char>(fp8 ? (size_t)m * P * ix->d : (size_t)m * ix->d * 2)
                      : nullptr;
        sc.pqn = fp8 ? b.take<float>((size_t)m * P) : nullptr;
        sc.pqsc = fp8 ? b.take<float>((size_t)m * P) : nullptr;
        float *cand_d = b.take<float>((size_t)m * pl.K);
        int64_t *cand_s = b.take<int64_t>((size_t)m * pl.K);
        const int64_t rows = coarse_rows(ix, m);
        float *Dbuf = b.take<float>((size_t)rows * L);
        CUDA_TRY(ix, cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s));
        const float *qq = q + q0 * ix->d;
        if (probes_in)
            CUDA_TRY(ix, cudaMemcpyAsync(probes, probes_in + q0 * P, sizeof(int32_t) * m * P,
                                         cudaMemcpyDeviceToDevice, s));
        else
            coarse_topP(ix, qq, m, P, probes, Dbuf, rows, s);
        if (!tc) {
            scan_lists(ix, qq, m, P, probes, probes_in != nullptr && !probes_unique, pl, sc, s);
            merge_topk(ix, m, P, probes, pl, sc, k, dist + q0 * k, labels + q0 * k, s);
        } else {
            const int esz = dtype == SIVF_BF16 ? 2 : 1;
            // per slab: payload copy, ||x||^2 and the validity bitmap
            const int64_t sb = (int64_t)ix->C * (ix->d * esz + 4) + ix->C / 8;
            CUDA_TRY(ix, cudaMemsetAsync(sc.thr, 0x7f, sizeof(float) * m, s));
            if (fp8) pair_prep(ix, qq, m, P, probes, sc.pqn, sc.pqsc, sc.qcast, s);
            else query_prep(ix, qq, m, sc.qn, sc.qsc, sc.qcast, s);
            int nphase = 1;
            const bool dd = probes_in != nullptr && !probes_unique;  // repeated probes dropped
            const int seed = (128 + ix->C - 1) / ix->C;  // slabs of the first 128 rows
            if (P > 1 && (pl.split == 2 || (pl.qt && pl.split))) {
                // a seed launch over the first 128 rows of every query's
                // nearest list publishes a bound per query (no candidates
                // kept); the main launch then streams every probed list once
                group_pairs(ix, m, P, 0, 1, probes, dd, pl, sc, sb, s, false);
                if (pl.qt) scan_lists_qt(ix, dtype, m, P, Kc, seed, pl.sel, sc, s);
                else scan_lists_tc(ix, dtype, qq, m, P, Kc, pl, sc, s, seed);
                CUDA_TRY(ix, cudaMemsetAsync(&ix->ctl->nruns, 0, sizeof(int32_t), s));
                group_pairs(ix, m, P, 0, P, probes, dd, pl, sc, sb, s);
                if (pl.qt) scan_lists_qt(ix, dtype, m, P, Kc, 0, pl.sel, sc, s);
                else scan_lists_tc(ix, dtype, qq, m, P, Kc, pl, sc, s);
            } else if (pl.qt) {
                group_pairs(ix, m, P, 0, P, probes, dd, pl, sc, sb, s);
                scan_lists_qt(ix, dtype, m, P, Kc, 0, pl.sel, sc, s);
            } else {
                // vector-row scan.  With split == 1, phase 1: every query's
                // nearest list alone sets a tight bound on its K'-th
                // distance; phase 2 scans the other lists under it
                const int split = P > 1 && pl.split == 1 ? 1 : P;
                group_pairs(ix, m, P, 0, split, probes, dd, pl, sc, sb, s);
                scan_lists_tc(ix, dtype, qq, m, P, Kc, pl, sc, s);
                if (split < P) {
                    SearchPlan pl2 = pl;  // the other lists: the plan's phase-2 tile
                    pl2.tq = pl.tq2;
                    pl2.M = pl.M2;
                    group_pairs(ix, m, P, split, P, probes, dd, pl2, sc, sb, s);
                    scan_lists_tc(ix, dtype, qq, m, P, Kc, pl2, sc, s);
                }
                nphase = split < P ? 2 : 1;
            }
            if (cand_only) {
                merge_tc(ix, m, nphase, sc, Kc, pl.RK, dist + q0 * k, labels + q0 * k, s);
                slots_to_ids(ix, labels + q0 * k, m * k, s);
            } else {
                merge_rerank(ix, qq, m, nphase, sc, Kc, pl.RK, k, cand_d, cand_s, dist + q0 * k,
                             labels + q0 * k, s);
            }
        }
        CUDA_TRY(ix, cudaGetLastError());
    }
    return SIVF_OK;
}

sivf_status sivf_search(sivf_index *ix, const float *q, int64_t nq, int k, int nprobe,
                        sivf_scan_dtype dtype, float *dist, int64_t *labels, void *stream)
{
    return search_impl(ix, q, nq, k, nprobe, nullptr, dtype, dist, labels, stream);
}

sivf_status sivf_search_candidates(sivf_index *ix, const float *q, int64_t nq, int kc,
                                   int nprobe, sivf_scan_dtype dtype, float *dist,
                                   int64_t *labels, void *stream)
{
    if (dtype == SIVF_FP32) return fail(ix, SIVF_E_ARG, "candidates need a reduced-precision dtype");
    return search_impl(ix, q, nq, kc, nprobe, nullptr, dtype, dist, labels, stream, 1);
}

}  // extern "C"

// a search whose probes come from the library's own selection (distinct
// lists per query): the executor selects them on a side stream
sivf_status sivf::search_probed(sivf_index *ix, const float *q, int64_t nq, int k, int nprobe,
                                const int32_t *probes, sivf_scan_dtype dtype, float *dist,
                                int64_t *labels, void *stream)
{
    return search_impl(ix, q, nq, k, nprobe, probes, dtype, dist, labels, stream, 0, true);
}

extern "C" {

sivf_status sivf_search_with_probes(sivf_index *ix, const float *q, int64_t nq, int k,
                                    int nprobe, const int32_t *probes, sivf_scan_dtype dtype,
                                    float *dist, int64_t *labels, void *stream)
{
    if (!probes && nq > 0) return fail(ix, SIVF_E_ARG, "null probes");
    return search_impl(ix, q, nq, k, nprobe, probes, dtype, dist, labels, stream);
}

static sivf_status coarse_only(sivf_index *ix, const float *x, int64_t n, int P, int32_t *out,
                               void *stream)
{
    if (!ix) return SIVF_E_ARG;
    if (n < 0 || P < 1 || P > ix->nlist || P > kMaxK || (n > 0 && (!x || !out)))
        return fail(ix, SIVF_E_ARG, "bad coarse arguments");
    if (!ix->have_centroids) return fail(ix, SIVF_E_STATE, "set_centroids first");
    if (n == 0) return SIVF_OK;
    Ctx *c;
    sivf_status st = get_ctx(ix, stream, coarse_bytes(ix, n), &c);
    if (st) return st;
    Bump b{c->scratch};
    const int64_t rows = coarse_rows(ix, n);
    float *Dbuf = b.take<float>((size_t)rows * ix->nlist);
    coarse_topP(ix, x, n, P, out, Dbuf, rows, (cudaStream_t)stream);
    CUDA_TRY(ix, cudaGetLastError());
    return SIVF_OK;
}

sivf_status sivf_assign(sivf_index *ix, const float *x, int64_t n, int32_t *labels,
                        void *stream)
{
    return coarse_only(ix, x, n, 1, labels, stream);
}

sivf_status sivf_probe(sivf_index *ix, const float *q, int64_t nq, int nprobe,
                       int32_t *probes, void *stream)
{
    return coarse_only(ix, q, nq, nprobe, probes, stream);
}

sivf_status sivf_sync(sivf_index *ix, void *stream, int64_t *count)
{
    if (!ix) return SIVF_E_ARG;
    return read_status(ix, stream, count);
}

sivf_status sivf_stats(sivf_index *ix, void *stream, sivf_stats_t *out)
{
    if (!ix || !out) return fail(ix, SIVF_E_ARG, "null argument");
    memset(out, 0, sizeof *out);
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    int64_t stat[4] = {0, 0, 0, 0};
    int32_t top = 0;
    uint32_t err = 0;
    CUDA_TRY(ix, cudaMemcpy(stat, ix->stat, sizeof stat, cudaMemcpyDeviceToHost));
    const int64_t live = stat[0];
    out->pairs_scanned = stat[1];
    out->slab_bytes_scanned = stat[2];
    out->list_bytes_scanned = stat[3];
    CUDA_TRY(ix, cudaMemcpy(&top, ix->free_top, 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(ix, cudaMemcpy(&err, ix->err, 4, cudaMemcpyDeviceToHost));
    out->ntotal = live;
    out->free_slabs = top;
    out->used_slabs = ix->n_slabs - top;
    out->error_bits = err;
    out->last_status = ex(ix).last_status;
    out->last_count = ex(ix).last_count;
    const size_t S = ix->n_slabs, rows = S * ix->C, L = ix->nlist;
    out->bytes_device =
        (int64_t)(rows * ix->d * (4 + (ix->xb16 ? 2 : 0) + (ix->x8 ? 1 : 0)) + rows * 12 +
                  S * (ix->W * 4 + 16 + 4) + L * (ix->d * 4 + 4 * 8) + L * ix->dir_cap * 4 +
                  (size_t)ix->n_max * 12 + (size_t)L * ix->nblk_max * 4);
    if (err) ex(ix).corrupt = true;
    return SIVF_OK;
}

sivf_status sivf_dump(sivf_index *ix, void *stream, int32_t *list_nslabs, int32_t *list_head,
                      int32_t *list_dir, int32_t *slab_meta, uint32_t *slab_bits,
                      int64_t *slab_ids, int64_t *att, int32_t *free_stack, int64_t *n_free)
{
    if (!ix) return SIVF_E_ARG;
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    const size_t L = ix->nlist, S = ix->n_slabs;
    if (list_nslabs) CUDA_TRY(ix, cudaMemcpy(list_nslabs, ix->nslabs, L * 4, cudaMemcpyDeviceToHost));
    if (list_head) CUDA_TRY(ix, cudaMemcpy(list_head, ix->head, L * 4, cudaMemcpyDeviceToHost));
    if (list_dir)
        CUDA_TRY(ix, cudaMemcpy(list_dir, ix->dir, L * ix->dir_cap * 4, cudaMemcpyDeviceToHost));
    if (slab_meta) {
        std::vector<SlabMeta> m(S);
        CUDA_TRY(ix, cudaMemcpy(m.data(), ix->meta, S * sizeof(SlabMeta), cudaMemcpyDeviceToHost));
        for (size_t s = 0; s < S; ++s) {
            slab_meta[3 * s] = m[s].list;
            slab_meta[3 * s + 1] = m[s].fill;
            slab_meta[3 * s + 2] = m[s].live;
        }
    }
    if (slab_bits)
        CUDA_TRY(ix, cudaMemcpy(slab_bits, ix->bits, S * ix->W * 4, cudaMemcpyDeviceToHost));
    if (slab_ids)
        CUDA_TRY(ix, cudaMemcpy(slab_ids, ix->ids, S * ix->C * 8, cudaMemcpyDeviceToHost));
    if (att) CUDA_TRY(ix, cudaMemcpy(att, ix->att, (size_t)ix->n_max * 8, cudaMemcpyDeviceToHost));
    int32_t top = 0;
    CUDA_TRY(ix, cudaMemcpy(&top, ix->free_top, 4, cudaMemcpyDeviceToHost));
    if (n_free) *n_free = top;
    if (free_stack && top > 0)
        CUDA_TRY(ix, cudaMemcpy(free_stack, ix->free_list, (size_t)std::min<int64_t>(top, S) * 4,
                                cudaMemcpyDeviceToHost));
    return SIVF_OK;
}

sivf_status sivf_set_chunk_bytes(sivf_index *ix, int64_t bytes)
{
    if (!ix) return SIVF_E_ARG;
    if (bytes < 0) return fail(ix, SIVF_E_ARG, "chunk bytes must be >= 0");
    ix->chunk_bytes = bytes;
    return SIVF_OK;
}

sivf_status sivf_set_wait_limit(sivf_index *ix, int64_t ns)
{
    if (!ix || ns < 0) return fail(ix, SIVF_E_ARG, "negative wait limit");
    ix->wait_ns = ns == 0 ? kWaitNs : (uint64_t)ns;
    return SIVF_OK;
}

sivf_status sivf_debug_set_error_bits(sivf_index *ix, uint32_t bits, void *stream)
{
    if (!ix) return SIVF_E_ARG;
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t word = 0;
    CUDA_TRY(ix, cudaMemcpy(&word, ix->err, 4, cudaMemcpyDeviceToHost));
    word |= bits;
    CUDA_TRY(ix, cudaMemcpy(ix->err, &word, 4, cudaMemcpyHostToDevice));
    return SIVF_OK;
}

sivf_status sivf_profile(sivf_index *ix, int enable)
{
    if (!ix) return SIVF_E_ARG;
    CUDA_TRY(ix, cudaDeviceSynchronize());
    prof_clear(ix);
    ix->prof_on = enable != 0;
    return SIVF_OK;
}

sivf_status sivf_profile_read(sivf_index *ix, const char *kernel, int64_t *launches,
                              double *total_ms)
{
    if (!ix || !kernel) return fail(ix, SIVF_E_ARG, "null argument");
    static const char *names[PROF_NKIND] = {"coarse", "insert", "remove", "group", "scan",
                                            "merge", "rerank", "compact"};
    int kind = -1;
    for (int k = 0; k < PROF_NKIND; ++k)
        if (!strcmp(kernel, names[k])) kind = k;
    if (!strcmp(kernel, "all")) {
        if (launches) *launches = ix->launches;
        if (total_ms) *total_ms = 0.0;
        return SIVF_OK;
    }
    if (kind < 0) return fail(ix, SIVF_E_ARG, "unknown kernel group");
    CUDA_TRY(ix, cudaDeviceSynchronize());
    int64_t n = 0;
    double ms = 0.0;
    for (auto &e : ix->prof) {
        if (e.kind != kind) continue;
        float t = 0.f;
        CUDA_TRY(ix, cudaEventElapsedTime(&t, e.start, e.stop));
        ms += t;
        n += e.launches;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    return SIVF_OK;
}

sivf_status sivf_list_sizes(sivf_index *ix, void *stream, int32_t *sizes)
{
    if (!ix || !sizes) return fail(ix, SIVF_E_ARG, "null argument");
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    CUDA_TRY(ix, cudaMemcpy(sizes, ix->list_live, (size_t)ix->nlist * 4, cudaMemcpyDeviceToHost));
    return SIVF_OK;
}

sivf_status sivf_dump_payload(sivf_index *ix, void *stream, float *x32, uint16_t *xb16,
                              uint8_t *x8, float *inv_scale)
{
    if (!ix) return SIVF_E_ARG;
    CUDA_TRY(ix, cudaStreamSynchronize((cudaStream_t)stream));
    const size_t rows = (size_t)ix->n_slabs * ix->C;
    if (x32) CUDA_TRY(ix, cudaMemcpy(x32, ix->x32, rows * ix->d * 4, cudaMemcpyDeviceToHost));
    if (xb16) {
        if (!ix->xb16) return fail(ix, SIVF_E_ARG, "no BF16 copy");
        CUDA_TRY(ix, cudaMemcpy(xb16, ix->xb16, rows * ix->d * 2, cudaMemcpyDeviceToHost));
    }
    if (x8) {
        if (!ix->x8) return fail(ix, SIVF_E_ARG, "no FP8 copy");
        CUDA_TRY(ix, cudaMemcpy(x8, ix->x8, rows * ix->d, cudaMemcpyDeviceToHost));
    }
    if (inv_scale)
        CUDA_TRY(ix, cudaMemcpy(inv_scale, ix->inv_scale8, ix->nlist * 4, cudaMemcpyDeviceToHost));
    return SIVF_OK;
}

}  // extern "C"
