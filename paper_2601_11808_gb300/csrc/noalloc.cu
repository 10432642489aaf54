// sivf_search_noalloc: the FP32 search with no device allocation at call
// time.
//
// Some callers cannot let a library allocate device memory when they call
// it: a serving process that has handed all device memory to its own pool
// (a cudaMalloc there fails or fragments the pool), or a latency-critical
// loop that must never enter the driver's allocator.  This entry point runs
// the same kernels as sivf_search (coarse selection, grouping by list, list
// scan, per-query merge) but takes every scratch buffer from one fixed
// array in device memory that the library declares at file scope, so the
// call itself allocates nothing.  The caller still owns and passes the
// queries and the output arrays.
//
// The array (SIVF_NOALLOC_SCRATCH_BYTES, 32 MiB) exists on every GPU that
// loads the library, from load until process exit.  In host code its name
// is only a host-side stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device.  All calls on a device share the array and it
// keeps the last call's contents; every buffer that must start at zero is
// cleared by each call.  Two calls whose work overlaps on the GPU (different
// streams, or different indexes on the same device) race on the array: the
// caller must order them.
#include <stdio.h>

#include <mutex>

#include "kernels.cuh"

namespace {

constexpr size_t kNoallocBytes = (size_t)SIVF_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
void *g_base[kMaxDevices];   // device address of the array, per device

// carve-up of the array for one call
struct Carve {
    char *base;
    size_t off = 0, cap;
    template <class T>
    T *take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += n * sizeof(T);
        return p;
    }
    bool ok() const { return off <= cap; }
};

size_t need_bytes(const sivf_index *ix, int64_t nq, int P, const sivf::SearchPlan &pl,
                  int64_t rows)
{
    const size_t L = ix->nlist;
    size_t b = 0;
    auto add = [&](size_t n) { b = ((b + 255) & ~(size_t)255) + n; };
    add(sizeof(sivf::Ctl));
    add((size_t)nq * P * 4);          // probes
    add(L * 4);                       // lcnt
    add((L + 1) * 4);                 // loff
    add((L + 1) * 4);                 // ibase
    add(L * 4);                       // nch
    add((size_t)nq * P * 4);          // prank
    add((size_t)nq * P * 4);          // qlist
    add((size_t)pl.run_cap * pl.K * 4);   // part_d
    add((size_t)pl.run_cap * pl.K * 8);   // part_i
    add((size_t)nq * 4);              // thr
    add((size_t)nq * P * 4);          // prun
    add((size_t)nq * 2 * 8);          // qrun
    add((size_t)pl.item_cap * 8);     // items
    add((size_t)rows * L * 4);        // coarse distances
    return b;
}

}  // namespace

extern "C" sivf_status sivf_search_noalloc(sivf_index *ix, const float *q, int64_t nq, int k,
                                           int nprobe, float *dist, int64_t *labels,
                                           void *stream)
{
    using namespace sivf;
    if (!ix) return SIVF_E_ARG;
    auto fail = [&](sivf_status st, const char *m) {
        ix->last_error = m;
        return st;
    };
    if (nq < 0 || k < 1 || k > kMaxK || nprobe < 1 || nprobe > ix->nlist || nprobe > kMaxK ||
        (nq > 0 && (!q || !dist || !labels)))
        return fail(SIVF_E_ARG, "bad search arguments");
    if (!ix->have_centroids) return fail(SIVF_E_STATE, "set_centroids first");
    const sivf_status health = index_health(ix);
    if (health != SIVF_OK) return health;
    if (nq == 0) return SIVF_OK;
    if (!scan_fits(ix, k)) return fail(SIVF_E_ARG, "k too large for this slab shape");

    // the plan of sivf_search, narrowed until its scratch fits the array
    const int P = nprobe, L = ix->nlist;
    SearchPlan pl = plan_search(ix, nq, P, k);
    int64_t rows = std::min<int64_t>(nq, std::max<int64_t>(1, ((int64_t)8 << 20) / (4 * L)));
    // fewer items per SM: fewer extra chunk runs
    while (need_bytes(ix, nq, P, pl, rows) > kNoallocBytes && pl.ips > 1) {
        pl.ips >>= 1;
        pl.run_cap = plan_run_cap(nq, P, pl.tq, pl.ips);
        pl.item_cap = plan_item_cap(nq, P, L, pl.ips);
    }
    while (need_bytes(ix, nq, P, pl, rows) > kNoallocBytes && rows > 1) rows >>= 1;
    if (need_bytes(ix, nq, P, pl, rows) > kNoallocBytes) {
        char b[200];
        snprintf(b, sizeof b,
                 "sivf_search_noalloc: %lld queries x nprobe %d x k %d need %zu bytes of "
                 "scratch, above the fixed %zu",
                 (long long)nq, P, k, need_bytes(ix, nq, P, pl, rows), kNoallocBytes);
        ix->last_error = b;
        return SIVF_E_ARG;
    }

    // device address of the array on the current device, looked up once
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(SIVF_E_CUDA, "cudaGetDevice failed");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_base[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return fail(SIVF_E_CUDA, "cudaGetSymbolAddress failed");
            g_base[dev] = p;
        }
        base = g_base[dev];
    }

    cudaStream_t s = (cudaStream_t)stream;
    Carve c{reinterpret_cast<char *>(base), 0, kNoallocBytes};
    Ctl *ctl = c.take<Ctl>(1);
    int32_t *probes = c.take<int32_t>((size_t)nq * P);
    SearchScratch sc{};
    sc.lcnt = c.take<int32_t>(L);
    sc.loff = c.take<int32_t>(L + 1);
    sc.ibase = c.take<int32_t>(L + 1);
    sc.nch = c.take<int32_t>(L);
    sc.prank = c.take<int32_t>((size_t)nq * P);
    sc.qlist = c.take<int32_t>((size_t)nq * P);
    sc.part_d = c.take<float>((size_t)pl.run_cap * pl.K);
    sc.part_i = c.take<int64_t>((size_t)pl.run_cap * pl.K);
    sc.thr = c.take<float>((size_t)nq);
    sc.prun = c.take<int32_t>((size_t)nq * P);
    sc.qrun = c.take<int2>((size_t)nq * 2);
    sc.items = c.take<int2>((size_t)pl.item_cap);
    float *Dbuf = c.take<float>((size_t)rows * L);
    if (!c.ok()) return fail(SIVF_E_ARG, "scratch carve-up overflow");

    // the control block starts at zero on every call (lcnt is cleared by
    // the grouping step itself); the kernels take the index's control
    // block pointer at launch, so the index's own one is put back after
    // the launches are enqueued
    Ctl *own = ix->ctl;
    ix->ctl = ctl;
    if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess) {
        ix->ctl = own;
        return fail(SIVF_E_CUDA, "cudaMemsetAsync failed");
    }
    coarse_topP(ix, q, nq, P, probes, Dbuf, rows, s);
    scan_lists(ix, q, nq, P, probes, false, pl, sc, s);
    merge_topk(ix, nq, P, probes, pl, sc, k, dist, labels, s);
    ix->ctl = own;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SIVF_E_CUDA, cudaGetErrorString(e));
    return SIVF_OK;
}
