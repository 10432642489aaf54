// Host-side drivers of the kernels, one per step of the hot path.  Each
// enqueues its kernels on `st` and returns; scratch pointers come from the
// caller's arena.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <utility>

#include "sivf_internal.cuh"

namespace sivf {

// ---- programmatic dependent launch
// Every kernel of the library is launched with launch_pdl: outside a graph
// recording the hardware may make its blocks resident while the kernel
// before it on the stream still runs, so its launch latency hides under
// that kernel's tail (a single insert of 10,000 vectors: 0.058 -> 0.038 ms).
// Each kernel therefore begins with pdl_begin(): wait until the previous
// kernel has completed and its writes are visible (nothing is read or
// written before), then allow the next kernel to be scheduled in turn.
// While a sivf_exec records its queue (tl_recording) the kernels keep
// ordinary dependencies: a graph already launches its nodes ahead, and
// programmatic edges made the replayed benchmark step slower (0.382
// against 0.368 ms).  Launched the ordinary way, both instructions do
// nothing.
extern thread_local bool tl_recording;

__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... P, typename... A>
inline void launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       A &&...args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = tl_recording ? 0 : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // a failed launch is left in the runtime's last error, which every
    // caller checks after its launches
    (void)cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// ---- coarse quantizer (coarse.cu)
void centroid_prep(sivf_index *ix, cudaStream_t st);
cudaError_t assign_stage_choose(sivf_index *ix, cudaStream_t st);
int first_stage_split(const sivf_index *ix, int P);
// exact top-P set of each row of x, in ascending list index; Dbuf holds
// rows_per_chunk * nlist floats
// rows of one coarse chunk and the scratch of a coarse selection of n rows
int64_t coarse_rows(const sivf_index *ix, int64_t n);
size_t coarse_bytes(const sivf_index *ix, int64_t n);
// the search of sivf_search_with_probes for probes the library selected
// itself (distinct per query, so not de-duplicated)
sivf_status search_probed(sivf_index *ix, const float *q, int64_t nq, int k, int nprobe,
                          const int32_t *probes, sivf_scan_dtype dtype, float *dist,
                          int64_t *labels, void *stream);
void coarse_topP(sivf_index *ix, const float *x, int64_t m, int P, int32_t *out,
                 float *Dbuf, int64_t rows_per_chunk, cudaStream_t st);

// ---- quantizer training (train.cu)
// centroids := the given training rows (device, nlist of them)
void train_gather(sivf_index *ix, const float *x, const int64_t *rows, cudaStream_t st);
// one Lloyd update from the labels of the n rows: FP64 sums and counts
// (scratch), then centroids := FP32(mean); empty centroids keep their value
void train_step(sivf_index *ix, const float *x, int64_t n, const int32_t *lab, double *sum,
                int32_t *cnt, cudaStream_t st);

// ---- insert / delete (mutate.cu)
struct InsertScratch {
    int32_t *lab;        // [n] list of each vector
    int32_t *rloc;       // [n] rank among winners of its list in its block
    int32_t *touched;    // [nlist]
    int32_t *bcnt;       // [nlist] vectors per touched list
    PlanEntry *plan;     // [nlist]
    int32_t *affected;   // [nlist]
};
void insert_batch(sivf_index *ix, const int64_t *ids, const float *x, int64_t n,
                  const InsertScratch &s, cudaStream_t st);
void remove_batch(sivf_index *ix, const int64_t *ids, int64_t n, int32_t *affected,
                  cudaStream_t st);

// ---- search (scan.cu)
struct SearchScratch {
    int32_t *lcnt;       // [nlist] (query, list) pairs per list
    int32_t *loff;       // [nlist + 1]
    int32_t *ibase;      // [nlist + 1] first work item of each list
    int32_t *nch;        // [nlist] slab chunks of each list
    int32_t *prank;      // [nq * P] rank of the pair inside its list group
    int32_t *qlist;      // [nq * P] pairs grouped by list (q * P + p)
    float *part_d;       // [run_cap * RK] item outputs: one run per (pair, chunk)
    int64_t *part_i;     // [run_cap * RK]
    int32_t *part_n;     // [run_cap] valid entries of each run (reduced precision)
    float *thr;          // [nq] shared bound of each query's k-th distance
    int32_t *prun;       // [nq * P] run of the pair's chunk 0 (chunk c writes run
                         // prun + c); -1: the pair is not scanned
    int2 *qrun;          // [2 * nq] (first run, runs) of each query in each scan
                         // phase; a query's runs of one phase are contiguous
    int2 *items;         // [item_cap] work items (list, tile << 8 | chunk)
    float *qn;           // [nq] ||q||^2 (reduced-precision scans)
    float *qsc;          // [nq] FP8 inverse scale of each query
    unsigned char *qcast; // [nq, d] queries rounded to BF16, or [nq * P, d]
                          // E4M3 residuals of each (query, probe) pair
    float *pqn;          // [nq * P] ||q - c_l||^2 of each pair (FP8)
    float *pqsc;         // [nq * P] FP8 inverse scale of each pair's residual
};
struct SearchPlan {
    int tq;              // queries per work item
    int ch;              // most slab chunks per list (P * ch <= 2048 runs per query)
    int slabs_per_chunk; // slabs per chunk before splitting stops
    int ips;             // work items per SM the chunking aims at
    int64_t run_cap;     // output runs of one query chunk (both phases)
    int64_t item_cap;    // work items of one scan launch
    int K;               // candidates kept per query (K' for the reduced dtypes)
    int RK;              // entries of one output run (K for FP32; K' plus the room
                         // an approximate reduction may keep for the reduced dtypes)
    int M;               // entries of each row's k-select / candidate buffer
    int split;           // reduced precision, queries probing several lists: 1 =
                         // each query's nearest list in a launch of its own, then
                         // the other lists; 2 = a seed launch over the first 128
                         // rows of each query's nearest list (bounds only), then
                         // one launch over every probed list
    int qt;              // reduced precision: the query-row scan (scan_qt.cu)
    int sel;             // the tile's select_slabs (query-row scan: buffer cap)
    int tq2, M2;         // split 1, the other lists: queries per tile and buffer
                         // entries (32 and one tile of room for K' > 128 when
                         // that fits beside two stages; else tq and M)
};
// tile choice for a batch: the installed one of its bucket, else the default
int tune_bucket(const sivf_index *ix, int64_t nq, int P);
int tune_kbucket(int K);
sivf_tile default_tile(const sivf_index *ix, int dtype, int64_t nq, int P, int K);
sivf_tile current_tile(const sivf_index *ix, int dtype, int64_t nq, int P, int K);
bool tile_valid(const sivf_index *ix, int dtype, const sivf_tile &t, int K);
SearchPlan plan_from_tile(const sivf_index *ix, int dtype, int64_t nq, int P, int K,
                          const sivf_tile &t);
// FP32 plan (dtype 0) with the batch's current tile
SearchPlan plan_search(const sivf_index *ix, int64_t nq, int P, int K);
// output runs and work items one query chunk of nq queries may need
int64_t plan_run_cap(int64_t nq, int P, int tq, int ips);
int64_t plan_item_cap(int64_t nq, int P, int L, int ips);
bool scan_fits(const sivf_index *ix, int K);   // shared memory for k = K
void scan_lists(sivf_index *ix, const float *q, int64_t nq, int P, const int32_t *probes,
                bool dedupe, const SearchPlan &pl, const SearchScratch &s, cudaStream_t st);
// group the pairs with probe rank in [p0, p1) by list and lay out the work
// items and output runs; `stats` adds the scan's pairs and bytes to the
// index's counters (off for the seed launch of the query-row scan)
void group_pairs(sivf_index *ix, int64_t nq, int P, int p0, int p1, const int32_t *probes,
                 bool dedupe, const SearchPlan &pl, const SearchScratch &s, int64_t slab_bytes,
                 cudaStream_t st, bool stats = true);
void merge_topk(sivf_index *ix, int64_t nq, int P, const int32_t *probes,
                const SearchPlan &pl, const SearchScratch &s, int k, float *dist,
                int64_t *labels, cudaStream_t st);

// ---- reduced-precision scan + re-rank (scan_tc.cu)
bool tc_make_maps(sivf_index *ix);
// BF16 form: ||q||^2, unit scale and the row rounded to BF16
void query_prep(sivf_index *ix, const float *q, int64_t nq, float *qn, float *qsc,
                unsigned char *qcast, cudaStream_t st);
// FP8 residual scan: per (query, probe) pair ||q - c_l||^2, scale, E4M3 row
void pair_prep(sivf_index *ix, const float *q, int64_t nq, int P, const int32_t *probes,
               float *qn, float *qsc, unsigned char *qcast, cudaStream_t st);
bool tc_fits(const sivf_index *ix, int Kc);
// buffer entries of 32-query tiles for K' > 128 with one tile of room and
// two A stages, or 0 when they do not fit
int tc_wide_entries(const sivf_index *ix, int dtype, int Kc);
// entries of a row's candidate buffer (sel: tiles of room, 0 = default) and
// whether a buffer of M entries fits in shared memory
int tc_buf_entries(const sivf_index *ix, int dtype, int Kc, int sel);
bool tc_buf_fits(const sivf_index *ix, int dtype, int Kc, int M);
int tc_tile_queries(int Kc);   // 48 (K' <= 64), 32 (<= 128) or 16 (<= 512)
// seed_slabs > 0: a seed launch over the first seed_slabs slabs of each item
// that publishes each query's bound and writes no runs
void scan_lists_tc(sivf_index *ix, int dtype, const float *q, int64_t nq, int P, int Kc,
                   const SearchPlan &pl, const SearchScratch &s, cudaStream_t st,
                   int seed_slabs = 0);
void slots_to_ids(sivf_index *ix, int64_t *v, int64_t n, cudaStream_t st);
// per query: the best Kc (distance, slot) of its reduced-precision item
// outputs (the runs of `nphase` scan phases), sorted ascending
void merge_tc(sivf_index *ix, int64_t nq, int nphase, const SearchScratch &s, int Kc, int RK,
              float *out_d, int64_t *out_s, cudaStream_t st);
int tc_run_len(int Kc);  // RK of the vector-row scan for K' = Kc
void rerank(sivf_index *ix, const float *q, int64_t nq, int Kc, const float *cand_d,
            const int64_t *cand_s, int k, float *dist, int64_t *labels, cudaStream_t st);
// merge of the reduced-precision scan's runs and FP32 re-rank, fused into
// one kernel for K' <= 128 (cand_d / cand_s are used only beyond that)
void merge_rerank(sivf_index *ix, const float *q, int64_t nq, int nphase,
                  const SearchScratch &s, int Kc, int RK, int k, float *cand_d,
                  int64_t *cand_s, float *dist, int64_t *labels, cudaStream_t st);

// ---- reduced-precision scan, queries on the tensor-memory lanes (scan_qt.cu)
struct QtShape {
    bool ok;             // the shape fits for this dtype, d, slab size and K'
    int KC;              // 128-byte chunks of a row in the scan format
    int NV;              // slab rows per B tile (128 / KC)
    int nst;             // B stages
    int ME;              // entries of a query row's candidate buffer
    size_t smem;         // dynamic shared memory of the CTA
};
QtShape qt_shape(const sivf_index *ix, int dtype, int Kc);
bool qt_make_maps(sivf_index *ix, PFN_cuTensorMapEncodeTiled_v12000 enc);
// the driver's cuTensorMapEncodeTiled (null when unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn();
// TMA descriptor of the BF16 centroids for the fused coarse first stage;
// false when the shape does not take that stage
bool coarse_make_map(sivf_index *ix);
// one launch over the grouped items; seed_slabs > 0 scans only the first
// seed_slabs slabs of each item and publishes the bounds, writing no runs;
// select_slabs is the tile's buffer-length knob (qt_mecap)
void scan_lists_qt(sivf_index *ix, int dtype, int64_t nq, int P, int Kc, int seed_slabs,
                   int select_slabs, const SearchScratch &s, cudaStream_t st);
int qt_mecap(int select_slabs);

// ---- compaction of partly-live slabs (compact.cu)
struct CompactArgs {
    int L, C, W, d;
    int64_t n_slabs, dir_cap, n_max;
    const int32_t *list_live;
    int32_t *nslabs, *dir, *head, *free_list, *free_top;
    uint32_t *bits;
    SlabMeta *meta;
    float *x32, *xnorm, *rnorm;
    __nv_bfloat16 *xb16;
    uint8_t *x8;
    int64_t *ids, *att;
    // scratch: selected lists, their member and slab offsets [L + 1], the
    // live members before each of their slabs, and the staged rows
    int32_t *sel;
    int64_t *voff, *soff;
    int32_t *sb;
    float *t32, *tn, *tr;
    __nv_bfloat16 *t16;
    uint8_t *t8;
    int64_t *ti;
    Ctl *ctl;
    uint32_t *err;
};
// one pass; the control block receives the lists (ntouched), the members
// rewritten (count) and the slabs freed (demand)
void compact_pass(sivf_index *ix, const CompactArgs &a, int min_free, int64_t max_moves,
                  cudaStream_t st);

// ---- C-ABI internals shared with the executor (abi.cu)
size_t op_need(const sivf_index *ix, const sivf_op &op);   // scratch of one batch
sivf_status reserve_stream(sivf_index *ix, void *stream, size_t need, int64_t max_add);
Ctl *stream_ctl(sivf_index *ix, void *stream);
void release_stream(sivf_index *ix, void *stream);        // free a stream's scratch
sivf_status set_error(sivf_index *ix, sivf_status st, const char *what);
void mark_corrupt(sivf_index *ix);
// SIVF_E_CORRUPT once a synchronising call has seen a device error bit (the
// index then refuses further work), else SIVF_OK
sivf_status index_health(sivf_index *ix);

}  // namespace sivf
