/*
 * sivf.h -- C ABI of libsivf, a GB300 (sm_103a) streaming IVF-Flat index
 * whose inverted lists are chains of fixed-size slabs, after
 * "SIVF: GPU-Resident IVF Index for Streaming Vector Search"
 * (arxiv 2601.11808).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments marked [device] are device pointers in the index's
 *    CUDA device; arrays marked [host] are host memory.  The caller owns
 *    every array it passes; the library never frees or keeps them past the
 *    call's stream work.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it and the call returns without waiting,
 *    except where an argument marked "forces a sync" is non-NULL.
 *  - Layouts are row-major and dense: a [n, d] float array holds vector i
 *    at elements i*d .. i*d+d-1.  Vectors are float32; ids are int64 in
 *    the dense id space [0, n_max) (the paper's data model, Sec. 3).
 *  - Distances are squared L2 (the paper writes d(q, x); squared L2 is the
 *    IVF-Flat convention it builds on), returned in float32.
 *  - Every call checks its host-visible arguments first and returns
 *    SIVF_E_ARG without enqueuing anything when one is wrong.  Conditions
 *    only the device can see (an id out of range inside a device array, a
 *    full slab pool) reject the whole batch on the device: no state
 *    changes, and the status is reported by the call itself when it syncs,
 *    otherwise by the next sivf_sync().
 *  - A device loop that hits its bound (a corrupt directory) records a
 *    sticky error and returns; nothing traps.  A device wait that runs out
 *    of time (2 s by default, sivf_set_wait_limit) records a sticky
 *    timeout the same way.  The next synchronising call returns
 *    SIVF_E_CORRUPT / SIVF_E_TIMEOUT and every later call returns
 *    SIVF_E_CORRUPT without enqueuing anything.
 *  - One index is driven by one host thread at a time.  Calls on the same
 *    stream are ordered; the library does not order calls across streams.
 *  - Scratch memory grows on demand with cudaMalloc; call sivf_reserve()
 *    first when the calls will be captured into a CUDA graph.
 */
#ifndef SIVF_H
#define SIVF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sivf_index sivf_index;

typedef enum {
    SIVF_OK = 0,
    SIVF_E_ARG = 1,      /* bad argument (host check, or an id out of range) */
    SIVF_E_NOMEM = 2,    /* slab pool, list directory or device memory full  */
    SIVF_E_STATE = 3,    /* set_centroids has not been called                */
    SIVF_E_CUDA = 4,     /* a CUDA call failed                               */
    SIVF_E_CORRUPT = 5,  /* a bounded device walk hit its bound (sticky)     */
    SIVF_E_TIMEOUT = 6   /* a bounded device wait ran out (sticky)           */
} sivf_status;

typedef enum {
    SIVF_FP32 = 0,       /* exact FP32 scan of the FP32 payload              */
    SIVF_BF16 = 1,       /* BF16 scan on tensor cores + FP32 re-rank         */
    SIVF_FP8E4M3 = 2     /* FP8 E4M3 scan (per-list scale) + FP32 re-rank    */
} sivf_scan_dtype;

typedef struct {
    int d;               /* dimension, 4 <= d <= 256, d % 4 == 0            */
    int nlist;           /* inverted lists, 1 <= nlist <= 65536             */
    int slab_size;       /* slab capacity C: 32, 64 or 128, C * d <= 20480   */
    int64_t n_max;       /* size of the dense id space [0, n_max)            */
    int64_t n_slabs;     /* slabs in the pre-allocated pool (the paper's S)  */
    int64_t dir_cap;     /* most slabs one list may hold (0 = n_slabs)       */
    uint32_t scan_dtypes;/* extra payload copies: bit (1<<SIVF_BF16) and/or
                            bit (1<<SIVF_FP8E4M3), which need d % 16 == 0;
                            the FP32 copy always exists                     */
} sivf_config;

typedef struct {
    int64_t ntotal;      /* live vectors                                     */
    int64_t free_slabs;  /* slabs on the free stack                          */
    int64_t used_slabs;  /* slabs held by lists                              */
    uint32_t error_bits; /* sticky device error word (0 = healthy)           */
    int32_t last_status; /* status of the last add/remove batch (sivf_status)*/
    int64_t last_count;  /* vectors added / removed by that batch            */
    int64_t bytes_device;/* device memory held by the index                  */
    int64_t pairs_scanned;      /* (query, live vector) pairs the list scans
                                   have scored since creation (FP32 path)    */
    int64_t slab_bytes_scanned; /* slab bytes the list scans streamed since
                                   creation (payload, ids or norms, bitmap),
                                   one read per (list, query tile)           */
    int64_t list_bytes_scanned; /* the same counted once per list a scan
                                   launch probes: the unique bytes of the
                                   probed lists, the list-centric bound     */
} sivf_stats_t;

/*
 * sivf_create -- allocate an empty index and its slab pool on the current
 * CUDA device (Sec. 3.1: a monolithic pre-allocated pool of S slabs of C
 * vectors, per-list heads, a free stack and the address translation table).
 * `cfg` [host] is read once.  On success *out receives the handle.
 * Errors: SIVF_E_ARG (bad config), SIVF_E_NOMEM (cudaMalloc failed).
 */
sivf_status sivf_create(const sivf_config *cfg, sivf_index **out);

/* sivf_destroy -- synchronize the device and free everything the index
 * holds.  NULL is accepted. */
sivf_status sivf_destroy(sivf_index *index);

/*
 * sivf_save -- checkpoint: write the index's configuration and every array
 * that carries its state (centroids, FP8 scales, the slab pool with its
 * payload copies, norms, ids, bitmaps and slab metadata, the free stack,
 * list heads, directories and live counts, the address table, the live
 * and scan counters) to the file `path` [host string].  Synchronizes
 * `stream`.  The paper has no counterpart (its index lives as long as its
 * process).  Errors: SIVF_E_ARG (file cannot be written), SIVF_E_CORRUPT
 * (the index has a sticky device error), SIVF_E_CUDA.
 *
 * sivf_load -- create an index on the current device from a file written by
 * sivf_save; every saved array is restored bit for bit (derived arrays are
 * recomputed), so searches and later updates give the same results as on
 * the saved index.  Scan tiles installed with sivf_set_tile are not saved.
 * Errors: SIVF_E_ARG (missing, foreign or truncated file), SIVF_E_NOMEM,
 * SIVF_E_CUDA.
 */
sivf_status sivf_save(sivf_index *index, const char *path, void *stream);
sivf_status sivf_load(const char *path, sivf_index **out);

/*
 * sivf_set_centroids -- load the coarse quantizer (Sec. 3.3: the lists are
 * the cells of nearest-centroid assignment).  `c` [device] is [nlist, d]
 * float32.  The index must be empty (SIVF_E_STATE otherwise).  Also sets
 * every list's FP8 inverse scale to fl32(448 / R_l), R_l the distance from
 * c_l to its nearest other centroid (FP64); with one list or R_l = 0,
 * fl32(448 / (2 * max_j |c_lj|)) (1.0 when the centroid is zero);
 * sivf_set_list_scales overrides it.  Then picks the first stage of
 * nearest-list assignment (sivf_assign_stage) from the centroid spacing
 * and synchronizes `stream`.
 */
sivf_status sivf_set_centroids(sivf_index *index, const float *c, void *stream);

/*
 * sivf_assign_stage -- the first stage that nearest-list assignment (the
 * insert's coarse step, sivf_assign, probe selection at nprobe 1) takes on
 * the current centroids: 1 the single BF16 tensor-core product, 3 the split
 * BF16 products (x_hi c_hi + x_hi c_lo + x_lo c_hi), 0 FP32; -1 for NULL or
 * an index without centroids.  Every stage gives the same assignment (the
 * FP64 nearest centroid, ties to the lowest index, Sec. 3.3): a row whose
 * first-stage bound does not isolate one list is re-decided exactly.  The
 * single product is taken unless twice its bound at the largest centroid
 * norm, 4 gamma max ||c||^2 with gamma = 2 (2 u + u^2 + d 2^-22 (1 + u)^2),
 * u = 2^-8, exceeds the median over lists of the squared distance from a
 * centroid to its nearest other centroid (FP32): then most rows would need
 * the re-decision and the split stage (a bound about 60x tighter) is taken.
 * Chosen by sivf_set_centroids, sivf_train and sivf_load.
 */
int32_t sivf_assign_stage(const sivf_index *index);

/*
 * sivf_train -- train the coarse quantizer by Lloyd's k-means and install
 * it as sivf_set_centroids does.  The paper uses a trained Faiss quantizer
 * and does not describe training (Sec. 4.1); this is the plain reading.
 *   x [device] float32[n, d] training rows, nlist <= n <= 2^31 - 1;
 *   iters >= 0 Lloyd iterations; seed picks the initial centroids.
 * Initial centroids: the training rows r_t = (t-th SplitMix64 output from
 * state `seed`) mod n, in draw order, rows already taken skipped, until
 * nlist rows are taken (SplitMix64: Steele, Lea and Flood, OOPSLA 2014).
 * One iteration: every row goes to its nearest centroid (exactly as
 * sivf_assign: FP64 definition, ties to the lowest index); every centroid
 * with at least one row becomes the FP32 rounding of the FP64 mean of its
 * rows; a centroid with no rows keeps its value.  The FP64 sums are
 * accumulated with device atomics, so their last bits may depend on the
 * order of the additions; the FP32 result is the same unless a mean lies
 * within an FP64 rounding of an FP32 rounding boundary.
 * The index must be empty (SIVF_E_STATE); synchronizes `stream` at entry.
 */
sivf_status sivf_train(sivf_index *index, const float *x, int64_t n, int iters,
                       uint64_t seed, void *stream);

/*
 * sivf_get_centroids -- copy the current coarse quantizer (as loaded by
 * sivf_set_centroids or produced by sivf_train) to `c` [device]
 * float32[nlist, d].  SIVF_E_STATE before any centroids exist.
 */
sivf_status sivf_get_centroids(sivf_index *index, float *c, void *stream);

/*
 * sivf_set_list_scales -- per-list FP8 E4M3 inverse scales: list l stores the
 * residual codes code(fl32(fl32(x_j - c_lj) * inv_scale[l])) and decodes
 * x_j ~ c_lj + code / inv_scale[l].
 * `inv_scale` [device] is [nlist] float32, each finite and > 0.  Must be
 * called while the index is empty.
 */
sivf_status sivf_set_list_scales(sivf_index *index, const float *inv_scale,
                                 void *stream);

/*
 * sivf_reserve -- pre-allocate the scratch of `stream` for batches up to the
 * given sizes so that later calls on that stream allocate nothing (needed
 * before CUDA-graph capture).  Scratch is per stream: calls on different
 * streams never share it.
 */
sivf_status sivf_reserve(sivf_index *index, int64_t max_add, int64_t max_remove,
                         int64_t max_queries, int max_k, int max_nprobe,
                         void *stream);

/*
 * sivf_add -- batched insert (Algorithm 2, redone as a conflict-free batch).
 *   ids [device] int64[n], x [device] float32[n, d].
 * Semantics of one batch:
 *   1. the last occurrence of each id wins;
 *   2. each kept vector goes to its nearest centroid's list, ties to the
 *      lowest list index (the assignment equals an FP64 argmin bit-exactly);
 *   3. admission, all or nothing: the slab demand of the batch, computed on
 *      the state before it, must fit the free slabs and every list's
 *      directory capacity, else SIVF_E_NOMEM (Sec. 3.2 fail-fast) and
 *      nothing changes; an id outside [0, n_max) gives SIVF_E_ARG, also with
 *      nothing changed;
 *   4. kept ids that are live are deleted first (delete-then-insert, Sec. 3);
 *   5. kept vectors are appended to their lists in batch order: a list fills
 *      its head slab, then takes fresh slabs from the free stack.  Each
 *      vector is published by setting its validity bit after its payload,
 *      id and address-table entry are written (Theorem 1).
 * n_added [host, optional]: if non-NULL the call forces a sync, stores the
 * number of kept ids and returns the batch status.
 */
sivf_status sivf_add(sivf_index *index, const int64_t *ids, const float *x,
                     int64_t n, void *stream, int64_t *n_added);

/*
 * sivf_remove -- batched delete (Algorithm 4: address-table lookup, atomic
 * clear of the validity bit, live-count decrement; a slab whose live count
 * reaches zero leaves its list and returns to the free stack).  Holes are
 * not refilled here (sivf_compact does that on request).  Absent and
 * repeated ids are no-ops (Theorem 3).
 *   ids [device] int64[n]; an id outside [0, n_max) rejects the batch with
 *   SIVF_E_ARG and nothing changes.
 * n_removed [host, optional]: if non-NULL the call forces a sync, stores the
 * number of ids actually removed and returns the batch status.
 */
sivf_status sivf_remove(sivf_index *index, const int64_t *ids, int64_t n,
                        void *stream, int64_t *n_removed);

/*
 * sivf_compact -- one pass of compaction of partly-live slabs.  Deletes
 * leave holes (a slab returns to the pool only when its last vector goes);
 * the paper names adaptive background compaction as future work
 * (Conclusion) and gives no algorithm, so this is a reading of it: a list
 * whose live members would fit in at least `min_free` (>= 1) fewer slabs is
 * rewritten densely in its member order (slab position, then slot): member
 * j moves to slot j mod C of the list's (j div C)-th slab, with its FP32
 * row, reduced-precision copies, norms, id and address-table entry; the
 * list keeps its first ceil(n / C) slabs (the last one stays open for
 * appends) and the rest go back on the free stack.  Lists are taken in
 * index order while the running total of rewritten members stays within
 * `max_moves` (>= 1); the first list that would pass it ends the pass.
 * Membership, member order and every search result are unchanged.  Scratch
 * grows by about max_moves rows (capped at n_max).
 * n_freed, n_moved [host, optional]: if either is non-NULL the call syncs
 * and stores the slabs returned to the pool and the members rewritten.
 */
sivf_status sivf_compact(sivf_index *index, int32_t min_free, int64_t max_moves,
                         void *stream, int64_t *n_freed, int64_t *n_moved);

/*
 * sivf_search -- batched k-NN (Algorithm 3 redone list-centrically): coarse
 * selection of the nprobe nearest lists (the exact FP64 top-nprobe set, ties
 * to the lowest index), a scan of every live slot of those lists, and a
 * top-k per query in ascending (distance, id) order.
 *   q [device] float32[nq, d]; dist [device] float32[nq, k];
 *   labels [device] int64[nq, k].  Missing results are (+inf, -1).
 *   1 <= k <= 1024 (and small enough that a slab pair plus 8 queries' best
 *   k fit in shared memory: SIVF_E_ARG otherwise); 1 <= nprobe <=
 *   min(nlist, 1024).
 * dtype SIVF_FP32 scans the FP32 payload with direct-form distances.
 * SIVF_BF16 / SIVF_FP8E4M3 scan the reduced copy (which must have been
 * enabled at create; d % 16 == 0) on tensor cores, keep the best 4k
 * candidates per query (k <= 128) and re-rank them with exact FP32
 * direct-form distances from the FP32 payload.  The FP8 copy holds the
 * residuals x - c_l of each list; the query is coded per (query, list)
 * pair as q - c_l with its own scale 448 / (2 max_j |q_j - c_lj|).
 */
sivf_status sivf_search(sivf_index *index, const float *q, int64_t nq, int k,
                        int nprobe, sivf_scan_dtype dtype, float *dist,
                        int64_t *labels, void *stream);

/*
 * sivf_search_candidates -- the first stage of a reduced-precision search
 * alone: the `kc` best candidates of each query by the reduced-precision
 * distance ||q||^2 + ||x||^2 - 2 s q^.x^ over the nprobe nearest lists
 * (q^, x^ the BF16 roundings of q and x, or for FP8 the E4M3 codes of the
 * residuals q - c_l, x - c_l with ||q - c_l||^2, ||x - c_l||^2 as the norms;
 * FP32 accumulation), ascending, ties to
 * the lower slot.  dist [device] float32[nq, kc] holds those approximate
 * distances, labels [device] int64[nq, kc] the ids; padding (+inf, -1).
 * 1 <= kc <= 128; dtype SIVF_BF16 or SIVF_FP8E4M3.
 */
sivf_status sivf_search_candidates(sivf_index *index, const float *q, int64_t nq,
                                   int kc, int nprobe, sivf_scan_dtype dtype,
                                   float *dist, int64_t *labels, void *stream);

/*
 * sivf_search_noalloc -- the FP32 search of sivf_search for callers that
 * cannot let a library allocate device memory during a call (a serving
 * process whose memory pool owns the whole device, a latency-critical loop
 * that must stay out of the allocator).  The paper has no counterpart; it
 * is an interface addition of this library.
 *   Same arguments, layouts, results and errors as sivf_search with
 *   dtype SIVF_FP32; the caller passes q [device], dist [device] and
 *   labels [device] as there.
 *   No cudaMalloc or cudaFree happens inside the call: every scratch buffer
 *   comes from one array of SIVF_NOALLOC_SCRATCH_BYTES bytes declared in
 *   the library's device code, held by every GPU that loads the library
 *   until the process exits.  A batch whose scratch does not fit (roughly
 *   (nq * nprobe + 2 * 152 * tq * ips) * k * 12 bytes of item outputs, tq
 *   the queries per scan tile and ips the tile's items per SM, which the
 *   call lowers to 1 before refusing, plus nlist-sized tables) is refused
 *   with SIVF_E_ARG and a message giving the bytes it needs.
 *   The first call on a device looks the array's device address up (once
 *   per device, with that device current); make that first call before any
 *   stream capture begins.
 *   All calls share the array and it keeps the last call's contents; calls
 *   whose work overlaps on the GPU (other streams, other indexes on the
 *   same device) race on it and must be ordered by the caller.
 */
#define SIVF_NOALLOC_SCRATCH_BYTES (32u << 20)
sivf_status sivf_search_noalloc(sivf_index *index, const float *q, int64_t nq,
                                int k, int nprobe, float *dist, int64_t *labels,
                                void *stream);

/*
 * sivf_search_with_probes -- the fine scan and top-k of sivf_search with
 * caller-given lists: probes [device] int32[nq, nprobe] (entries outside
 * [0, nlist) are skipped; a list given twice is scanned once).
 */
sivf_status sivf_search_with_probes(sivf_index *index, const float *q,
                                    int64_t nq, int k, int nprobe,
                                    const int32_t *probes, sivf_scan_dtype dtype,
                                    float *dist, int64_t *labels, void *stream);

/*
 * sivf_assign -- the coarse assignment step of sivf_add alone:
 * labels [device] int32[n] = argmin_l ||x_i - c_l||^2, ties to the lowest l.
 */
sivf_status sivf_assign(sivf_index *index, const float *x, int64_t n,
                        int32_t *labels, void *stream);

/*
 * sivf_probe -- the coarse selection step of sivf_search alone:
 * probes [device] int32[nq, nprobe] holds the nprobe nearest lists of each
 * query; the set equals the FP64 top-nprobe by (distance, index), listed
 * nearest first by the FP32 approximate distance (ties to the lower index).
 */
sivf_status sivf_probe(sivf_index *index, const float *q, int64_t nq,
                       int nprobe, int32_t *probes, void *stream);

/*
 * sivf_sync -- wait for the stream and return the status of the last
 * add/remove batch (or a sticky error); *count [host, optional] receives the
 * vectors that batch added or removed.
 */
sivf_status sivf_sync(sivf_index *index, void *stream, int64_t *count);

/* sivf_stats -- forces a sync; fills `out` [host]. */
sivf_status sivf_stats(sivf_index *index, void *stream, sivf_stats_t *out);

/*
 * sivf_dump -- copy the bookkeeping state to host arrays for invariant
 * checks (forces a sync).  Any pointer may be NULL to skip that array.
 *   list_nslabs [host] int32[nlist]; list_head [host] int32[nlist];
 *   list_dir [host] int32[nlist * dir_cap] (row l holds list l's slabs in
 *     chain order, oldest first);
 *   slab_meta [host] int32[n_slabs * 3]: {list, fill, live} per slab;
 *   slab_bits [host] uint32[n_slabs * slab_size / 32]: validity bitmaps;
 *   slab_ids [host] int64[n_slabs * slab_size];
 *   att [host] int64[n_max]: (slab << 32) | slot, or -1;
 *   free_stack [host] int32[n_slabs], *n_free [host].
 */
sivf_status sivf_dump(sivf_index *index, void *stream, int32_t *list_nslabs,
                      int32_t *list_head, int32_t *list_dir, int32_t *slab_meta,
                      uint32_t *slab_bits, int64_t *slab_ids, int64_t *att,
                      int32_t *free_stack, int64_t *n_free);

/*
 * sivf_dump_payload -- copy slab payload rows to host (forces a sync):
 * the FP32 rows [n_slabs * slab_size, d] (x32, optional), the BF16 copy as
 * uint16 (xb16, optional), the FP8 copy as uint8 (x8, optional) and the
 * per-list FP8 inverse scales float32[nlist] (inv_scale, optional).
 */
sivf_status sivf_dump_payload(sivf_index *index, void *stream, float *x32,
                              uint16_t *xb16, uint8_t *x8, float *inv_scale);

/*
 * sivf_list_sizes -- live vectors of every list (forces a sync):
 * sizes [host] int32[nlist].
 */
sivf_status sivf_list_sizes(sivf_index *index, void *stream, int32_t *sizes);

/*
 * sivf_set_wait_limit -- the time after which a device wait inside the list
 * scan (a TMA copy, an MMA, a stage hand-over between the roles of a CTA)
 * gives up: it records a sticky timeout bit, stops every role of the scan
 * (copies already in flight are drained first) and the next synchronising
 * call returns SIVF_E_TIMEOUT, after which the index refuses work.  ns = 0
 * restores the default, 2 s (far above any healthy wait, a slow scan of a
 * long list included).  The paper has no counterpart: it names a traversal
 * bound and fail-fast errors (Sec. 3.2, Sec. 3.3) but no timing.
 */
sivf_status sivf_set_wait_limit(sivf_index *index, int64_t ns);

/*
 * sivf_debug_set_error_bits -- test hook: ORs `bits` into the index's sticky
 * device error word (forces a sync), as a device-side bound or timeout
 * would, so the failure paths can be exercised without a device fault.
 * bits: 1 a bad slab reference, 2 a directory past its capacity, 4 the free
 * stack, 8 a timeout, 16 the coarse selection, 32 a search plan.
 */
sivf_status sivf_debug_set_error_bits(sivf_index *index, uint32_t bits, void *stream);

/*
 * sivf_set_chunk_bytes -- the scratch budget of one query chunk of a search:
 * a batch whose scratch (per-pair candidate runs, coarse rows, plans) would
 * exceed it is searched in chunks of as many queries as fit (at least 256),
 * each chunk streaming the lists its queries probe.  bytes = 0 restores the
 * default, 6 GiB; a smaller budget trades list re-reads for device memory.
 * Results do not depend on the chunking.  Returns SIVF_E_ARG for bytes < 0.
 * The paper has no counterpart (its batches fit its scratch).
 */
sivf_status sivf_set_chunk_bytes(sivf_index *index, int64_t bytes);

/*
 * sivf_profile -- tracing.  enable != 0 starts recording a CUDA event pair
 * on the launching stream around every kernel group the index enqueues
 * (forces a device sync and clears earlier records); enable == 0 stops.
 * Not for use while a stream is being captured into a graph.
 */
sivf_status sivf_profile(sivf_index *index, int enable);

/*
 * sivf_profile_read -- forces a device sync.  For `kernel` one of "coarse"
 * (approximate-distance GEMM + exact selection), "insert", "remove",
 * "group" (pairs grouped by list), "scan" (the list scan), "merge" (per-query
 * top-k): *launches = kernels launched in that group while recording and
 * *total_ms = the summed event time.  For "all": *launches = every kernel
 * the index has launched since creation, *total_ms = 0.
 */
sivf_status sivf_profile_read(sivf_index *index, const char *kernel,
                              int64_t *launches, double *total_ms);

/* ------------------------------------------------------------------------
 * Scan tiles and the autotuner.  The list scan's work split is chosen per
 * batch from a small table held by the index; a bucket of the table covers
 * one scan dtype, one power-of-two range of (query, list) pairs per list
 * (nq * nprobe / nlist, from 2^-8 to 2^15) and one range of kept
 * candidates per (query, list) (k for SIVF_FP32, 4k for the reduced
 * dtypes: <= 16, <= 64, <= 256, larger).  Buckets nobody set use built-in
 * defaults.  The paper has no counterpart: its scan has one fixed shape.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t queries_per_tile; /* SIVF_FP32: 8, 16, 32 or 64 queries share
                                 each slab load.  Reduced dtypes: 64 = the
                                 vector-row scan (slab rows on the MMA's M,
                                 up to 48 queries as N; the default), 128 =
                                 the query-row scan (up to 128 (query,
                                 probe) pairs of a list on the tensor-memory
                                 lanes, slab rows as N; only where its
                                 candidate buffers fit)                    */
    int32_t slabs_per_chunk;  /* 1..16: a list is split into slab chunks
                                 of at least this many slabs              */
    int32_t items_per_sm;     /* 1..16: a list is split into chunks so that
                                 no work item exceeds 1 / (items_per_sm x
                                 152) of the scan's work (query tiles x
                                 slabs over the probed lists): a heavy list
                                 of a skewed index spreads over many SMs  */
    int32_t select_slabs;     /* SIVF_FP32, 0..8: the k-select buffer of
                                 each query row holds its best k plus room
                                 for this many slabs of candidates (0: the
                                 built-in width, two slabs while that stays
                                 within 256 entries).  Reduced dtypes,
                                 vector-row scan, 0..3: room for this many
                                 128-row tiles of candidates beside the
                                 held 4k (0: two where shared memory keeps
                                 three load stages, else one); query-row
                                 scan, 0..3: the longest candidate buffer
                                 of one row (0, 1: 255, 2: 1023, 3: 2047)  */
    int32_t nearest_first;    /* reduced dtypes, queries probing several
                                 lists: 0 = one launch over every probe;
                                 1 = each query's nearest list in a launch
                                 of its own first, so the other lists meet
                                 a tight bound (the query-row scan reads 1
                                 as 2); 2 = a seed launch over the first
                                 128 rows of each query's nearest list
                                 publishes a bound per query, then one
                                 launch streams every probed list once     */
} sivf_tile;

/*
 * sivf_set_tile -- install `tile` [host] for the bucket that a search of
 * nq queries, k results and nprobe lists with `dtype` falls in; NULL
 * clears the bucket (back to the defaults).  A tile whose buffers would not
 * fit in shared memory for that batch is rejected with SIVF_E_ARG.
 * sivf_get_tile stores in *out the tile a search of that shape would use
 * now (the installed one or the default).
 */
sivf_status sivf_set_tile(sivf_index *index, sivf_scan_dtype dtype, int64_t nq,
                          int k, int nprobe, const sivf_tile *tile);
sivf_status sivf_get_tile(sivf_index *index, sivf_scan_dtype dtype, int64_t nq,
                          int k, int nprobe, sivf_tile *out);

/*
 * sivf_autotune -- time sivf_search on the queries q [device] float32[nq, d]
 * for a set of tiles (coordinate descent over the fields of sivf_tile,
 * starting from the current tile), `reps` timed searches per tile after one
 * warm-up, CUDA events on `stream`; install the fastest for the batch's
 * bucket.  *best [host] receives it and *best_ms (optional) its mean time
 * per search.  Forces syncs; allocates and frees its own output buffers.
 * Results of the searches it runs are discarded; the index is not changed.
 */
sivf_status sivf_autotune(sivf_index *index, const float *q, int64_t nq, int k,
                          int nprobe, sivf_scan_dtype dtype, int reps,
                          void *stream, sivf_tile *best, double *best_ms);

/* ------------------------------------------------------------------------
 * Mixed-batch executor.  A queue of uneven add, remove and search batches
 * (each search with its own k, nprobe and dtype) is recorded once into a
 * CUDA graph and then replayed with one graph launch per queue.  Every
 * batch reads its inputs from, and writes its outputs to, the device
 * addresses given when the queue was recorded, so a caller refills those
 * buffers in place between launches.  The batches run in queue order with
 * the semantics of the single calls (sivf_add, sivf_remove, sivf_search,
 * sivf_compact: a queue can carry compaction passes between its batches),
 * and the executor records, per batch, its status, its count and a device
 * timestamp.  The paper runs each batch as separate launches; this has no
 * counterpart there.
 * ---------------------------------------------------------------------- */
typedef enum {
    SIVF_OP_ADD = 0,
    SIVF_OP_REMOVE = 1,
    SIVF_OP_SEARCH = 2,
    SIVF_OP_COMPACT = 3  /* executor only: one sivf_compact pass, k = min_free,
                            n = max_moves; the result's count = members moved */
} sivf_op_kind;

typedef struct {
    int32_t kind;        /* sivf_op_kind                                     */
    int32_t dtype;       /* search: sivf_scan_dtype                          */
    int32_t k;           /* search: results per query; compact: min_free     */
    int32_t nprobe;      /* search: lists probed per query                   */
    int64_t n;           /* ids (add, remove), queries (search) or the
                            member budget (compact), >= 1                    */
    const int64_t *ids;  /* add, remove [device] int64[n]                    */
    const float *x;      /* add: vectors, search: queries [device] [n, d]    */
    float *dist;         /* search [device] float32[n, k]                    */
    int64_t *labels;     /* search [device] int64[n, k]                      */
} sivf_op;

typedef struct {
    int32_t status;      /* sivf_status of the batch (add: admission and id
                            checks; remove: id checks; search: SIVF_OK)     */
    int32_t pad;
    int64_t count;       /* ids added / removed; queries answered           */
    double device_ms;    /* device time from the end of the previous batch
                            (or the start of the queue) to its end         */
} sivf_op_result;

typedef struct sivf_exec sivf_exec;

/*
 * sivf_exec_create -- check the `nops` batches of `ops` [host] (every
 * argument rule of the single calls), reserve all the scratch they need
 * (owned by the executor: it never shares scratch with the index's own
 * calls), and record them into a CUDA graph.  The ops are copied; the
 * device buffers they point to must stay valid while the executor lives.
 * Recording enqueues nothing: the queue runs only at sivf_exec_launch.
 * Errors: SIVF_E_ARG with the index's last error naming the bad batch.
 */
sivf_status sivf_exec_create(sivf_index *index, const sivf_op *ops, int nops,
                             sivf_exec **out);

/*
 * sivf_exec_launch -- run the whole queue with one graph launch on
 * `stream`.  Launches of one executor must not overlap each other or other
 * work on the same index (order them on one stream).
 */
sivf_status sivf_exec_launch(sivf_exec *exec, void *stream);

/*
 * sivf_exec_results -- per-batch results of the last launch (forces a
 * sync): results [host] sivf_op_result[nops].  Returns SIVF_E_CORRUPT or
 * SIVF_E_TIMEOUT when the device error word is set, else SIVF_OK (the
 * batches' own statuses are in the array).
 */
sivf_status sivf_exec_results(sivf_exec *exec, void *stream, sivf_op_result *results);

/* sivf_exec_kernels -- kernel launches one sivf_exec_launch performs. */
int64_t sivf_exec_kernels(const sivf_exec *exec);

/* sivf_exec_destroy -- synchronize and free the graph and its scratch. */
sivf_status sivf_exec_destroy(sivf_exec *exec);

/* ------------------------------------------------------------------------
 * Serving loop.  A server owns the index while it lives and drives it from
 * one worker thread; callers on any thread submit requests (inserts,
 * deletes, queries) from host memory and wait for them.  The worker serves
 * the request queue in arrival order, coalescing each run of same-kind
 * requests at the head into one batch (continuous batching: whatever
 * arrived while earlier batches were on the GPU joins the next batch), and
 * keeps up to `depth` batches in flight, each in its own slot (stream,
 * pinned staging, device buffers, scratch).  Host-to-device copies, kernels
 * and result copies of different slots overlap; query batches run
 * concurrently with each other, and a mutation batch waits, on the device,
 * for every batch launched before it (and every batch after it waits for
 * it), so each request sees exactly the mutations served before it.
 * Admission by free slabs: inserts are coalesced only while the batch's
 * worst-case slab demand (ceil(n / C) plus one slab per touched list) fits
 * the free slabs known on the host net of in-flight inserts; otherwise the
 * worker waits for in-flight mutations, then serves the request alone and
 * the device's exact all-or-nothing admission decides (SIVF_E_NOMEM).
 * The paper has no serving loop; this follows the mixed
 * insert/search/delete stream of its evaluation.
 * ---------------------------------------------------------------------- */
typedef struct sivf_server sivf_server;

typedef struct {
    int32_t k;                /* results per query                           */
    int32_t nprobe;           /* lists probed per query                      */
    int32_t dtype;            /* sivf_scan_dtype of every search             */
    int32_t depth;            /* batches in flight, 1..8                     */
    int32_t max_query_batch;  /* queries per search launch, >= 1             */
    int32_t max_insert_batch; /* vectors per add launch, >= 1                */
    int32_t max_delete_batch; /* ids per remove launch (evictions included)  */
    int32_t compact_min_free; /* > 0: whenever the worker is idle, one
                                 compaction pass (sivf_compact, at most
                                 max_insert_batch members) over lists that
                                 would free at least this many slabs,
                                 repeated until a pass moves nothing, then
                                 again after the next mutation batch (the
                                 first passes run at start); 0: off        */
} sivf_server_config;

typedef struct {
    int32_t kind;             /* SIVF_OP_ADD / SIVF_OP_REMOVE / SIVF_OP_SEARCH */
    int32_t status;           /* status of the batch that served it          */
    int64_t count;            /* vectors / ids / queries it carried (0 when
                                 its batch was rejected)                     */
    int64_t batch;            /* serving order: sequence number of its batch */
    double latency_ms;        /* arrival -> completion seen by the worker    */
    double queue_ms;          /* arrival -> launch of its batch              */
} sivf_request_info;

typedef struct {
    int64_t requests[3];      /* completed requests per kind (SIVF_OP_*)     */
    int64_t batches[3];       /* batches per kind                            */
    int64_t items[3];         /* vectors / ids / queries per kind            */
    int64_t deferred;         /* times an insert waited for free slabs       */
    int64_t rejected;         /* requests whose batch was rejected           */
    int64_t max_in_flight;    /* most batches seen in flight at once         */
    int64_t compact_passes;   /* idle compaction passes that moved members   */
    int64_t compact_freed;    /* slabs they returned to the pool             */
    int64_t compact_moved;    /* members they rewrote                        */
} sivf_server_stats_t;

/*
 * sivf_server_create -- start a server on `index` (which must have its
 * centroids).  Reserves every slot's buffers and scratch, then starts the
 * worker.  While the server lives, no other call may use the index.
 */
sivf_status sivf_server_create(sivf_index *index, const sivf_server_config *cfg,
                               sivf_server **out);

/* sivf_server_now_ns -- the steady clock (ns) that arrival times use. */
int64_t sivf_server_now_ns(void);

/*
 * sivf_server_submit -- queue one request; *req receives its id (ids count
 * up from 0).  kind SIVF_OP_ADD: ids [host] int64[n], x [host] float32[n,d],
 * and optionally evict [host] int64[n_evict] removed just before the insert
 * (a sliding window's overflow), within the same batch; SIVF_OP_REMOVE:
 * ids [host] int64[n]; SIVF_OP_SEARCH: x [host] float32[n, d] queries,
 * dist [host] float32[n, k] and labels [host] int64[n, k] receive the
 * results.  The host arrays must stay valid until the request completes.
 * n must fit the kind's batch limit.  arrival_ns: when the request arrived,
 * on sivf_server_now_ns's clock (0 = now); latency is measured from it.
 */
sivf_status sivf_server_submit(sivf_server *server, int kind, int64_t n, const int64_t *ids,
                               const float *x, int64_t n_evict, const int64_t *evict,
                               float *dist, int64_t *labels, int64_t arrival_ns,
                               int64_t *req);

/*
 * sivf_server_wait -- wait up to timeout_us (< 0: forever) for request
 * `req`; on completion fills *info (optional) and returns SIVF_OK, else
 * SIVF_E_TIMEOUT.  A sticky device error is returned as SIVF_E_CORRUPT /
 * SIVF_E_TIMEOUT once the worker has seen it.
 */
sivf_status sivf_server_wait(sivf_server *server, int64_t req, int64_t timeout_us,
                             sivf_request_info *info);

/* sivf_server_drain -- wait (up to timeout_us, < 0 forever) until every
 * request submitted so far has completed. */
sivf_status sivf_server_drain(sivf_server *server, int64_t timeout_us);

/* sivf_server_stats -- counters since the server started. */
sivf_status sivf_server_stats(sivf_server *server, sivf_server_stats_t *out);

/* sivf_server_destroy -- serve what is queued, stop the worker, free the
 * slots.  The index is usable by other calls again afterwards. */
sivf_status sivf_server_destroy(sivf_server *server);

/* sivf_last_error -- text of the last error on this index (never NULL). */
const char *sivf_last_error(const sivf_index *index);

/* sivf_version -- library version string. */
const char *sivf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SIVF_H */
