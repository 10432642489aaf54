// Internal declarations of libsivf: the device-resident index state, the
// control block that carries batch status between kernels of one call, and
// small device helpers (bulk copies into shared memory, mbarrier waits with
// an iteration limit, warp utilities).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sivf.h"

namespace sivf {

constexpr int kMaxD = 256;          // largest supported dimension
constexpr int kMaxK = 1024;         // largest k of one search
constexpr int kRankTile = 1024;     // vectors per block of the stable ranking
constexpr int kMaxChunks = 64;      // most slab chunks one list is split into
constexpr size_t kMaxStageBytes = 160 * 1024;  // two slab stages in shared memory
// default time a device wait may take before it gives up: far above any
// healthy wait (a slow scan of a long list included)
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

// sticky device error bits (index->err)
enum : uint32_t {
    ERR_BAD_SLAB = 1u,   // a directory entry or address-table entry points
                         // outside the pool or at a slab of another list
    ERR_DIR_BOUND = 2u,  // a list directory longer than its capacity
    ERR_STACK = 4u,      // free stack under- or overflow
    ERR_TIMEOUT = 8u,    // an mbarrier wait ran out of iterations
    ERR_SELECT = 16u,    // coarse selection could not place a row
    ERR_PLAN = 32u,      // a search plan outgrew the scratch sized for it
};

// batch flags (Ctl::flags)
enum : int32_t {
    FLAG_BAD_ID = 1,     // an id outside [0, n_max)
    FLAG_DIR_FULL = 2,   // a list would exceed its directory capacity
};

// Per-call control block in device memory, zeroed at the start of every
// add / remove / search.
struct Ctl {
    int32_t status;      // sivf_status of the current batch
    int32_t flags;       // FLAG_*
    int64_t count;       // vectors added or removed
    int64_t demand;      // slabs the batch needs (admission)
    int32_t ntouched;    // lists receiving vectors
    int32_t naffected;   // lists that lost a slab
    int32_t nitems;      // search work items
    int32_t next_item;   // search work-queue cursor
    int32_t nscan;       // (query, list) pairs in the search
    int32_t nruns;       // search output runs reserved so far
    int32_t pad[6];
};

struct SlabMeta {        // 16 bytes per slab
    int32_t list;        // owning list, -1 when on the free stack
    int32_t fill;        // slots written since the slab was taken
    int32_t live;        // validity bits set
    int32_t pad;
};

struct PlanEntry {       // per list touched by an insert batch
    int32_t head_old;    // head slab before the batch (-1: none)
    int32_t fill_old;    // its fill
    int32_t into_head;   // vectors that go into the old head
    int32_t dir_pos0;    // directory position of the first new slab
};

// Kernel groups timed by the profiler (sivf_profile / sivf_profile_read).
enum ProfKind { PROF_COARSE = 0, PROF_INSERT, PROF_REMOVE, PROF_GROUP, PROF_SCAN,
                PROF_MERGE, PROF_RERANK, PROF_COMPACT, PROF_NKIND };

struct ProfEvent {
    int kind;
    int launches;
    cudaEvent_t start, stop;
};

// Installed scan tiles (sivf_set_tile / sivf_autotune): one per scan dtype,
// log2 bucket of (query, list) pairs per list and bucket of kept candidates.
constexpr int kTuneB = 24;           // pairs per list 2^-8 .. 2^15
constexpr int kTuneK = 4;            // kept candidates <= 16, 64, 256, more
struct TileChoice {
    int set;
    sivf_tile t;
};

}  // namespace sivf

// The index handle.  Every array is device memory unless noted.
struct sivf_index {
    // configuration
    int d, nlist, C, W;            // W = C / 32 bitmap words per slab
    int64_t n_max, n_slabs, dir_cap;
    uint32_t dtypes;
    int device;
    bool have_centroids;
    int64_t ntotal_hint;           // host estimate, refreshed on sync

    // coarse quantizer
    float *cent;                   // [nlist, d]
    float *cnorm;                  // [nlist] fl32(||c||^2), from an FP64 sum
    float *cnrm_up;                // [nlist] upper bound of ||c||
    uint16_t *cent_bf16;           // [nlist, d] bf16(c) (tensor-core coarse stage)
    uint16_t *cent_lo;             // [nlist, d] bf16(c - bf16(c)) (split stage)

    // slab pool (Sec. 3.1)
    float *x32;                    // [S, C, d] FP32 payload
    __nv_bfloat16 *xb16;           // [S, C, d] BF16 copy or null
    uint8_t *x8;                   // [S, C, d] FP8 E4M3 copy or null
    float *xnorm;                  // [S, C] fl32(||x||^2)
    float *rnorm;                  // [S, C] fl32(||x - c_l||^2) (FP8 residual copy) or null
    int64_t *ids;                  // [S, C] label of each slot
    uint32_t *bits;                // [S, W] validity bitmaps
    sivf::SlabMeta *meta;          // [S]
    int32_t *free_list;            // [S] free stack
    int32_t *free_top;             // [1] number of free slabs

    // lists
    int32_t *head;                 // [nlist] open (head) slab or -1
    int32_t *nslabs;               // [nlist] directory length
    int32_t *list_live;            // [nlist] live vectors per list
    int32_t *dir;                  // [nlist, dir_cap] slabs of each list
    float *inv_scale8;             // [nlist] FP8 inverse scale
    // TMA descriptors (CUtensorMap, 128 bytes) of the BF16 / FP8 copies
    alignas(64) unsigned char tmap_bf16[128];
    alignas(64) unsigned char tmap_fp8[128];
    // the same copies with boxes of 128 rows (a tile of consecutive slabs,
    // slabs of fewer than 128 rows only; tmap_tile_ok when made)
    alignas(64) unsigned char tmap_bf16_t[128];
    alignas(64) unsigned char tmap_fp8_t[128];
    bool tmap_tile_ok;
    // the same copies with boxes of min(C, 64) rows (query-row scan)
    alignas(64) unsigned char tmap_qt_bf16[128];
    alignas(64) unsigned char tmap_qt_fp8[128];
    // the BF16 centroids in boxes of 64 x 256 (fused coarse first stage)
    alignas(64) unsigned char tmap_cent[128];
    bool tmap_cent_ok;
    // nearest-list assignment takes the split-BF16 first stage (the single
    // BF16 product's bound is wide against the centroid spacing)
    bool assign_split;
    bool tmaps_ready;

    // address translation table (Sec. 3.4)
    int64_t *att;                  // [n_max] (slab << 32) | slot, or -1

    // batch bookkeeping kept zeroed / at -1 between calls
    int32_t *claim;                // [n_max] -1, last batch index of an id
    int32_t *list_flag;            // [nlist] 0, touched index + 1
    int32_t *aff_flag;             // [nlist] 0, 1 while in `affected`
    int32_t *runcnt;               // [nlist, nblk_max] 0
    int nblk_max;                  // rank blocks the runcnt rows hold

    sivf::Ctl *ctl;                // control block of the current call's stream
    uint32_t *err;                 // sticky error bits
    uint64_t wait_ns;              // time after which a list-scan wait gives up
    int64_t chunk_bytes;           // query-chunk scratch budget (0: the default)
    int64_t *stat;                 // [4] persistent counters: [0] live vectors,
                                   // [1] (query, vector) pairs scanned,
                                   // [2] slab bytes streamed by list scans
    void *extra;                   // host-side bookkeeping (abi.cu)

    // scratch arena (grown on demand, reset per call)
    char *scratch;
    size_t scratch_bytes;

    // scan tiles chosen per batch bucket (zero = defaults)
    sivf::TileChoice tune[3][sivf::kTuneB][sivf::kTuneK];
    bool capturing;                // a sivf_exec is recording: no profiler events

    // tracing: CUDA events around kernel groups, launch counts
    bool prof_on;
    std::vector<sivf::ProfEvent> prof;
    int64_t launches;              // kernels launched since creation

    std::string last_error;
};

namespace sivf {
// Record the start of a group of `n` kernel launches of kind `k` on `st`;
// returns a token for prof_end (or -1 when profiling is off).
int prof_begin(sivf_index *ix, int k, int n, cudaStream_t st);
void prof_end(sivf_index *ix, int tok, cudaStream_t st);
}  // namespace sivf
