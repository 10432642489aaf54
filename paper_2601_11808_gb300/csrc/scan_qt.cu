// Reduced-precision list scan with the queries on the tensor-memory lanes
// (the precision pattern of the hot path; the paper's Algorithm 3 scans
// FP32 payloads only).  Each probed list is streamed from HBM once per
// search: one launch over all (query, probe) pairs, after a short seed
// launch when queries probe more than one list.
//
// One persistent CTA per SM takes work items (list, tile of up to 128
// (query, probe) pairs of that list, slab chunk).  The tile's query rows,
// rounded to the scan format, are the A operand (M = 128 rows, staged once
// per item); the list's slab rows stream through shared memory as the B
// operand (TMA 2-D loads with the 128-byte swizzle, NV = 128 / KC rows, 16
// KB per stage); tcgen05.mma accumulates the 128 x NV dot products in FP32
// into one of four tensor-memory buffers.
//
// An epilogue thread owns one query row; item row i sits on tensor-memory
// lane (i % 4) * 32 + i / 4, so a thin item's rows spread over the four
// epilogue warps.  A thread reads its row of NV dot products 32 columns at a
// time (tcgen05.ld), forms ||x||^2 - 2 s q.x for each column (s the
// dequantisation scale; ||x||^2 of the unrounded vector) and compares it
// with the row's bound: the K'-th smallest distance the query has so far,
// minus ||q||^2, plus a few ulps so that rounding never drops a candidate
// that belongs to the best K'.  The 32 validity bits of the columns mask the
// result, so deleted slots, slots past a slab's fill and rows of missing
// slabs never pass.  Passing columns are written into the row's own
// candidate buffer in shared memory as (distance, slot): all 32 at once when
// all pass, else one by one through a per-warp staging area.  The item's
// rows share the buffer pool, so the fewer rows an item has the longer each
// buffer (a list probed by a few queries keeps every distance without any
// reduction).  A row whose buffer fills is reduced to its best K' by its
// warp (a bisection on order-preserving keys held in registers for short
// buffers, a radix select through shared memory for long ones; ties go to
// the lower slot), which also lowers the row's bound.  No barrier spans the
// CTA per tile: the four epilogue warps (one per tensor-memory lane quarter)
// run independently, up to four accumulators apart.
//
// Bounds: a row starts from its query's shared bound (the smallest K'-th
// distance any item has published), re-reads it every tile, and publishes
// its own after every reduction and at the end of the item.  When queries
// probe several lists, a seed launch first scans the first 128 rows of each
// query's nearest list and publishes the bound only; the main launch then
// meets a bound in every other list from its first tile.  Each item writes
// its rows' best K' unsorted into the row's output run; a per-query merge
// selects and sorts the best K' of all of them.
//
// Roles: warp 0 (one lane) TMA loads of the B tiles and bulk copies of the
// rows' ||x||^2 with L2 prefetches ahead; warp 1 (one lane) issues the MMAs;
// warp 2 stages the item contexts (pairs, norms, scales, bounds, slab ids,
// bitmaps) one item ahead and owns the tensor memory; warp 3 builds the
// query tiles (two buffers); warps 4-7 are the epilogue.  Every wait is
// bounded, and a wait that gives up stops every role.
#include <cudaTypedefs.h>
#include <math.h>

#include "device_utils.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace sivf {

constexpr int QT_M = 128;       // query rows per item (MMA M, tensor-memory lanes)
constexpr int QT_NB = 4;        // accumulator buffers
constexpr int QT_BCOL = 128;    // tensor-memory columns per buffer (NV <= 128)
constexpr int QT_XR = 8;        // entries of the ||x||^2 ring (one per B tile)
constexpr int QT_META = 256;    // slabs of one sub-item (ids and bitmaps staged together)
constexpr int QT_CTX = 2;       // item contexts in flight
constexpr int QT_NT = 256;      // threads: 4 role warps + 4 epilogue warps
constexpr int QT_MAXST = 4;     // most B stages
constexpr int QT_MAXEK = 8;     // register bisection for buffers up to 32 * 8 entries
constexpr int QT_MECAP = 2047;  // longest buffer of one row
constexpr int QT_HIST = 256;    // radix-select bins per epilogue warp
constexpr float QT_NOBOUND = 1e38f;  // a row bound at or above this: no bound yet
constexpr int QT_PF_BYTES = 192 * 1024;  // L2 prefetch distance per CTA

enum : int { QF_FIRST = 1, QF_LAST = 2, QF_STOP = 4 };

struct QtArgs {
    int64_t nq;
    int P, K, ME;               // K' kept per row, ME entries of a row's buffer
    const int32_t *qlist, *loff, *lcnt, *nch;
    const int32_t *prun;        // first output run of each pair (-1: not scanned)
    const int2 *items;
    const float *qn, *qsc;      // per query (BF16) or per pair (FP8)
    const unsigned char *qcast; // rounded query rows (BF16) or pair residual codes (FP8)
    int per_pair;
    float *part_d;
    int64_t *part_i;            // global slot (slab * C + slot) of each candidate
    int32_t *part_n;            // candidates in each run
    float *thr;                 // per query: smallest published K'-th distance
    const float *xnorm;
    const uint32_t *bits;
    const int32_t *nslabs, *dir;
    const float *inv_scale8;
    const unsigned char *pay;   // the scanned copy (BF16 or E4M3 rows)
    int64_t n_slabs, dir_cap;
    int d, C, KC, NV, nst;
    int seed_slabs;             // > 0: seed launch over the first slabs of each item
    int mecap;                  // longest candidate buffer of one row (odd)
    uint64_t wait_ns;           // time after which a wait of the scan gives up
    int pf_tiles;               // B tiles prefetched into L2 ahead of the loads
    Ctl *ctl;
    uint32_t *err;
};

// One item context: header, per item row (pair, norm, scale, bound, query
// row, output run), per slab of the sub-item (slab id, four bitmap words).
//   hdr: list, m, first slab, slabs, tiles, -, -, chunk, flags, inv scale
__host__ __device__ constexpr size_t qt_ctx_bytes()
{
    return 64 + (size_t)24 * QT_M + (size_t)4 * QT_META + (size_t)16 * QT_META;
}

struct QtSmem {
    size_t a, b, xn, bd, bs, scr, hist, ctx, bars, total;
};
// ME: buffer entries per row when all 128 rows are used (the pool holds
// 128 * ME entries)
__host__ __device__ inline QtSmem qt_smem(int KC, int nst, int ME)
{
    QtSmem s;
    s.a = 0;                                              // 2 x KC x 16 KB query tiles
    s.b = s.a + (size_t)QT_CTX * KC * QT_M * 128;         // nst x 16 KB B stages
    s.xn = s.b + (size_t)nst * 16384;
    s.bd = s.xn + (size_t)QT_XR * QT_BCOL * 4;
    s.bs = s.bd + (size_t)QT_M * ME * 4;
    s.scr = s.bs + (size_t)QT_M * ME * 4;                 // 4 warps x 32 x 32 staged values
    s.hist = s.scr + (size_t)4 * 32 * 32 * 4;
    s.ctx = s.hist + (size_t)4 * QT_HIST * 4;
    s.bars = s.ctx + (size_t)QT_CTX * qt_ctx_bytes();
    s.total = s.bars + 64 * 8 + 1024;                     // + base alignment slack
    return s;
}

// prune threshold of a row in the units the epilogue compares
// (||x||^2 - 2 s q.x against kd - ||q||^2), raised by a few ulps of the
// terms so that rounding never drops a candidate at or below kd
__device__ __forceinline__ float qt_bound(float kd, float qn)
{
    return kd - qn + (fabsf(kd) + fabsf(qn)) * 9.5367431640625e-7f;  // 2^-20
}

// Keep the K smallest (distance, slot) of the row's n > K entries bd/bs[0,
// n), unsorted, in bd/bs[0, K); returns the K-th smallest distance.  The
// keys (order-preserving 32-bit images of the distances) and slots are held
// in registers: the K-th key is found by bisection on its value with
// ballot counts, stopping early at any value with exactly K keys at or
// below it; distance ties at the K-th place keep the lowest slots.
template <int EK>
__device__ float qt_fold(float *bd, int32_t *bs, int n, int K, int lane)
{
    uint32_t key[EK];
    int32_t slt[EK];
#pragma unroll
    for (int e = 0; e < EK; ++e) {
        const int i = lane + 32 * e;
        key[e] = i < n ? fkey(bd[i]) : 0xffffffffu;
        slt[e] = i < n ? bs[i] : 0x7fffffff;
    }
    uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
    for (int e = 0; e < EK; ++e)
        if (key[e] != 0xffffffffu) {
            kmin = min(kmin, key[e]);
            kmax = max(kmax, key[e]);
        }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    uint32_t lo = kmin, hi = kmax;
    bool exact = false;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        uint32_t c = 0;
#pragma unroll
        for (int e = 0; e < EK; ++e) c += __popc(__ballot_sync(0xffffffffu, key[e] <= mid));
        if (c == (uint32_t)K) {
            lo = mid;
            exact = true;
            break;
        }
        if (c > (uint32_t)K) hi = mid;
        else lo = mid + 1;
    }
    if (exact) {  // every key <= lo is kept; the K-th is their maximum
        uint32_t kk = 0u;
#pragma unroll
        for (int e = 0; e < EK; ++e)
            if (key[e] <= lo) kk = max(kk, key[e]);
        lo = __reduce_max_sync(0xffffffffu, kk);
    }
    const uint32_t kth = lo;
    uint32_t clt = 0, ceq = 0;
#pragma unroll
    for (int e = 0; e < EK; ++e) {
        clt += key[e] < kth;
        ceq += key[e] == kth;
    }
    clt = __reduce_add_sync(0xffffffffu, clt);
    ceq = __reduce_add_sync(0xffffffffu, ceq);
    const uint32_t need = (uint32_t)K - clt;  // 1 <= need <= ceq
    int32_t cut = 0x7fffffff;                 // tied entries kept: slot <= cut
    if (ceq > need) {
        int32_t slo = 0, shi = 0x7fffffff;
        while (slo < shi) {
            const int32_t mid = slo + ((shi - slo) >> 1);
            uint32_t c = 0;
#pragma unroll
            for (int e = 0; e < EK; ++e)
                c += __popc(__ballot_sync(0xffffffffu, key[e] == kth && slt[e] <= mid));
            if (c >= need) shi = mid;
            else slo = mid + 1;
        }
        cut = slo;
    }
    __syncwarp();  // every lane holds its entries before any is overwritten
    int w = 0;
#pragma unroll
    for (int e = 0; e < EK; ++e) {
        const bool take = key[e] < kth || (key[e] == kth && slt[e] <= cut);
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        if (take) {
            const int p = w + __popc(mk & lanemask_lt());
            bd[p] = fkey_inv(key[e]);
            bs[p] = slt[e];
        }
        w += __popc(mk);
    }
    __syncwarp();
    return fkey_inv(kth);
}

// Long buffers: the same selection by a radix select over the 64-bit keys
// (distance key, slot), 8 bits per pass from the highest bit where the keys
// differ, each pass a histogram of the keys still in play (one warp, bins in
// shared memory), stopping at the first pass whose chosen bin is taken whole;
// then a stable in-place compaction of the K kept entries.
__device__ float qt_radix_keep(float *bd, int32_t *bs, int n, int K, uint32_t *hist, int lane)
{
    auto key = [&](int i) -> uint64_t {
        return ((uint64_t)fkey(bd[i]) << 32) | (uint32_t)bs[i];
    };
    uint64_t kmin = ~0ull, kmax = 0ull;
    for (int i = lane; i < n; i += 32) {
        const uint64_t k = key(i);
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmin, o));
        kmax = max(kmax, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmax, o));
    }
    const uint64_t diff = kmin ^ kmax;
    const int top = diff ? 63 - __clzll((long long)diff) : 0;
    uint64_t mask = top >= 63 ? 0ull : ~((2ull << top) - 1ull);
    uint64_t prefix = kmin & mask;
    uint32_t need = (uint32_t)K;
    for (int hi = top; hi >= 0; hi -= 8) {
        const int shift = max(hi - 7, 0);
        const uint32_t bmask = (1u << (hi - shift + 1)) - 1u;
#pragma unroll
        for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0u;
        __syncwarp();
        for (int i0 = 0; i0 < n; i0 += 32) {  // one add per distinct bin per round
            const int i = i0 + lane;
            uint32_t bin = 0xffffffffu;
            if (i < n) {
                const uint64_t k = key(i);
                if ((k & mask) == prefix) bin = (uint32_t)(k >> shift) & bmask;
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, bin);
            if (bin != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
        }
        __syncwarp();
        uint32_t loc[8], sum = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            loc[b] = hist[lane * 8 + b];
            sum += loc[b];
        }
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t excl = incl - sum;
        const bool mine = excl < need && incl >= need;
        uint32_t bin = 0, below = 0, cnt = 0;
        if (mine) {
            uint32_t cum = excl;
            for (int b = 0; b < 8; ++b) {
                if (cum + loc[b] >= need) {
                    bin = (uint32_t)(lane * 8 + b);
                    below = cum;
                    cnt = loc[b];
                    break;
                }
                cum += loc[b];
            }
        }
        const uint32_t who = __ballot_sync(0xffffffffu, mine);
        const int src = who ? __ffs(who) - 1 : 0;
        bin = __shfl_sync(0xffffffffu, bin, src);
        below = __shfl_sync(0xffffffffu, below, src);
        cnt = __shfl_sync(0xffffffffu, cnt, src);
        prefix |= (uint64_t)bin << shift;
        mask |= (uint64_t)bmask << shift;
        need -= below;
        __syncwarp();
        if (cnt == need) break;
    }
    // keep the keys with (key & mask) <= prefix: exactly the K smallest
    int w = 0;
    float dmax = -INFINITY;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        float dv = 0.f;
        int32_t sv = 0;
        bool take = false;
        if (i < n) {
            dv = bd[i];
            sv = bs[i];
            take = ((((uint64_t)fkey(dv) << 32) | (uint32_t)sv) & mask) <= prefix;
        }
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        __syncwarp();  // this round's entries are read before any is overwritten
        if (take) {
            const int p = w + __popc(mk & lanemask_lt());
            bd[p] = dv;
            bs[p] = sv;
            dmax = fmaxf(dmax, dv);
        }
        w += __popc(mk);
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    return dmax;
}

__device__ __forceinline__ float qt_fold_any(float *bd, int32_t *bs, int n, int K,
                                             uint32_t *hist, int lane)
{
    if (n <= 64) return qt_fold<2>(bd, bs, n, K, lane);
    if (n <= 128) return qt_fold<4>(bd, bs, n, K, lane);
    if (n <= 192) return qt_fold<6>(bd, bs, n, K, lane);
    if (n <= 256) return qt_fold<8>(bd, bs, n, K, lane);
    return qt_radix_keep(bd, bs, n, K, hist, lane);
}

// mbarrier wait bounded in time (the index's wait limit) that also gives
// up as soon as another role of the CTA has stopped (abort flag in shared
// memory); a wait that runs out sets ERR_TIMEOUT and the abort flag
__device__ __forceinline__ bool qt_wait(uint64_t *bar, uint32_t parity, uint32_t *err,
                                        volatile int *abort_flag, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    for (uint32_t it = 1; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && *abort_flag) return false;
        if (gtimer_ns() - t0 > limit_ns) break;
    }
    atomicOr(err, ERR_TIMEOUT);
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void qt_cp_async16(void *dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void qt_cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void qt_prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

template <int DT>  // 0 = BF16, 1 = FP8 E4M3
__global__ __launch_bounds__(QT_NT, 1) void k_scan_qt(const __grid_constant__ CUtensorMap tmap,
                                                       QtArgs a)
{
    pdl_begin();
    constexpr int ESZ = DT == 0 ? 2 : 1;
    constexpr int EPC = 128 / ESZ;  // elements per 128-byte chunk
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int KC = a.KC, NV = a.NV, NST = a.nst, ME = a.ME, K = a.K, C = a.C, d = a.d;
    const QtSmem L = qt_smem(KC, NST, ME);
    unsigned char *A = smem + L.a;
    unsigned char *B = smem + L.b;
    float *XN = reinterpret_cast<float *>(smem + L.xn);
    float *BD = reinterpret_cast<float *>(smem + L.bd);
    int32_t *BS = reinterpret_cast<int32_t *>(smem + L.bs);
    float *SCR = reinterpret_cast<float *>(smem + L.scr);
    uint32_t *HIST = reinterpret_cast<uint32_t *>(smem + L.hist);
    unsigned char *CTX = smem + L.ctx;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *full = bars, *empty = bars + 4, *tfull = bars + 8, *tempty = bars + 12,
             *xfull = bars + 16, *xempty = bars + 24, *cfull = bars + 32, *cempty = bars + 34,
             *afull = bars + 36, *afree = bars + 38;
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(bars + 48);
    volatile int *s_abort = reinterpret_cast<volatile int *>(bars + 49);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t idesc = DT == 0 ? mma_idesc(1, 1, QT_M, NV) : mma_idesc(0, 0, QT_M, NV);
    const int Cb = min(C, 64);  // rows per TMA box
    constexpr size_t CB = qt_ctx_bytes();
    auto hdr = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CB); };
    auto c_qpair = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CB + 64); };
    auto c_qn = [&](int j) { return reinterpret_cast<float *>(CTX + j * CB + 64 + 4 * QT_M); };
    auto c_qsc = [&](int j) { return reinterpret_cast<float *>(CTX + j * CB + 64 + 8 * QT_M); };
    auto c_kd0 = [&](int j) { return reinterpret_cast<float *>(CTX + j * CB + 64 + 12 * QT_M); };
    auto c_qi = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CB + 64 + 16 * QT_M); };
    auto c_run = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CB + 64 + 20 * QT_M); };
    auto c_sl = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CB + 64 + 24 * QT_M); };
    auto c_bits = [&](int j) {
        return reinterpret_cast<uint32_t *>(CTX + j * CB + 64 + 24 * QT_M + 4 * QT_META);
    };

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < QT_NB; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 4);
        }
        for (int i = 0; i < QT_XR; ++i) {
            mbar_init(&xfull[i], 1);
            mbar_init(&xempty[i], 4);
        }
        for (int i = 0; i < QT_CTX; ++i) {
            mbar_init(&cfull[i], 32);
            mbar_init(&cempty[i], 4);
            mbar_init(&afull[i], 32);
            mbar_init(&afree[i], 1);
        }
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == 2) tmem_alloc(tmem_base, QT_NB * QT_BCOL);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_base;

    if (warp == 2) {
        // ---- item contexts
        int sub = 0, nsub = 0, l = 0, m = 0, s0 = 0, ns = 0, chunk = 0, qb = 0;
        float inv_l = 1.f;
        for (int it = 0;; ++it) {
            const int j = it % QT_CTX;
            const uint32_t cu = (uint32_t)(it / QT_CTX);
            bool ok = cu == 0 || qt_wait(&cempty[j], (cu - 1) & 1, a.err, s_abort, a.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            int32_t *h = hdr(j);
            bool stop = false;
            if (sub == nsub) {
                int nx = 0, go = 0;
                if (lane == 0) {
                    nx = atomicAdd(&a.ctl->next_item, 1);
                    go = nx < a.ctl->nitems && !*s_abort;
                }
                nx = __shfl_sync(0xffffffffu, nx, 0);
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    stop = true;
                } else {
                    const int2 itv = a.items[nx];
                    l = itv.x;
                    const int nc_l = a.nch[l];
                    const int tile = itv.y >> 8;
                    chunk = itv.y & 255;
                    const int r0 = tile * QT_M;
                    m = min(QT_M, a.lcnt[l] - r0);
                    int ns_total = a.nslabs[l];
                    if (ns_total > a.dir_cap) {
                        if (lane == 0) atomicOr(a.err, ERR_DIR_BOUND);
                        ns_total = (int)a.dir_cap;
                    }
                    s0 = (int)((int64_t)ns_total * chunk / nc_l);
                    ns = (int)((int64_t)ns_total * (chunk + 1) / nc_l) - s0;
                    if (a.seed_slabs > 0) ns = chunk == 0 ? min(ns, a.seed_slabs) : 0;
                    nsub = max(1, (ns + QT_META - 1) / QT_META);
                    sub = 0;
                    qb = a.loff[l] + r0;
                    inv_l = DT == 1 ? a.inv_scale8[l] : 1.f;
                }
            }
            __syncwarp();
            if (stop) {
                if (lane == 0) h[8] = QF_STOP;
                __syncwarp();
                mbar_arrive(&cfull[j]);
                break;
            }
            const int ss0 = s0 + sub * QT_META;
            const int sns = max(0, min(QT_META, ns - sub * QT_META));
            const int nblk = (sns * C + NV - 1) / NV;
            if (lane == 0) {
                h[0] = l;
                h[1] = m;
                h[2] = ss0;
                h[3] = sns;
                h[4] = nblk;
                h[7] = chunk;
                h[8] = (sub == 0 ? QF_FIRST : 0) | (sub + 1 == nsub ? QF_LAST : 0);
                h[9] = __float_as_int(inv_l);
            }
            int32_t *qp = c_qpair(j), *cqi = c_qi(j), *crun = c_run(j);
            float *cqn = c_qn(j), *cqsc = c_qsc(j), *ckd = c_kd0(j);
            for (int r = lane; r < QT_M; r += 32) {
                const int pr = r < m ? a.qlist[qb + r] : -1;
                const int qi = pr >= 0 ? pr / a.P : 0;
                const int qrow = a.per_pair ? (pr >= 0 ? pr : 0) : qi;
                qp[r] = pr;
                cqi[r] = qrow;
                cqn[r] = pr >= 0 ? a.qn[qrow] : 0.f;
                cqsc[r] = pr >= 0 ? a.qsc[qrow] : 1.f;
                ckd[r] = pr >= 0 ? __ldcg(a.thr + qi) : INFINITY;
                crun[r] = (pr >= 0 && a.seed_slabs == 0) ? a.prun[pr] : -1;
            }
            int32_t *sl = c_sl(j);
            uint32_t *bt = c_bits(j);
            const int32_t *dirl = a.dir + (size_t)l * a.dir_cap + ss0;
            const int W = C / 32;
            const uint32_t pay_bytes = (uint32_t)(C * d * ESZ);
            for (int i = lane; i < sns; i += 32) {
                const int s = dirl[i];
                const bool okk = s >= 0 && s < a.n_slabs;
                if (!okk) atomicOr(a.err, ERR_BAD_SLAB);
                sl[i] = okk ? s : -1;
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    bt[i * 4 + w] = (okk && w < W) ? __ldg(a.bits + (size_t)s * W + w) : 0u;
                if (okk && i * C < a.pf_tiles * NV) {
                    qt_prefetch_l2(a.pay + (size_t)s * pay_bytes, pay_bytes);
                    qt_prefetch_l2(a.xnorm + (size_t)s * C, (uint32_t)(C * 4));
                }
            }
            __syncwarp();
            mbar_arrive(&cfull[j]);
            ++sub;
        }
    } else if (warp == 3) {
        // ---- query tiles (A operand), rounded and swizzled
        for (int it = 0;; ++it) {
            const int j = it % QT_CTX;
            bool ok = qt_wait(&cfull[j], (uint32_t)(it / QT_CTX) & 1, a.err, s_abort, a.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            if (hdr(j)[8] & QF_STOP) break;
            ok = it < QT_CTX ||
                 qt_wait(&afree[j], (uint32_t)(it / QT_CTX - 1) & 1, a.err, s_abort, a.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int32_t *cqi = c_qi(j);
            const int m = hdr(j)[1];
            unsigned char *Ab = A + (size_t)j * KC * QT_M * 128;
            // 16-byte asynchronous copies of the rounded query rows straight
            // into the swizzled tile; item row i goes to tile row
            // (i % 4) * 32 + i / 4 (tensor-memory lane quarter i % 4);
            // chunks past the row (d * ESZ < KC * 128) are zero-filled; rows
            // past m are left as they are (their lanes are never read)
            const int rowc = d * ESZ / 16, CPR = KC * 8;
            for (int e = lane; e < m * CPR; e += 32) {
                const int i = e / CPR;
                const int r = (i & 3) * 32 + (i >> 2);
                const int c = e - i * CPR, kc = c >> 3, cc = c & 7;
                const bool in = c < rowc;
                const unsigned char *src =
                    a.qcast + (in ? ((size_t)cqi[i] * d * ESZ + (size_t)c * 16) : 0);
                qt_cp_async16(Ab + (size_t)kc * QT_M * 128 + (size_t)(r >> 3) * 1024 +
                                  (r & 7) * 128 + ((cc ^ (r & 7)) << 4),
                              src, in ? 16u : 0u);
            }
            qt_cp_async_wait_all();
            fence_proxy_async_smem();  // the tile is read by the tensor cores (async proxy)
            mbar_arrive(&afull[j]);
        }
    } else if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            uint32_t g = 0;
            const uint32_t pay_bytes = (uint32_t)(C * d * ESZ);
            const int LPT = NV / Cb;  // loads per B tile
            for (int it = 0;; ++it) {
                const int j = it % QT_CTX;
                if (!qt_wait(&cfull[j], (uint32_t)(it / QT_CTX) & 1, a.err, s_abort, a.wait_ns)) break;
                const int32_t *h = hdr(j);
                if (h[8] & QF_STOP) break;
                const int sns = h[3], nblk = h[4];
                const int32_t *sl = c_sl(j);
                bool ab = false;
                for (int b = 0; b < nblk; ++b, ++g) {
                    const uint32_t st = g % NST, u = g / NST, xs = g % QT_XR, xu = g / QT_XR;
                    if (u >= 1 && !qt_wait(&empty[st], (u - 1) & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    if (xu >= 1 && !qt_wait(&xempty[xs], (xu - 1) & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    int okc = 0;
                    for (int i = 0; i < LPT; ++i) {
                        const int rho = b * NV + i * Cb, mi = rho / C;
                        okc += mi < sns && sl[mi] >= 0;
                    }
                    mbar_arrive_expect_tx(&full[st], (uint32_t)(okc * KC * Cb * 128));
                    mbar_arrive_expect_tx(&xfull[xs], (uint32_t)(okc * Cb * 4));
                    for (int i = 0; i < LPT; ++i) {
                        const int rho = b * NV + i * Cb, mi = rho / C, off = rho - mi * C;
                        if (mi >= sns) break;
                        const int s = sl[mi];
                        if (s < 0) continue;
                        for (int kc = 0; kc < KC; ++kc)
                            tma_load_2d(B + (size_t)st * KC * NV * 128 + (size_t)kc * NV * 128 +
                                            (size_t)i * Cb * 128,
                                        &tmap, kc * EPC, s * C + off, &full[st]);
                        bulk_g2s(XN + (size_t)xs * QT_BCOL + i * Cb,
                                 a.xnorm + (size_t)s * C + off, (uint32_t)(Cb * 4), &xfull[xs]);
                    }
                    // keep the L2 prefetch ahead: the slabs that start in tile b + pf
                    const int bp = b + a.pf_tiles;
                    if (bp < nblk) {
                        const int m0 = (bp * NV + C - 1) / C, m1 = min(sns, ((bp + 1) * NV + C - 1) / C);
                        for (int mi = m0; mi < m1; ++mi) {
                            const int s = sl[mi];
                            if (s < 0) continue;
                            qt_prefetch_l2(a.pay + (size_t)s * pay_bytes, pay_bytes);
                            qt_prefetch_l2(a.xnorm + (size_t)s * C, (uint32_t)(C * 4));
                        }
                    }
                }
                if (ab) break;
            }
            // the copies of the last tiles issued have landed before exit
            for (uint32_t t = g > (uint32_t)NST ? g - NST : 0; t < g; ++t)
                mbar_wait_bounded(&full[t % NST], (t / NST) & 1, a.err);
            for (uint32_t t = g > (uint32_t)QT_XR ? g - QT_XR : 0; t < g; ++t)
                mbar_wait_bounded(&xfull[t % QT_XR], (t / QT_XR) & 1, a.err);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            uint32_t g = 0;
            for (int it = 0;; ++it) {
                const int j = it % QT_CTX;
                if (!qt_wait(&cfull[j], (uint32_t)(it / QT_CTX) & 1, a.err, s_abort, a.wait_ns)) break;
                if (hdr(j)[8] & QF_STOP) break;
                const int nblk = hdr(j)[4];
                if (!qt_wait(&afull[j], (uint32_t)(it / QT_CTX) & 1, a.err, s_abort, a.wait_ns)) break;
                const uint32_t abase = smem_u32(A + (size_t)j * KC * QT_M * 128);
                bool ab = false;
                for (int b = 0; b < nblk; ++b, ++g) {
                    const uint32_t st = g % NST, u = g / NST, buf = g % QT_NB, ub = g / QT_NB;
                    if (!qt_wait(&full[st], u & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    if (ub >= 1 && !qt_wait(&tempty[buf], (ub - 1) & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t bbase = smem_u32(B + (size_t)st * KC * NV * 128);
                    for (int kc = 0; kc < KC; ++kc)
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad =
                                smem_desc_sw128(abase + kc * QT_M * 128 + ks * 32, 1024);
                            const uint64_t bd = smem_desc_sw128(bbase + kc * NV * 128 + ks * 32, 1024);
                            const uint32_t acc = (kc | ks) != 0;
                            if (DT == 0) mma_bf16(tbase + buf * QT_BCOL, ad, bd, idesc, acc);
                            else mma_fp8(tbase + buf * QT_BCOL, ad, bd, idesc, acc);
                        }
                    mma_commit(&tfull[buf]);
                    mma_commit(&empty[st]);
                }
                if (ab) break;
                mma_commit(&afree[j]);
            }
            // the last accumulator is written before the tensor memory is released
            if (g > 0) mbar_wait_bounded(&tfull[(g - 1) % QT_NB], ((g - 1) / QT_NB) & 1, a.err);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp 4 + q owns tensor-memory lanes 32q .. 32q + 31,
        // the item rows i = 4 * lane + q
        const int q = warp - 4;
        const int irow = lane * 4 + q;
        float *scr = SCR + q * 32 * 32;      // staged dot products, [column][lane]
        uint32_t *hist = HIST + q * QT_HIST;
        float *bd = BD;
        int32_t *bs = BS;
        int pr = -1, qi = 0, cnt = 0, run = -1, L4 = 1, MEr = ME;
        float qn = 0.f, sc2 = 2.f, kd = INFINITY, t = -INFINITY, gth = INFINITY;
        uint32_t g = 0;
        const int NCH = NV / 32;  // 32-column chunks per B tile
        // reduce row (lane l of this warp) to its best K'; the new K'-th
        // distance lowers its bound and is published for the query
        auto fold_lane = [&](int l) {
            const int n = __shfl_sync(0xffffffffu, cnt, l);
            const size_t off = (size_t)q * 32 * ME + (size_t)l * MEr;
            const float nk = qt_fold_any(BD + off, BS + off, n, K, hist, lane);
            if (lane == l) {
                cnt = K;
                kd = nk;
                t = fminf(t, qt_bound(nk, qn));
            }
            return nk;
        };
        for (int it = 0;; ++it) {
            const int j = it % QT_CTX;
            const bool ok = qt_wait(&cfull[j], (uint32_t)(it / QT_CTX) & 1, a.err, s_abort, a.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int32_t *h = hdr(j);
            const int flags = h[8];
            if (flags & QF_STOP) break;
            const int m = h[1], sns = h[3], nblk = h[4], chunk = h[7];
            const int32_t *sl = c_sl(j);
            const uint32_t *bt = c_bits(j);
            if (flags & QF_FIRST) {
                const bool act = irow < m;
                pr = act ? c_qpair(j)[irow] : -1;
                qi = pr >= 0 ? pr / a.P : 0;
                qn = act ? c_qn(j)[irow] : 0.f;
                sc2 = DT == 0 ? 2.f : 2.f / (__int_as_float(h[9]) * (act ? c_qsc(j)[irow] : 1.f));
                gth = pr >= 0 ? c_kd0(j)[irow] : INFINITY;
                kd = INFINITY;
                t = pr >= 0 ? qt_bound(gth, qn) : -INFINITY;
                cnt = 0;
                run = act ? c_run(j)[irow] : -1;
                // this warp's quarter of the pool (32 * ME entries) split over
                // its ceil(m / 4) rows, an odd row length; the warps move
                // from item to item independently, so each keeps to its own
                // quarter
                L4 = (m + 3) >> 2;
                MEr = min(a.mecap, (32 * ME) / L4);
                if ((MEr & 1) == 0) --MEr;
                bd = BD + (size_t)q * 32 * ME + (size_t)lane * MEr;
                bs = BS + (size_t)q * 32 * ME + (size_t)lane * MEr;
            }
            bool run_ok = true;
            for (int b = 0; b < nblk; ++b, ++g) {
                const uint32_t buf = g % QT_NB, ub = g / QT_NB, xs = g % QT_XR, xu = g / QT_XR;
                bool wok = qt_wait(&xfull[xs], xu & 1, a.err, s_abort, a.wait_ns);
                wok = wok && qt_wait(&tfull[buf], ub & 1, a.err, s_abort, a.wait_ns);
                wok = __all_sync(0xffffffffu, wok);  // tcgen05.ld is warp-aligned
                if (!wok) {
                    run_ok = false;
                    break;
                }
                tc_fence_after();
                // the query's shared bound, as read one tile ago; read it again
                if (pr >= 0) {
                    t = fminf(t, qt_bound(gth, qn));
                    gth = __ldcg(a.thr + qi);
                }
                for (int c = 0; c < NCH; ++c) {
                    float acc[32];
                    tmem_ld32(tbase + buf * QT_BCOL + c * 32 + ((uint32_t)(q * 32) << 16), acc);
                    tmem_ld_wait();
                    if (c == NCH - 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[buf]);
                    }
                    // the chunk's 32 rows of the list: slab, offset, validity
                    const int rho = b * NV + c * 32, mi = rho / C, off = rho - mi * C;
                    const bool has = mi < sns;
                    const uint32_t vw = has ? bt[mi * 4 + (off >> 5)] : 0u;
                    const int32_t base = has ? sl[mi] * C + off : 0;
                    const float *xnc = XN + xs * QT_BCOL + c * 32;
                    float xn[32];
                    const float4 *x4 = reinterpret_cast<const float4 *>(xnc);
#pragma unroll
                    for (int i4 = 0; i4 < 8; ++i4) {
                        const float4 v = x4[i4];
                        xn[4 * i4] = v.x;
                        xn[4 * i4 + 1] = v.y;
                        xn[4 * i4 + 2] = v.z;
                        xn[4 * i4 + 3] = v.w;
                    }
                    uint32_t pm = 0u;
                    if (__all_sync(0xffffffffu, pr < 0 || t >= QT_NOBOUND)) {
                        pm = vw;  // no row of the warp has a bound yet: every valid column
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            if (fmaf(-sc2, acc[jj], xn[jj]) <= t) pm |= 1u << jj;
                        pm &= vw;
                    }
                    if (pr < 0) pm = 0u;
                    if (!__any_sync(0xffffffffu, pm != 0u)) continue;
                    // every column passes and fits: stored at once
                    if (pm == 0xffffffffu && cnt + 32 <= MEr) {
                        const float qx = qn;
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            bd[cnt + jj] = fmaf(-sc2, acc[jj], qx + xn[jj]);
                            bs[cnt + jj] = base + jj;
                        }
                        cnt += 32;
                        pm = 0u;
                    }
                    if (!__any_sync(0xffffffffu, pm != 0u)) continue;
                    // the rest one by one: the chunk's dot products are staged
                    // in shared memory ([column][lane]) so each lane walks its
                    // own passing columns; a row whose buffer fills is reduced
                    // by the warp and its remaining columns are tested again
                    // against the lowered bound
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) scr[jj * 32 + lane] = acc[jj];
                    __syncwarp();
                    for (int guard = 0; guard < 64; ++guard) {
                        while (pm != 0u && cnt < MEr) {
                            const int jj = __ffs(pm) - 1;
                            pm &= pm - 1u;
                            const float av = scr[jj * 32 + lane], xv = xnc[jj];
                            if (fmaf(-sc2, av, xv) <= t) {
                                bd[cnt] = fmaf(-sc2, av, qn + xv);
                                bs[cnt] = base + jj;
                                ++cnt;
                            }
                        }
                        uint32_t fullr = __ballot_sync(0xffffffffu, pm != 0u);
                        if (!fullr) break;
                        while (fullr) {
                            const int l = __ffs(fullr) - 1;
                            fullr &= fullr - 1;
                            const float nk = fold_lane(l);
                            if (lane == l && nk >= 0.f && nk < INFINITY)
                                atomicMin(reinterpret_cast<int *>(a.thr) + qi, __float_as_int(nk));
                        }
                    }
                    if (pm) atomicOr(a.err, ERR_PLAN);  // unreachable: ME > K'
                    __syncwarp();
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&xempty[xs]);
            }
            if (!run_ok) {
                if (lane == 0) *s_abort = 1;
                break;
            }
            if (flags & QF_LAST) {
                // rows holding more than K': their best K'; the K'-th becomes
                // a bound of the query for the items that follow
                uint32_t over = __ballot_sync(0xffffffffu, pr >= 0 && cnt > K);
                while (over) {
                    const int l = __ffs(over) - 1;
                    over &= over - 1;
                    fold_lane(l);
                }
                if (pr >= 0 && cnt >= K && kd >= 0.f && kd < INFINITY)
                    atomicMin(reinterpret_cast<int *>(a.thr) + qi, __float_as_int(kd));
                // each row's run: its candidates unsorted, with their count
                uint32_t rows = __ballot_sync(0xffffffffu, pr >= 0 && run >= 0);
                while (rows) {
                    const int l = __ffs(rows) - 1;
                    rows &= rows - 1;
                    const int n = __shfl_sync(0xffffffffu, cnt, l);
                    const int rn = __shfl_sync(0xffffffffu, run, l);
                    const size_t off = (size_t)q * 32 * ME + (size_t)l * MEr;
                    const int64_t ob = ((int64_t)rn + chunk) * K;
                    for (int i = lane; i < n; i += 32) {
                        a.part_d[ob + i] = BD[off + i];
                        a.part_i[ob + i] = (int64_t)BS[off + i];
                    }
                    if (lane == 0) a.part_n[rn + chunk] = n;
                }
                __syncwarp();
            }
            if (lane == 0) mbar_arrive(&cempty[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tbase, QT_NB * QT_BCOL);
}

// --------------------------------------------------------------- host side
// dynamic shared memory one CTA may take (the kernel has no static arrays)
constexpr size_t kQtSmemMax = 227 * 1024 - 1024;

QtShape qt_shape(const sivf_index *ix, int dtype, int Kc)
{
    QtShape s{};
    const int esz = dtype == SIVF_BF16 ? 2 : 1;
    s.KC = (ix->d * esz + 127) / 128;
    s.NV = 128 / s.KC;
    if (s.NV < 32 || s.NV % std::min(ix->C, 64) || (s.NV < ix->C && ix->C % s.NV)) return s;
    // the deepest buffer that fits beside as many B stages as possible,
    // preferring room for 48 candidates beyond K' over a fourth stage
    for (int pass = 0; pass < 2; ++pass)
        for (int nst = QT_MAXST; nst >= 2; --nst) {
            const size_t fixed = qt_smem(s.KC, nst, 0).total;
            if (fixed >= kQtSmemMax) continue;
            int me = (int)((kQtSmemMax - fixed) / (QT_M * 8));
            me = std::min(me, 32 * QT_MAXEK);
            if (me % 2 == 0) --me;  // odd row stride: appends of one warp hit distinct banks
            const int want = Kc + (pass == 0 ? 48 : 16);
            if (me >= want) {
                s.nst = nst;
                s.ME = me;
                s.smem = qt_smem(s.KC, nst, me).total;
                s.ok = true;
                return s;
            }
        }
    return s;
}

bool qt_make_maps(sivf_index *ix, PFN_cuTensorMapEncodeTiled_v12000 enc)
{
    const cuuint64_t rows = (cuuint64_t)ix->n_slabs * ix->C;
    const cuuint32_t cb = (cuuint32_t)std::min(ix->C, 64);
    if (ix->xb16) {
        cuuint64_t dims[2] = {(cuuint64_t)ix->d, rows};
        cuuint64_t strides[1] = {(cuuint64_t)ix->d * 2};
        cuuint32_t box[2] = {64, cb};
        cuuint32_t es[2] = {1, 1};
        if (enc(reinterpret_cast<CUtensorMap *>(ix->tmap_qt_bf16), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                2, ix->xb16, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    if (ix->x8) {
        cuuint64_t dims[2] = {(cuuint64_t)ix->d, rows};
        cuuint64_t strides[1] = {(cuuint64_t)ix->d};
        cuuint32_t box[2] = {128, cb};
        cuuint32_t es[2] = {1, 1};
        if (enc(reinterpret_cast<CUtensorMap *>(ix->tmap_qt_fp8), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                ix->x8, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

template <int DT>
static void launch_qt(const unsigned char *tmap, const QtArgs &a, size_t smem, cudaStream_t st)
{
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_scan_qt<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    launch_pdl(k_scan_qt<DT>, 152, QT_NT, smem, st, *reinterpret_cast<const CUtensorMap *>(tmap),
               a);
}

// longest candidate buffer of one row for the tile's select_slabs (0: 255,
// a bisection in registers; 1, 2, 3: 255, 1023, 2047, radix selects past 256)
int qt_mecap(int select_slabs)
{
    return select_slabs <= 1 ? 255 : select_slabs == 2 ? 1023 : QT_MECAP;
}

void scan_lists_qt(sivf_index *ix, int dtype, int64_t nq, int P, int Kc, int seed_slabs,
                   int select_slabs, const SearchScratch &s, cudaStream_t st)
{
    const QtShape sh = qt_shape(ix, dtype, Kc);
    QtArgs a;
    a.nq = nq;
    a.P = P;
    a.K = Kc;
    a.ME = sh.ME;
    a.qlist = s.qlist;
    a.loff = s.loff;
    a.lcnt = s.lcnt;
    a.nch = s.nch;
    a.prun = s.prun;
    a.items = s.items;
    a.per_pair = dtype == SIVF_FP8E4M3;
    a.qn = a.per_pair ? s.pqn : s.qn;
    a.qsc = a.per_pair ? s.pqsc : s.qsc;
    a.qcast = s.qcast;
    a.part_d = s.part_d;
    a.part_i = s.part_i;
    a.part_n = s.part_n;
    a.thr = s.thr;
    a.xnorm = a.per_pair ? ix->rnorm : ix->xnorm;
    a.bits = ix->bits;
    a.nslabs = ix->nslabs;
    a.dir = ix->dir;
    a.inv_scale8 = ix->inv_scale8;
    const int esz = dtype == SIVF_BF16 ? 2 : 1;
    a.pay = dtype == SIVF_BF16 ? reinterpret_cast<const unsigned char *>(ix->xb16) : ix->x8;
    a.n_slabs = ix->n_slabs;
    a.dir_cap = ix->dir_cap;
    a.d = ix->d;
    a.C = ix->C;
    a.KC = sh.KC;
    a.NV = sh.NV;
    a.nst = sh.nst;
    a.seed_slabs = seed_slabs;
    a.mecap = qt_mecap(select_slabs);
    a.wait_ns = ix->wait_ns;
    a.pf_tiles = std::max(2, QT_PF_BYTES / (sh.NV * ix->d * esz));
    a.ctl = ix->ctl;
    a.err = ix->err;
    const int tok = prof_begin(ix, PROF_SCAN, 1, st);
    if (dtype == SIVF_BF16) launch_qt<0>(ix->tmap_qt_bf16, a, sh.smem, st);
    else launch_qt<1>(ix->tmap_qt_fp8, a, sh.smem, st);
    prof_end(ix, tok, st);
}

}  // namespace sivf
