// Reduced-precision list scan on the tensor cores, then an exact FP32
// re-rank (the precision pattern of the hot path; the paper scans FP32
// only).
//
// Lists keep a BF16 or an FP8 E4M3 copy of every payload row (per-list
// scale for FP8).  One persistent CTA per SM takes (list, tile of up to TN
// queries, slab chunk) items from a work counter.  The list's slabs stream
// through shared memory as 128-row A tiles (TMA 2-D loads, 128-byte
// swizzle); the query tile, rounded to the same format, is the B operand;
// tcgen05.mma accumulates the 128 x TN dot products in FP32 in tensor
// memory (two accumulators, so the next tile's MMAs overlap the epilogue of
// this one).  The epilogue forms the expanded distance
// ||q||^2 + ||x||^2 - 2 s q.x (FP32 norms of the unrounded vectors, s the
// dequantisation scale), and every query keeps its best K' (= 4k)
// (distance, slot) candidates.  A per-query shared bound (the K'-th
// distance any item has found) prunes the rest.  A final pass recomputes
// the K' survivors' distances exactly in FP32 from the FP32 payload and
// keeps the best k by (distance, id).
//
// Roles inside the CTA, all running one item ahead of the epilogue:
//   warp 2  item contexts: takes the next item, stages its queries' norms,
//           scales and bounds, its slab ids and validity bitmaps, and
//           prefetches the first slabs into L2 (two contexts in flight);
//   warp 3  builds the rounded, swizzled query tile (two B buffers);
//   warp 0  (one lane) TMA loads of the A tiles, plus L2 prefetches of
//           the payload rows and their ||x||^2 further ahead in the list;
//   warp 1  (one lane) issues the MMAs; warp 2 also owns the TMEM;
//   warps 4.. the epilogue: TN / 16 warps per TMEM lane quarter, 16
//           query columns each; each thread reads its row's ||x||^2 from
//           global memory (L2) before it waits for the accumulator.
// A tile's passing rows are appended to their query's buffer at positions
// reserved by one shared atomic per (warp, query); a buffer is reduced to
// its best K' (radix select, left unsorted) only after a tile that leaves
// it too full for the next one, so most tiles end on a single barrier.
// Each item writes its rows' best K' unsorted; a per-query merge selects
// and sorts the best K' of all its items.  Every wait is bounded, and a
// wait that gives up stops every role.
#include <cudaTypedefs.h>
#include <math.h>

#include "device_utils.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace sivf {

constexpr int TC_M = 128;       // rows per A tile (MMA M)
constexpr int TC_NCOL = 16;     // query columns per epilogue warp
constexpr int TC_META = 256;    // slabs of one sub-item (ids and bitmaps staged together)
constexpr int TC_CTX = 2;       // item contexts in flight
constexpr int TC_MAXST = 4;     // most A-tile stages
constexpr int TC_HIST = 256;    // radix-select bins per epilogue warp
constexpr int TC_PF_BYTES = 192 * 1024;  // L2 prefetch distance per CTA

// Query tiles: 48 queries for K' <= 64 (small enough candidate buffers for
// three A stages), 32 for K' <= 128, 16 (and candidate buffers up to
// K' = 512) for deeper re-ranks.  TN / 16 epilogue warps per TMEM lane
// quarter, 16 query columns each.
template <int TN> struct TcShape {
    static constexpr int N = TN;                        // queries per tile (MMA N)
    static constexpr int EW = 4 * (TN / TC_NCOL);       // epilogue warps
    static constexpr int EPI = EW * 32;                 // epilogue threads
    static constexpr int NT = 128 + EPI;                // + TMA, MMA, context, B warps
    static constexpr int KMAX = TN == 48 ? 64 : TN == 32 ? 128 : 512;  // deepest K'
    // TMEM columns per accumulator buffer (power of two, >= 32)
    static constexpr int TB = TN <= 32 ? 32 : 64;
};

struct TcArgs {
    const float *q;
    int64_t nq;
    int P, K, M;
    const int32_t *qlist, *loff, *lcnt, *ibase, *nch;
    const int32_t *prun;  // first output run of each pair (-1: not scanned)
    const int2 *items;
    const float *qn, *qsc;
    const unsigned char *qcast;  // [nq, d] queries in the scan format (BF16), or
                                 // [nq * P, d] residuals q - c_l of each pair (E4M3)
    int per_pair;                // qn, qsc, qcast are per (query, probe) pair (FP8)
    float *part_d;
    int64_t *part_i;  // global slot (slab * C + slot) of each candidate
    int32_t *part_n;  // candidates in each run (at most RK)
    int RK;           // run length: K' plus room an approximate reduction may keep
    float *thr;
    const float *xnorm;
    const uint32_t *bits;
    const int32_t *nslabs, *dir;
    const float *inv_scale8;
    const unsigned char *pay;  // the scanned copy (BF16 or E4M3 rows)
    int64_t n_slabs, dir_cap;
    int L, d, C, KC;  // KC = 128-byte K chunks per row
    int nst;          // A-tile stages
    int pf_tiles;     // A tiles prefetched into L2 ahead of the loads
    uint64_t wait_ns; // time after which a wait of the scan gives up
    int seed_slabs;   // > 0: seed launch: the first seed_slabs slabs of each
                      // item, bounds published, no runs written
    int tile_box;     // the 128-row map is valid: a tile of consecutive slabs
                      // is one TMA box
    Ctl *ctl;
    uint32_t *err;
};

// One item context: a header, the tile's queries, the sub-item's slabs.
//   int32 hdr[16]: list, m, first slab, slabs, A tiles, row stride ME,
//                  -, chunk, flags (1 first, 2 last, 4 stop), inv scale
//   int32 qpair[TN]; float qn[TN], qsc[TN], kd0[TN]; int32 qi[TN];
//   int32 sl[TC_META]; uint32 bits[TC_META][4]
enum : int { CF_FIRST = 1, CF_LAST = 2, CF_STOP = 4 };
__host__ __device__ constexpr size_t tc_ctx_bytes(int TN)
{
    return 64 + (size_t)20 * TN + (size_t)4 * TC_META + (size_t)16 * TC_META;
}

struct TcSmem {
    size_t a, b, xn, bd, bs, ctx, hist, bars, total;
};
template <int TN>
__host__ __device__ inline TcSmem tc_smem(int KC, int M, int nst)
{
    using S = TcShape<TN>;
    TcSmem s;
    s.a = 0;                                             // nst x KC x 16 KB
    s.b = s.a + (size_t)nst * KC * TC_M * 128;           // 2 x KC x TN rows x 128 B
    s.xn = s.b + (size_t)2 * KC * TN * 128;              // (no norm ring)
    s.bd = s.xn;
    s.bs = s.bd + (size_t)TN * M * 4;
    s.ctx = s.bs + (size_t)TN * M * 4;
    s.hist = s.ctx + (size_t)TC_CTX * tc_ctx_bytes(TN);
    s.bars = s.hist + (size_t)S::EW * TC_HIST * 4;
    s.total = s.bars + 48 * 8 + 1024;                    // + base alignment slack
    return s;
}

// (distance, slot) order with pads (+inf, INT_MAX) last
__device__ __forceinline__ bool ds_less(float a, int32_t sa, float b, int32_t sb)
{
    return a < b || (a == b && sa < sb);
}

// 64-bit key with the (distance, slot) order
__device__ __forceinline__ uint64_t ds_key(float d, int32_t s)
{
    return ((uint64_t)fkey(d) << 32) | (uint32_t)s;
}

// Ascending bitonic sort of 32*E (distance, slot) pairs held E per lane.
template <int E>
__device__ __forceinline__ void warp_sort32(float (&v)[E], int32_t (&s)[E], int lane)
{
    constexpr int N = 32 * E;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1)
#pragma unroll
        for (int st = size >> 1; st > 0; st >>= 1)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane + 32 * e;
                const bool up = (i & size) == 0;
                if (st >= 32) {
                    const int pe = e ^ (st >> 5);
                    if (pe > e) {
                        const bool sw = up ? ds_less(v[pe], s[pe], v[e], s[e])
                                           : ds_less(v[e], s[e], v[pe], s[pe]);
                        if (sw) {
                            const float tv = v[e];
                            v[e] = v[pe];
                            v[pe] = tv;
                            const int32_t ts = s[e];
                            s[e] = s[pe];
                            s[pe] = ts;
                        }
                    }
                } else {
                    const float ov = __shfl_xor_sync(0xffffffffu, v[e], st);
                    const int32_t os = __shfl_xor_sync(0xffffffffu, s[e], st);
                    const bool lower = (lane & st) == 0;
                    const bool take = (lower == up) ? ds_less(ov, os, v[e], s[e])
                                                    : ds_less(v[e], s[e], ov, os);
                    if (take) {
                        v[e] = ov;
                        s[e] = os;
                    }
                }
            }
}

// Radix select over n distinct 64-bit keys key(i), i < n: returns the
// (prefix, mask) for which exactly the K smallest keys satisfy
// (key & mask) <= prefix.  Keys equal to ~0 are padding: they never count
// among the K smallest, and at least K keys are not padding.  8 bits per
// pass, starting at the highest bit where the keys differ and stopping at
// the first pass whose chosen bin is taken whole.
template <class KeyF>
__device__ __forceinline__ void warp_radix_kth(KeyF key, int n, int K, uint32_t *hist, int lane,
                                               uint64_t &prefix_out, uint64_t &mask_out)
{
    uint64_t kmin = ~0ull, kmax = 0ull;
    for (int i = lane; i < n; i += 32) {
        const uint64_t k = key(i);
        if (k != ~0ull) {
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
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
        for (int i = lane; i < n; i += 32) {
            const uint64_t k = key(i);
            if (k != ~0ull && (k & mask) == prefix)
                atomicAdd(&hist[(uint32_t)(k >> shift) & bmask], 1u);
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
    prefix_out = prefix;
    mask_out = mask;
}

// Keep in bd/bs[0, K) the K smallest (distance, slot) entries of the two
// unsorted runs [0, nb) and [PB, PB + nc) (PB >= K), with nb + nc > K; the kept
// entries stay unsorted (a slot appears once per buffer, so the keys are
// distinct).  Returns the largest kept distance.
__device__ float warp_select_keep(float *bd, int32_t *bs, int K, int PB, int nb, int nc,
                                  uint32_t *hist, int lane)
{
    auto at = [&](int i) { return i < nb ? i : PB + (i - nb); };
    uint64_t prefix, mask;
    warp_radix_kth([&](int i) { return ds_key(bd[at(i)], bs[at(i)]); }, nb + nc, K, hist, lane,
                   prefix, mask);
    // stable compaction in place (every write index <= its read index)
    int w = 0;
    float dmax = -INFINITY;
    for (int i0 = 0; i0 < nb; i0 += 32) {
        const int i = i0 + lane;
        float dv = 0.f;
        int32_t sv = 0;
        bool take = false;
        if (i < nb) {
            dv = bd[i];
            sv = bs[i];
            take = (ds_key(dv, sv) & mask) <= prefix;
        }
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        __syncwarp();
        if (take) {
            const int p = w + __popc(mk & lanemask_lt());
            bd[p] = dv;
            bs[p] = sv;
            dmax = fmaxf(dmax, dv);
        }
        w += __popc(mk);
        __syncwarp();
    }
    for (int i0 = 0; i0 < nc; i0 += 32) {
        const int i = PB + i0 + lane;
        float dv = 0.f;
        int32_t sv = 0;
        bool take = false;
        if (i0 + lane < nc) {
            dv = bd[i];
            sv = bs[i];
            take = (ds_key(dv, sv) & mask) <= prefix;
        }
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        if (take) {
            const int p = w + __popc(mk & lanemask_lt());
            if (p < K) {
                bd[p] = dv;
                bs[p] = sv;
            }
            dmax = fmaxf(dmax, dv);
        }
        w += __popc(mk);
    }
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    return dmax;
}

// Reduce the two unsorted runs [0, nb) and [PB, PB + nc) of one row
// (nb + nc <= 32 * EK, more than Kw entries) to between K and Kw of their
// smallest (distance, slot) entries, written unsorted to [0, kept); returns
// the largest kept distance, a bound on the row's K-th smallest.  The
// 32-bit distance keys and the slots live in registers; a bisection on the
// key value with ballot counts stops at the first value with between K and
// Kw keys at or below it, which takes a few rounds where the exact K-th
// needs one per key bit.  Only when ties at the K-th key span past Kw is
// the cut made exact (K kept, ties to the lower slots).
template <int EK>
__device__ float warp_select_window(float *bd, int32_t *bs, int K, int Kw, int PB, int nb,
                                    int nc, int lane, int &kept)
{
    const int n = nb + nc;
    uint32_t key[EK];
    int32_t slt[EK];
#pragma unroll
    for (int e = 0; e < EK; ++e) {
        const int i = lane + 32 * e;
        const int ai = i < nb ? i : PB + (i - nb);
        key[e] = i < n ? fkey(bd[ai]) : 0xffffffffu;
        slt[e] = i < n ? bs[ai] : 0x7fffffff;
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
    // invariant: #(key <= hi) >= K; stop at any value with K..Kw keys below
    uint32_t lo = kmin, hi = kmax, cnt = 0;
    bool found = false;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        uint32_t c = 0;
#pragma unroll
        for (int e = 0; e < EK; ++e) c += __popc(__ballot_sync(0xffffffffu, key[e] <= mid));
        if (c >= (uint32_t)K && c <= (uint32_t)Kw) {
            lo = mid;
            cnt = c;
            found = true;
            break;
        }
        if (c > (uint32_t)Kw) hi = mid;
        else lo = mid + 1;
    }
    const uint32_t v = lo;  // found: K..Kw keys <= v; else v is the K-th key
    if (!found) {
        uint32_t c = 0;
#pragma unroll
        for (int e = 0; e < EK; ++e) c += __popc(__ballot_sync(0xffffffffu, key[e] <= v));
        cnt = c;
    }
    int32_t cut = 0x7fffffff;  // entries equal to v kept: slot <= cut
    if (cnt > (uint32_t)Kw) {  // ties at v span past Kw: keep exactly K
        uint32_t clt = 0;
#pragma unroll
        for (int e = 0; e < EK; ++e) clt += __popc(__ballot_sync(0xffffffffu, key[e] < v));
        const uint32_t need = (uint32_t)K - clt;
        int32_t slo = 0, shi = 0x7fffffff;
        while (slo < shi) {
            const int32_t mid = slo + ((shi - slo) >> 1);
            uint32_t c = 0;
#pragma unroll
            for (int e = 0; e < EK; ++e)
                c += __popc(__ballot_sync(0xffffffffu, key[e] == v && slt[e] <= mid));
            if (c >= need) shi = mid;
            else slo = mid + 1;
        }
        cut = slo;
    }
    __syncwarp();  // every lane has read its entries before any is written
    int w = 0;
    uint32_t kk = 0u;
#pragma unroll
    for (int e = 0; e < EK; ++e) {
        const bool take = key[e] < v || (key[e] == v && slt[e] <= cut);
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        if (take) {
            const int p = w + __popc(mk & lanemask_lt());
            bd[p] = fkey_inv(key[e]);
            bs[p] = slt[e];
            kk = max(kk, key[e]);
        }
        w += __popc(mk);
    }
    __syncwarp();
    kept = w;
    return fkey_inv(__reduce_max_sync(0xffffffffu, kk));
}

// Fold the nc pending candidates of one row (at [PB, PB + nc)) into its
// held set [0, nb): when the union holds more than Kw entries it is reduced
// to between K and Kw of its smallest (exactly K for long buffers, by the
// radix select), else the pending entries move down whole.  Returns a bound
// on the row's K-th smallest distance (+inf while fewer than K are held).
__device__ __forceinline__ float fold_row(float *bd, int32_t *bs, int K, int Kw, int PB, int &nb,
                                          int nc, uint32_t *hist, int lane)
{
    const int n = nb + nc;
    if (n > Kw) {
        int kept = K;
        const float kd = n <= 64    ? warp_select_window<2>(bd, bs, K, Kw, PB, nb, nc, lane, kept)
                         : n <= 128 ? warp_select_window<4>(bd, bs, K, Kw, PB, nb, nc, lane, kept)
                         : n <= 192 ? warp_select_window<6>(bd, bs, K, Kw, PB, nb, nc, lane, kept)
                         : n <= 320 ? warp_select_window<10>(bd, bs, K, Kw, PB, nb, nc, lane, kept)
                                    : warp_select_keep(bd, bs, K, PB, nb, nc, hist, lane);
        nb = kept;
        return kd;
    }
    for (int i = lane; i < nc; i += 32) {  // write index < PB <= read index
        const float dv = bd[PB + i];
        const int32_t sv = bs[PB + i];
        bd[nb + i] = dv;
        bs[nb + i] = sv;
    }
    nb += nc;
    __syncwarp();
    if (nb < K) return INFINITY;
    float dmax = -INFINITY;
    for (int i = lane; i < nb; i += 32) dmax = fmaxf(dmax, bd[i]);
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    return dmax;
}

// mbarrier wait bounded in time (the index's wait limit) that also gives
// up as soon as another role of the CTA has stopped (abort flag in shared
// memory); a wait that runs out sets ERR_TIMEOUT and the abort flag.
// Copies already in flight are drained by the producer with the default
// limit before the CTA exits.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *bar, uint32_t parity, uint32_t *err,
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

// named barrier over `n` threads that also returns the AND of `pred`
__device__ __forceinline__ bool named_bar_and(int id, int n, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// named barrier over `n` threads that also returns the OR of `pred`
__device__ __forceinline__ bool named_bar_or(int id, int n, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// 16-byte asynchronous copy global -> shared; bytes past `src_bytes` (0 or
// 16) are zero-filled
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

template <int DT, int TN>  // DT: 0 = BF16, 1 = FP8 E4M3; TN: queries per tile
__global__ __launch_bounds__(TcShape<TN>::NT, 1) void k_scan_tc(
    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_t,
    TcArgs a)
{
    pdl_begin();
    using S = TcShape<TN>;
    constexpr int EW = S::EW, EPI = S::EPI, TB = S::TB;
    constexpr int ESZ = DT == 0 ? 2 : 1;
    constexpr int EPC = 128 / ESZ;  // elements per 128-byte chunk
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled operand tiles
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int KC = a.KC, M = a.M, K = a.K, C = a.C, d = a.d, NST = a.nst;
    const TcSmem L = tc_smem<TN>(KC, M, NST);
    unsigned char *A = smem + L.a;
    unsigned char *B = smem + L.b;
    float *BD = reinterpret_cast<float *>(smem + L.bd);
    int32_t *BS = reinterpret_cast<int32_t *>(smem + L.bs);
    unsigned char *CTX = smem + L.ctx;
    uint32_t *Hist = reinterpret_cast<uint32_t *>(smem + L.hist);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *full = bars, *empty = bars + 4, *tfull = bars + 8, *tempty = bars + 10,
             *cfull = bars + 28, *cempty = bars + 30,
             *bfull = bars + 32, *bfree = bars + 34;
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(bars + 40);
    volatile int *s_abort = reinterpret_cast<volatile int *>(bars + 41);
    __shared__ int32_t s_cnt[TN], s_nb[TN];  // pending candidates, held best
    __shared__ float s_kd[TN];
    __shared__ __align__(16) float s_t[TN];   // kd - ||q||^2 of each row
    __shared__ __align__(16) float s_sc[TN];  // 2 x dequantisation scale of each row

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int SPB = TC_M / C;  // slabs per A tile
    const uint32_t idesc = DT == 0 ? mma_idesc(1, 1, TC_M, TN) : mma_idesc(0, 0, TC_M, TN);
    constexpr size_t CTXB = tc_ctx_bytes(TN);
    auto hdr = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CTXB); };
    auto c_qpair = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CTXB + 64); };
    auto c_qn = [&](int j) { return reinterpret_cast<float *>(CTX + j * CTXB + 64 + 4 * TN); };
    auto c_qsc = [&](int j) { return reinterpret_cast<float *>(CTX + j * CTXB + 64 + 8 * TN); };
    auto c_kd0 = [&](int j) { return reinterpret_cast<float *>(CTX + j * CTXB + 64 + 12 * TN); };
    auto c_qi = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CTXB + 64 + 16 * TN); };
    auto c_sl = [&](int j) { return reinterpret_cast<int32_t *>(CTX + j * CTXB + 64 + 20 * TN); };
    auto c_bits = [&](int j) {
        return reinterpret_cast<uint32_t *>(CTX + j * CTXB + 64 + 20 * TN + 4 * TC_META);
    };

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], EW);
            mbar_init(&bfull[i], 32);
            mbar_init(&bfree[i], 1);
        }
        for (int i = 0; i < TC_CTX; ++i) {
            mbar_init(&cfull[i], 32);
            mbar_init(&cempty[i], EW);
        }
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == 2) tmem_alloc(tmem_base, 2 * TB);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_base;

    if (warp == 2) {
        // ---- item contexts
        int sub = 0, nsub = 0, l = 0, m = 0, s0 = 0, ns = 0, chunk = 0, qb = 0;
        float inv_l = 1.f;
        for (int it = 0;; ++it) {
            const int j = it % TC_CTX;
            const uint32_t cu = (uint32_t)(it / TC_CTX);
            bool ok = cu == 0 || mbar_wait_ab(&cempty[j], (cu - 1) & 1, a.err, s_abort, a.wait_ns);
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
                    const int r0 = tile * TN;
                    m = min(TN, a.lcnt[l] - r0);
                    int ns_total = a.nslabs[l];
                    if (ns_total > a.dir_cap) {
                        if (lane == 0) atomicOr(a.err, ERR_DIR_BOUND);
                        ns_total = (int)a.dir_cap;
                    }
                    s0 = (int)((int64_t)ns_total * chunk / nc_l);
                    ns = (int)((int64_t)ns_total * (chunk + 1) / nc_l) - s0;
                    if (a.seed_slabs > 0) ns = chunk == 0 ? min(ns, a.seed_slabs) : 0;
                    nsub = max(1, (ns + TC_META - 1) / TC_META);
                    sub = 0;
                    qb = a.loff[l] + r0;
                    inv_l = DT == 1 ? a.inv_scale8[l] : 1.f;
                }
            }
            __syncwarp();
            if (stop) {
                if (lane == 0) h[8] = CF_STOP;
                __syncwarp();
                mbar_arrive(&cfull[j]);
                break;
            }
            const int ss0 = s0 + sub * TC_META;
            const int sns = max(0, min(TC_META, ns - sub * TC_META));
            const int nblk = (sns + SPB - 1) / SPB;
            if (lane == 0) {
                h[0] = l;
                h[1] = m;
                h[2] = ss0;
                h[3] = sns;
                h[4] = nblk;
                h[5] = max(M, ((TN * M) / max(m, 1)) & ~7);  // rows of a thin tile get longer buffers
                h[7] = chunk;
                h[8] = (sub == 0 ? CF_FIRST : 0) | (sub + 1 == nsub ? CF_LAST : 0);
                h[9] = __float_as_int(inv_l);
            }
            int32_t *qp = c_qpair(j), *cqi = c_qi(j);
            float *cqn = c_qn(j), *cqsc = c_qsc(j), *ckd = c_kd0(j);
            for (int r = lane; r < TN; r += 32) {
                const int pr = r < m ? a.qlist[qb + r] : -1;
                const int qi = pr >= 0 ? pr / a.P : 0;
                const int qrow = a.per_pair ? (pr >= 0 ? pr : 0) : qi;  // row of qn, qsc, qcast
                qp[r] = pr;
                cqi[r] = qrow;
                cqn[r] = pr >= 0 ? a.qn[qrow] : 0.f;
                cqsc[r] = pr >= 0 ? a.qsc[qrow] : 1.f;
                ckd[r] = pr >= 0 ? __ldcg(a.thr + qi) : INFINITY;
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
                for (int w = 0; w < W; ++w) bt[i * 4 + w] = okk ? __ldg(a.bits + (size_t)s * W + w) : 0u;
                if (okk && i < a.pf_tiles * SPB) {
                    prefetch_l2(a.pay + (size_t)s * pay_bytes, pay_bytes);
                    prefetch_l2(a.xnorm + (size_t)s * C, (uint32_t)(C * 4));
                }
            }
            __syncwarp();
            mbar_arrive(&cfull[j]);
            ++sub;
        }
    } else if (warp == 3) {
        // ---- query tiles (B operand), rounded and swizzled
        for (int it = 0;; ++it) {
            const int j = it % TC_CTX, bb = it & 1;
            bool ok = mbar_wait_ab(&cfull[j], (uint32_t)(it / TC_CTX) & 1, a.err, s_abort, a.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            if (hdr(j)[8] & CF_STOP) break;
            ok = it < 2 || mbar_wait_ab(&bfree[bb], (uint32_t)((it >> 1) - 1) & 1, a.err, s_abort, a.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int32_t *cqi = c_qi(j);
            const int m = hdr(j)[1];
            unsigned char *Bb = B + (size_t)bb * KC * TN * 128;
            // 16-byte asynchronous copies of the rounded query rows straight
            // into the swizzled tile (no registers, every copy in flight at
            // once); chunks past the row (d * ESZ < KC * 128) are zero-filled
            const int rowc = d * ESZ / 16, CPR = KC * 8;
            for (int e = lane; e < m * CPR; e += 32) {
                const int r = (CPR & (CPR - 1)) == 0 ? e >> (__ffs(CPR) - 1) : e / CPR;
                const int c = e - r * CPR, kc = c >> 3, cc = c & 7;
                const bool in = c < rowc;
                const unsigned char *src = a.qcast + (in ? ((size_t)cqi[r] * d * ESZ + (size_t)c * 16) : 0);
                cp_async16(Bb + (size_t)kc * TN * 128 + (size_t)(r >> 3) * 1024 + (r & 7) * 128 +
                               ((cc ^ (r & 7)) << 4),
                           src, in ? 16u : 0u);
            }
            cp_async_wait_all();
            fence_proxy_async_smem();  // B is read by the tensor cores (async proxy)
            mbar_arrive(&bfull[bb]);
        }
    } else if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            uint32_t g = 0;
            const uint32_t pay_bytes = (uint32_t)(C * d * ESZ);
            for (int it = 0;; ++it) {
                const int j = it % TC_CTX;
                if (!mbar_wait_ab(&cfull[j], (uint32_t)(it / TC_CTX) & 1, a.err, s_abort, a.wait_ns)) break;
                const int32_t *h = hdr(j);
                if (h[8] & CF_STOP) break;
                const int sns = h[3], nblk = h[4];
                const int32_t *sl = c_sl(j);
                bool ab = false;
                for (int b = 0; b < nblk; ++b, ++g) {
                    const uint32_t st = g % NST, u = g / NST;
                    if (u >= 1 && !mbar_wait_ab(&empty[st], (u - 1) & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    const int nsl = min(SPB, sns - b * SPB);
                    int okc = 0;
                    for (int jj = 0; jj < nsl; ++jj) okc += sl[b * SPB + jj] >= 0;
                    mbar_arrive_expect_tx(&full[st], (uint32_t)(okc * KC * C * 128));
                    // a whole tile of consecutive slabs s0 .. s0 + SPB - 1 is one
                    // 128-row box (the same bytes, the same swizzled layout)
                    auto consecutive = [&](int bb, int ns) {
                        const int s0 = sl[bb * SPB];
                        bool r = a.tile_box && ns == SPB && s0 >= 0;
                        for (int jj = 1; jj < ns && r; ++jj) r = sl[bb * SPB + jj] == s0 + jj;
                        return r;
                    };
                    if (consecutive(b, nsl)) {
                        const int s0 = sl[b * SPB];
                        for (int kc = 0; kc < KC; ++kc)
                            tma_load_2d(A + (size_t)st * KC * TC_M * 128 + (size_t)kc * TC_M * 128,
                                        &tmap_t, kc * EPC, s0 * C, &full[st]);
                    } else {
                        for (int jj = 0; jj < nsl; ++jj) {
                            const int s = sl[b * SPB + jj];
                            if (s < 0) continue;
                            for (int kc = 0; kc < KC; ++kc)
                                tma_load_2d(A + (size_t)st * KC * TC_M * 128 +
                                                (size_t)kc * TC_M * 128 + (size_t)jj * C * 128,
                                            &tmap, kc * EPC, s * C, &full[st]);
                        }
                    }
                    const int bp = b + a.pf_tiles;  // keep the L2 prefetch ahead
                    if (bp < nblk) {
                        const int nsp = min(SPB, sns - bp * SPB);
                        if (consecutive(bp, nsp)) {
                            const int s0 = sl[bp * SPB];
                            prefetch_l2(a.pay + (size_t)s0 * pay_bytes, (uint32_t)(SPB * pay_bytes));
                            prefetch_l2(a.xnorm + (size_t)s0 * C, (uint32_t)(SPB * C * 4));
                        } else {
                            for (int jj = 0; jj < nsp; ++jj) {
                                const int s = sl[bp * SPB + jj];
                                if (s < 0) continue;
                                prefetch_l2(a.pay + (size_t)s * pay_bytes, pay_bytes);
                                prefetch_l2(a.xnorm + (size_t)s * C, (uint32_t)(C * 4));
                            }
                        }
                    }
                }
                if (ab) break;
            }
            // the copies of the last tiles issued have landed before exit
            for (uint32_t t = g > (uint32_t)NST ? g - NST : 0; t < g; ++t)
                mbar_wait_bounded(&full[t % NST], (t / NST) & 1, a.err);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            uint32_t g = 0;
            for (int it = 0;; ++it) {
                const int j = it % TC_CTX, bb = it & 1;
                if (!mbar_wait_ab(&cfull[j], (uint32_t)(it / TC_CTX) & 1, a.err, s_abort, a.wait_ns)) break;
                if (hdr(j)[8] & CF_STOP) break;
                const int nblk = hdr(j)[4];
                if (!mbar_wait_ab(&bfull[bb], (uint32_t)(it >> 1) & 1, a.err, s_abort, a.wait_ns)) break;
                const uint32_t bbase = smem_u32(B + (size_t)bb * KC * TN * 128);
                bool ab = false;
                for (int b = 0; b < nblk; ++b, ++g) {
                    const uint32_t st = g % NST, u = g / NST, buf = g & 1, ub = g >> 1;
                    if (!mbar_wait_ab(&full[st], u & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    if (ub >= 1 && !mbar_wait_ab(&tempty[buf], (ub - 1) & 1, a.err, s_abort, a.wait_ns)) {
                        ab = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t abase = smem_u32(A + (size_t)st * KC * TC_M * 128);
                    for (int kc = 0; kc < KC; ++kc)
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = smem_desc_sw128(abase + kc * TC_M * 128 + ks * 32, 1024);
                            const uint64_t bd = smem_desc_sw128(bbase + kc * TN * 128 + ks * 32, 1024);
                            const uint32_t acc = (kc | ks) != 0;
                            if (DT == 0) mma_bf16(tbase + buf * TB, ad, bd, idesc, acc);
                            else mma_fp8(tbase + buf * TB, ad, bd, idesc, acc);
                        }
                    mma_commit(&tfull[buf]);
                    mma_commit(&empty[st]);
                }
                if (ab) break;
                mma_commit(&bfree[bb]);
            }
            // the last accumulator is written before TMEM is released
            if (g > 0) mbar_wait_bounded(&tfull[(g - 1) & 1], ((g - 1) >> 1) & 1, a.err);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---- epilogue
        const int ew = warp - 4;             // epilogue warp
        const int qt = ew & 3;               // its TMEM lane quarter (warp % 4)
        const int c0 = (ew >> 2) * TC_NCOL;  // its first query column
        const int et = ew * 32 + lane;       // epilogue thread
        const int v = qt * 32 + lane;        // A row = vector of the tile
        uint32_t *hist = Hist + ew * TC_HIST;
        uint32_t g = 0;
        for (int it = 0;; ++it) {
            const int j = it % TC_CTX;
            const bool ok = mbar_wait_ab(&cfull[j], (uint32_t)(it / TC_CTX) & 1, a.err, s_abort, a.wait_ns);
            if (!named_bar_and(1, EPI, ok && !*s_abort)) break;
            const int32_t *h = hdr(j);
            const int flags = h[8];
            if (flags & CF_STOP) break;
            const int m = h[1], sns = h[3], nblk = h[4], ME = h[5], chunk = h[7];
            const float inv_l = __int_as_float(h[9]);
            // a row holds [0, nb) (at most RK) and appends at RK; its pending
            // candidates are folded once a tile leaves more than FT of them:
            // FT plus one tile always fits.  A fold keeps K' .. Kw.  For
            // K' <= 128, past 224 pending rows a fold costs more than the
            // extra folds that a lower trigger brings (measured at K' = 40:
            // 224 beats 256, 192 and 160); deeper sets fold only when the
            // room is full (the held K' dominate a fold's cost)
            const int RK = a.RK, Kw = K + ((RK - K) >> 1);
            const int FT = min(ME - RK, K > 128 ? ME - RK : 224) - TC_M;
            const int32_t *qp = c_qpair(j);
            const float *cqn = c_qn(j), *cqsc = c_qsc(j), *ckd = c_kd0(j);
            const int32_t *sl = c_sl(j);
            const uint32_t *bt = c_bits(j);
            if (flags & CF_FIRST) {
                for (int r = et; r < TN; r += EPI) {
                    const bool on = r < m;
                    s_cnt[r] = 0;
                    s_nb[r] = 0;
                    s_kd[r] = on ? ckd[r] : INFINITY;
                    s_t[r] = on ? ckd[r] - cqn[r] : -INFINITY;
                    s_sc[r] = DT == 0 ? 2.f : 2.f / (inv_l * cqsc[r]);
                }
            }
            named_bar_sync(1, EPI);
            bool run = true;
            // this thread's row's slab in A tile bb of the item, and that
            // row's ||x||^2 read one tile ahead (its L2 latency hides behind
            // the tile before)
            auto row_slab = [&](int bb) {
                return v / C < min(SPB, sns - bb * SPB) ? sl[bb * SPB + v / C] : -1;
            };
            const int s_first = nblk > 0 ? row_slab(0) : -1;
            float xn_next = s_first >= 0 ? __ldg(a.xnorm + (size_t)s_first * C + v % C) : 0.f;
            for (int b = 0; b < nblk; ++b, ++g) {
                const uint32_t buf = g & 1, ub = g >> 1;
                // row of this thread in the tile
                const int nsl = min(SPB, sns - b * SPB);
                const int jr = v / C, slot = v % C, mi = b * SPB + jr;
                const int s = jr < nsl ? sl[mi] : -1;
                const bool live = s >= 0 && ((bt[mi * 4 + (slot >> 5)] >> (slot & 31)) & 1u);
                const int32_t gslot = s * C + slot;
                const float xn = xn_next;
                if (b + 1 < nblk) {
                    const int s2 = row_slab(b + 1);
                    xn_next = s2 >= 0 ? __ldg(a.xnorm + (size_t)s2 * C + slot) : 0.f;
                }
                bool wok = mbar_wait_ab(&tfull[buf], ub & 1, a.err, s_abort, a.wait_ns);
                wok = __all_sync(0xffffffffu, wok);  // tcgen05.ld is warp-aligned
                tc_fence_after();
                const bool cols = c0 < m;           // warp-uniform
                float dv[TC_NCOL];
                if (wok && cols) {
                    tmem_ld16(tbase + buf * TB + c0 + ((uint32_t)(qt * 32) << 16), dv);
                    tmem_ld_wait();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);

                // a row passes for query n when -s q.x + ||x||^2 <= kd_n - ||q_n||^2:
                // the 16 ballots first (independent), then, only if a row
                // passed, lane i reserves column i's buffer positions with one
                // shared atomic and the passing rows are written
                bool need = false;
                if (wok && cols) {
                    uint32_t mk[TC_NCOL];
                    const float4 *t4 = reinterpret_cast<const float4 *>(s_t + c0);
                    const float4 *sc4 = reinterpret_cast<const float4 *>(s_sc + c0);
#pragma unroll
                    for (int i4 = 0; i4 < TC_NCOL / 4; ++i4) {
                        const float4 tv = t4[i4];
                        const float tt[4] = {tv.x, tv.y, tv.z, tv.w};
                        float sc[4] = {2.f, 2.f, 2.f, 2.f};
                        if (DT == 1) {
                            const float4 sv = sc4[i4];
                            sc[0] = sv.x;
                            sc[1] = sv.y;
                            sc[2] = sv.z;
                            sc[3] = sv.w;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int i = 4 * i4 + c;
                            const float part = fmaf(-sc[c], dv[i], xn);
                            mk[i] = __ballot_sync(0xffffffffu, live && c0 + i < m && part <= tt[c]);
                        }
                    }
                    uint32_t any = 0u;
#pragma unroll
                    for (int i = 0; i < TC_NCOL; ++i) any |= mk[i];
                    if (any) {
                        uint32_t my = 0u;
#pragma unroll
                        for (int i = 0; i < TC_NCOL; ++i)
                            if (lane == i) my = mk[i];
                        int mybase = 0;
                        if (my) {
                            mybase = atomicAdd(&s_cnt[c0 + lane], __popc(my));
                            need = mybase + __popc(my) > FT;
                        }
#pragma unroll
                        for (int i = 0; i < TC_NCOL; ++i) {
                            if (!mk[i]) continue;
                            const int n = c0 + i;
                            const int base = __shfl_sync(0xffffffffu, mybase, i);
                            if ((mk[i] >> lane) & 1u) {
                                const int p = RK + base + __popc(mk[i] & lanemask_lt());
                                BD[(size_t)n * ME + p] = fmaf(-s_sc[n], dv[i], cqn[n] + xn);
                                BS[(size_t)n * ME + p] = gslot;
                            }
                        }
                    }
                }
                if (named_bar_or(1, EPI, need || !wok || *s_abort)) {
                    run = named_bar_and(1, EPI, wok && !*s_abort);
                    if (!run) break;
                    // fold the rows whose pending candidates passed FT
                    for (int n = ew; n < m; n += EW) {
                        const int cc = s_cnt[n];
                        if (cc <= FT) continue;
                        int nb = s_nb[n];
                        const float kd = fold_row(BD + (size_t)n * ME, BS + (size_t)n * ME, K, Kw,
                                                  RK, nb, cc, hist, lane);
                        if (lane == 0) {
                            s_nb[n] = nb;
                            s_cnt[n] = 0;
                            if (kd < s_kd[n]) {
                                s_kd[n] = kd;
                                s_t[n] = kd - cqn[n];
                            }
                        }
                        __syncwarp();
                    }
                    named_bar_sync(1, EPI);
                }
            }
            if (!run) {
                if (et == 0) *s_abort = 1;
                break;
            }
            if (flags & CF_LAST) {
                // each row's run: between K' and RK of its smallest
                // candidates (all of them when fewer), unsorted, with their
                // count (the per-query merge selects and sorts the best K');
                // a bound on its K'-th distance becomes a bound of the query
                // for the items that follow
                named_bar_sync(1, EPI);
                for (int n = ew; n < m; n += EW) {
                    const int cc = s_cnt[n];
                    int nb = s_nb[n];
                    float *bd = BD + (size_t)n * ME;
                    int32_t *bs = BS + (size_t)n * ME;
                    float kd = s_kd[n];
                    if (cc > 0) kd = fminf(kd, fold_row(bd, bs, K, RK, RK, nb, cc, hist, lane));
                    const int run = a.seed_slabs > 0 ? -1 : a.prun[qp[n]];
                    const int64_t base = ((int64_t)run + chunk) * RK;
                    for (int i = lane; i < nb && run >= 0; i += 32) {
                        a.part_d[base + i] = bd[i];
                        a.part_i[base + i] = (int64_t)bs[i];
                    }
                    if (lane == 0 && run >= 0) a.part_n[run + chunk] = nb;
                    if (lane == 0 && kd >= 0.f && kd < INFINITY)
                        atomicMin(reinterpret_cast<int *>(a.thr) + qp[n] / a.P, __float_as_int(kd));
                    __syncwarp();
                }
            }
            named_bar_sync(1, EPI);
            if (lane == 0) mbar_arrive(&cempty[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tbase, 2 * TB);
}

// ------------------------------------------------------- per-query merge
// One warp per query: the best K' (distance, slot) of the query's item
// outputs (runs of RK entries of which the first part_n[run] are valid,
// unsorted; the runs of one scan phase are contiguous, qrun[phase][q] =
// (first run, runs)) by a radix select over the 64-bit (distance, slot)
// keys of the valid entries, then sorted ascending, padded with (+inf, -1).
constexpr int MT_NT = 128;
// The selection of one query (one warp): its best K' valid entries, unsorted,
// into sd / ss (32 E entries of the warp's shared memory); returns their
// number, min(valid entries, K').  hist: TC_HIST words of shared memory.
template <int E>
__device__ int merge_select(const int2 *__restrict__ qrun, int64_t nq, int64_t q, int nphase,
                            int K, int RK, const int32_t *__restrict__ part_n,
                            const float *__restrict__ part_d, const int64_t *__restrict__ part_i,
                            uint32_t *hist, float *sd, int32_t *ss, int lane)
{
    const int2 r0 = qrun[q];
    const int2 r1 = nphase > 1 ? qrun[nq + q] : make_int2(0, 0);
    const int NR = r0.y + r1.y;
    auto run_of = [&](int t) -> int64_t { return t < r0.y ? r0.x + t : r1.x + (t - r0.y); };
    auto key_at = [&](int64_t e) -> uint64_t { return ds_key(part_d[e], (int32_t)part_i[e]); };
    // visit every valid entry: f(valid, index) for 32 entries at a time,
    // called by the whole warp (the loops are warp-uniform)
    auto each = [&](auto f) {
        for (int t = 0; t < NR; ++t) {
            const int64_t rb = run_of(t);
            const int c = min(part_n[rb], RK);
            for (int j0 = 0; j0 < c; j0 += 32) f(j0 + lane < c, rb * RK + j0 + lane);
        }
    };
    int nv = 0;
    for (int t = lane; t < NR; t += 32) nv += min(part_n[run_of(t)], RK);
    for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    uint64_t prefix = ~0ull, mask = 0ull;  // keep every valid entry
    if (nv > K) {
        // radix select: 8 bits per pass from the highest bit where the keys
        // differ, stopping at the first pass whose chosen bin is taken whole
        uint64_t kmin = ~0ull, kmax = 0ull;
        each([&](bool ok, int64_t e) {
            if (ok) {
                const uint64_t k = key_at(e);
                kmin = min(kmin, k);
                kmax = max(kmax, k);
            }
        });
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmin, o));
            kmax = max(kmax, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmax, o));
        }
        const uint64_t diff = kmin ^ kmax;
        const int top = diff ? 63 - __clzll((long long)diff) : 0;
        mask = top >= 63 ? 0ull : ~((2ull << top) - 1ull);
        prefix = kmin & mask;
        uint32_t need = (uint32_t)K;
        for (int hi = top; hi >= 0; hi -= 8) {
            const int shift = max(hi - 7, 0);
            const uint32_t bmask = (1u << (hi - shift + 1)) - 1u;
#pragma unroll
            for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0u;
            __syncwarp();
            each([&](bool ok, int64_t e) {
                if (ok) {
                    const uint64_t k = key_at(e);
                    if ((k & mask) == prefix) atomicAdd(&hist[(uint32_t)(k >> shift) & bmask], 1u);
                }
            });
            __syncwarp();
            uint32_t loc[8], sum = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                loc[b] = hist[lane * 8 + b];
                sum += loc[b];
            }
            uint32_t incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t tv = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += tv;
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
    }
    int w = 0;
    each([&](bool ok, int64_t e) {
        bool take = false;
        float dv = 0.f;
        int32_t sv = 0;
        if (ok) {
            dv = part_d[e];
            sv = (int32_t)part_i[e];
            take = (ds_key(dv, sv) & mask) <= prefix;
        }
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        if (take) {
            const int p = w + __popc(mk & lanemask_lt());
            if (p < 32 * E) {
                sd[p] = dv;
                ss[p] = sv;
            }
        }
        w += __popc(mk);
    });
    __syncwarp();
    return min(w, K);
}

template <int E>
__global__ __launch_bounds__(MT_NT) void k_merge_tc(const int2 *__restrict__ qrun, int64_t nq,
                                                    int nphase, int K, int RK,
                                                    const int32_t *__restrict__ part_n,
                                                    const float *__restrict__ part_d,
                                                    const int64_t *__restrict__ part_i,
                                                    float *__restrict__ out_d,
                                                    int64_t *__restrict__ out_s)
{
    pdl_begin();
    constexpr int NW = MT_NT / 32;
    __shared__ uint32_t hist_s[NW][TC_HIST];
    __shared__ float sd[NW][32 * E];
    __shared__ int32_t ss[NW][32 * E];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)MT_NT + threadIdx.x) >> 5;
    if (q >= nq) return;  // whole warps
    uint32_t *hist = hist_s[warp];
    const int nk = merge_select<E>(qrun, nq, q, nphase, K, RK, part_n, part_d, part_i, hist,
                                   sd[warp], ss[warp], lane);
    float v[E];
    int32_t sv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        v[e] = i < nk ? sd[warp][i] : INFINITY;
        sv[e] = i < nk ? ss[warp][i] : 0x7fffffff;
    }
    warp_sort32<E>(v, sv, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < K) {
            out_d[q * K + i] = i < nk ? v[e] : INFINITY;
            out_s[q * K + i] = i < nk ? (int64_t)sv[e] : -1;
        }
    }
}

void merge_tc(sivf_index *ix, int64_t nq, int nphase, const SearchScratch &s, int Kc, int RK,
              float *out_d, int64_t *out_s, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((nq * 32 + MT_NT - 1) / MT_NT);
    const int tok = prof_begin(ix, PROF_MERGE, 1, st);
#define SIVF_MTC(E_)                                                                               \
    launch_pdl(k_merge_tc<E_>, blocks, MT_NT, 0, st, s.qrun, nq, nphase, Kc, RK, s.part_n,         \
               s.part_d, s.part_i, out_d, out_s)
    if (Kc <= 32) SIVF_MTC(1);
    else if (Kc <= 64) SIVF_MTC(2);
    else if (Kc <= 128) SIVF_MTC(4);
    else if (Kc <= 256) SIVF_MTC(8);
    else SIVF_MTC(16);
#undef SIVF_MTC
    prof_end(ix, tok, st);
}

// ---------------------------------------------------------------- re-rank
// One warp per query: exact FP32 direct-form distances of the K' merged
// candidates (global slots) from the FP32 payload, then the best k by
// (distance, id).  Eight lanes share a candidate row: lane t of a group
// holds query chunks t, t + 8, ... (16 bytes each) in registers and reads
// the same chunks of the row, so one load instruction of the warp covers
// four whole 128-byte lines; RK_UNR rounds of four candidates are loaded
// before any is reduced (the group's partial sums meet by shuffles).  The
// candidates' slots are staged in shared memory first; their ids are read
// into the owning lanes' registers then and used only by the sort.
constexpr int RK_NT = 128;
constexpr int RK_UNR = 4;  // measured best of 2, 4, 5, 8 and 10
template <int E, int NQ>  // E: candidates per lane in the sort; NQ: chunks per lane (d <= 32 NQ)
__global__ __launch_bounds__(RK_NT) void k_rerank(const float *__restrict__ q, int64_t nq, int d,
                                                int Kc, const float *__restrict__ cand_d,
                                                const int64_t *__restrict__ cand_s,
                                                const float *__restrict__ x32,
                                                const int64_t *__restrict__ ids, int k,
                                                float *__restrict__ dist, int64_t *__restrict__ labels)
{
    pdl_begin();
    __shared__ int64_t sgs[RK_NT / 32][32 * E];
    __shared__ float sd[RK_NT / 32][32 * E];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 3, t = lane & 7;
    const int64_t qi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (qi >= nq) return;  // whole warps
    const int n4 = d >> 2;
    // candidate slots (-1: none); ids into registers, read by the sort
    int64_t id[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        int64_t gs = -1;
        if (c < Kc) {
            gs = cand_s[qi * Kc + c];
            if (!(cand_d[qi * Kc + c] < INFINITY)) gs = -1;
        }
        sgs[w][c] = gs;
        id[e] = gs >= 0 ? __ldg(ids + gs) : -1;
    }
    const float4 *q4 = reinterpret_cast<const float4 *>(q + (size_t)qi * d);
    float4 qv[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u)
        qv[u] = t + 8 * u < n4 ? __ldg(q4 + t + 8 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    const float4 *x4 = reinterpret_cast<const float4 *>(x32);
    for (int c0 = 0; c0 < Kc; c0 += 4 * RK_UNR) {
        float4 xv[RK_UNR][NQ];
        int64_t gs[RK_UNR];
#pragma unroll
        for (int r = 0; r < RK_UNR; ++r) {
            const int c = c0 + 4 * r + g;
            gs[r] = c < Kc ? sgs[w][c] : -1;
#pragma unroll
            for (int u = 0; u < NQ; ++u)
                xv[r][u] = gs[r] >= 0 && t + 8 * u < n4 ? __ldg(x4 + gs[r] * n4 + t + 8 * u)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < RK_UNR; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                float dd = qv[u].x - xv[r][u].x;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].y - xv[r][u].y;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].z - xv[r][u].z;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].w - xv[r][u].w;
                acc = fmaf(dd, dd, acc);
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            const int c = c0 + 4 * r + g;
            if (t == 0 && c < Kc) sd[w][c] = gs[r] >= 0 ? acc : INFINITY;
        }
    }
    __syncwarp();
    float v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        v[e] = c < Kc && id[e] >= 0 ? sd[w][c] : INFINITY;
    }
    warp_bitonic_sort<E>(v, id, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < k) {
            dist[qi * k + i] = id[e] >= 0 ? v[e] : INFINITY;
            labels[qi * k + i] = id[e];
        }
    }
}

// The per-query merge and the re-rank in one warp per query (K' <= 128):
// merge_select leaves the query's best K' (distance, slot) entries in shared
// memory, and the warp re-ranks those slots exactly as k_rerank does (eight
// lanes per candidate row, RK_UNR rounds of four, the query in registers),
// so the candidate lists never go through global memory and nothing sorts
// them by approximate distance.
// rounds of four candidate rows per warp batch of the re-ranks that run with
// more resident warps (fused merge + re-rank, wide re-rank)
constexpr int RR_UNR = 2;
// d <= 128: nine blocks of four warps per SM (at most 56 registers, no
// spills), 5,472 resident warps, so 10,000 queries take two waves instead of
// the three of eight blocks (0.062 -> 0.052 ms, same results)
template <int E, int NQ>
__global__ __launch_bounds__(MT_NT, NQ <= 4 ? 9 : 2) void k_merge_rerank(
    const int2 *__restrict__ qrun, int64_t nq, int nphase, int K, int RK,
    const int32_t *__restrict__ part_n, const float *__restrict__ part_d,
    const int64_t *__restrict__ part_i, const float *__restrict__ q, int d,
    const float *__restrict__ x32, const int64_t *__restrict__ ids, int k,
    float *__restrict__ dist, int64_t *__restrict__ labels)
{
    pdl_begin();
    constexpr int NW = MT_NT / 32;
    __shared__ uint32_t hist_s[NW][TC_HIST];
    __shared__ float sd[NW][32 * E];
    __shared__ int32_t ss[NW][32 * E];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 3, t = lane & 7;
    const int64_t qi = (blockIdx.x * (int64_t)MT_NT + threadIdx.x) >> 5;
    if (qi >= nq) return;  // whole warps
    const int nk = merge_select<E>(qrun, nq, qi, nphase, K, RK, part_n, part_d, part_i,
                                   hist_s[warp], sd[warp], ss[warp], lane);
    int64_t id[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        id[e] = c < nk ? __ldg(ids + ss[warp][c]) : -1;
    }
    const int n4 = d >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(q + (size_t)qi * d);
    float4 qv[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u)
        qv[u] = t + 8 * u < n4 ? __ldg(q4 + t + 8 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 *x4 = reinterpret_cast<const float4 *>(x32);
    for (int c0 = 0; c0 < nk; c0 += 4 * RR_UNR) {
        float4 xv[RR_UNR][NQ];
        int64_t gs[RR_UNR];
#pragma unroll
        for (int r = 0; r < RR_UNR; ++r) {
            const int c = c0 + 4 * r + g;
            gs[r] = c < nk ? (int64_t)ss[warp][c] : -1;
#pragma unroll
            for (int u = 0; u < NQ; ++u)
                xv[r][u] = gs[r] >= 0 && t + 8 * u < n4 ? __ldg(x4 + gs[r] * n4 + t + 8 * u)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < RR_UNR; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                float dd = qv[u].x - xv[r][u].x;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].y - xv[r][u].y;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].z - xv[r][u].z;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].w - xv[r][u].w;
                acc = fmaf(dd, dd, acc);
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            const int c = c0 + 4 * r + g;
            __syncwarp();
            if (t == 0 && c < nk) sd[warp][c] = acc;  // the approximate distance is no longer needed
        }
    }
    __syncwarp();
    float v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        v[e] = c < nk ? sd[warp][c] : INFINITY;
    }
    warp_bitonic_sort<E>(v, id, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < k) {
            dist[qi * k + i] = id[e] >= 0 ? v[e] : INFINITY;
            labels[qi * k + i] = id[e];
        }
    }
}

// Deep re-rank (K' up to 512): one block per query; its warps compute the
// candidates' exact FP32 direct-form distances into shared memory (eight
// lanes per candidate row with 16-byte loads, RR_UNR rounds of four rows
// per warp loaded before they are reduced, the query in registers), then
// the block sorts them by (distance, id) with a bitonic network and writes
// the best k.  Two rounds per batch keep the registers low enough for four
// blocks per SM: the gather is bound by loads in flight, i.e. by resident
// warps.
constexpr int RR_NT = 256;
constexpr int RR_MAX = 512;
template <int NQ>  // 16-byte chunks of the row per lane (d <= 32 NQ)
__global__ __launch_bounds__(RR_NT, NQ <= 4 ? 4 : 1) void k_rerank_wide(const float *__restrict__ q, int64_t nq,
                                                       int d, int Kc,
                                                       const float *__restrict__ cand_d,
                                                       const int64_t *__restrict__ cand_s,
                                                       const float *__restrict__ x32,
                                                       const int64_t *__restrict__ ids, int k,
                                                       float *__restrict__ dist,
                                                       int64_t *__restrict__ labels)
{
    pdl_begin();
    __shared__ float sd[RR_MAX];
    __shared__ int64_t si[RR_MAX];
    const int64_t qi = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 3, t = lane & 7;
    const int64_t PAD = 0x7fffffffffffffffLL;  // pads sort after every id
    int N = 32;
    while (N < Kc) N <<= 1;
    const int n4 = d >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(q + (size_t)qi * d);
    const float4 *x4 = reinterpret_cast<const float4 *>(x32);
    float4 qv[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u)
        qv[u] = t + 8 * u < n4 ? __ldg(q4 + t + 8 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
    constexpr int CPW = 4 * RR_UNR;  // candidates per warp and batch
    for (int c0 = warp * CPW; c0 < N; c0 += (RR_NT / 32) * CPW) {
        float4 xv[RR_UNR][NQ];
        int64_t gs[RR_UNR];
#pragma unroll
        for (int r = 0; r < RR_UNR; ++r) {
            const int c = c0 + 4 * r + g;
            gs[r] = -1;
            if (c < Kc) {
                const int64_t s0 = cand_s[qi * Kc + c];
                if (s0 >= 0 && cand_d[qi * Kc + c] < INFINITY) gs[r] = s0;
            }
#pragma unroll
            for (int u = 0; u < NQ; ++u)
                xv[r][u] = gs[r] >= 0 && t + 8 * u < n4 ? __ldg(x4 + gs[r] * n4 + t + 8 * u)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < RR_UNR; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                float dd = qv[u].x - xv[r][u].x;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].y - xv[r][u].y;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].z - xv[r][u].z;
                acc = fmaf(dd, dd, acc);
                dd = qv[u].w - xv[r][u].w;
                acc = fmaf(dd, dd, acc);
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            const int c = c0 + 4 * r + g;
            if (t == 0 && c < N) {
                sd[c] = gs[r] >= 0 ? acc : INFINITY;
                si[c] = gs[r] >= 0 ? __ldg(ids + gs[r]) : PAD;
            }
        }
    }
    __syncthreads();
    for (int size = 2; size <= N; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < N / 2; t += RR_NT) {
                const int i = 2 * t - (t & (stride - 1)), j = i + stride;
                const bool up = (i & size) == 0;
                const bool lt = dk_less(sd[j], si[j], sd[i], si[i]);
                if (lt == up) {
                    const float td = sd[i];
                    sd[i] = sd[j];
                    sd[j] = td;
                    const int64_t ti = si[i];
                    si[i] = si[j];
                    si[j] = ti;
                }
            }
            __syncthreads();
        }
    for (int i = tid; i < k; i += RR_NT) {
        const bool ok = i < N && si[i] != PAD;
        dist[qi * k + i] = ok ? sd[i] : INFINITY;
        labels[qi * k + i] = ok ? si[i] : -1;
    }
}

// per query (BF16 form): FP32 ||q||^2, unit scale, and the row rounded to
// BF16 (round to nearest even).  The FP8 form codes each (query, probe)
// pair instead (k_pair_prep).
__global__ void k_query_prep(const float *__restrict__ q, int64_t nq, int d,
                             float *__restrict__ qn, float *__restrict__ qsc,
                             unsigned char *__restrict__ qcast)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= nq) return;
    const float *qr = q + (size_t)i * d;
    float ss = 0.f;
    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(qcast) + (size_t)i * d;
    for (int j = lane; j < d; j += 32) {
        const float v = qr[j];
        ss = fmaf(v, v, ss);
        o[j] = __float2bfloat16_rn(v);
    }
    ss = warp_sum(ss);
    if (lane == 0) {
        qn[i] = ss;
        qsc[i] = 1.f;
    }
}

void query_prep(sivf_index *ix, const float *q, int64_t nq, float *qn, float *qsc,
                unsigned char *qcast, cudaStream_t st)
{
    ix->launches += 1;
    launch_pdl(k_query_prep, (unsigned)((nq * 32 + 255) / 256), 256, 0, st, q, nq, ix->d, qn, qsc,
               qcast);
}

// FP8 residual scan: per (query, probe) pair e = q * P + p with list l =
// probes[e]: the residual r = fl32(q - c_l), ||r||^2 (FP32), its inverse
// scale 448 / (2 max_j |r_j|) (1 when r = 0) and the row E4M3(fl32(r_j *
// scale)) (round to nearest even, saturated).  One warp per pair; pairs with
// no list are left untouched (they are never scanned).
constexpr int PP_V4 = 2;  // float4 of the residual per lane (d <= 256)
__global__ void k_pair_prep(const float *__restrict__ q, int64_t npairs, int P, int d, int L,
                            const int32_t *__restrict__ probes, const float *__restrict__ cent,
                            float *__restrict__ qn, float *__restrict__ qsc,
                            unsigned char *__restrict__ qcast)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (e >= npairs) return;
    const int l = probes[e];
    if (l < 0 || l >= L) return;
    const float *qr = q + (size_t)(e / P) * d;
    const float *cl = cent + (size_t)l * d;
    unsigned char *o = qcast + (size_t)e * d;
    float ss = 0.f, mx = 0.f;
    if ((d & 3) == 0 && d <= 32 * 4 * PP_V4) {
        // the residual held in registers, one float4 per lane and round
        const int n4 = d >> 2;
        float4 r4[PP_V4];
#pragma unroll
        for (int u = 0; u < PP_V4; ++u) {
            const int j4 = lane + 32 * u;
            r4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j4 < n4) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(qr) + j4);
                const float4 b = __ldg(reinterpret_cast<const float4 *>(cl) + j4);
                r4[u] = make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y),
                                    __fsub_rn(a.z, b.z), __fsub_rn(a.w, b.w));
            }
            ss = fmaf(r4[u].x, r4[u].x, ss);
            ss = fmaf(r4[u].y, r4[u].y, ss);
            ss = fmaf(r4[u].z, r4[u].z, ss);
            ss = fmaf(r4[u].w, r4[u].w, ss);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(r4[u].x), fabsf(r4[u].y)),
                                 fmaxf(fabsf(r4[u].z), fabsf(r4[u].w))));
        }
        ss = warp_sum(ss);
        for (int o2 = 16; o2 > 0; o2 >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
        const float sc = mx > 0.f ? 448.f / (2.f * mx) : 1.f;
        if (lane == 0) {
            qn[e] = ss;
            qsc[e] = sc;
        }
#pragma unroll
        for (int u = 0; u < PP_V4; ++u) {
            const int j4 = lane + 32 * u;
            if (j4 >= n4) break;
            const uint32_t lo = __nv_cvt_float2_to_fp8x2(
                make_float2(__fmul_rn(r4[u].x, sc), __fmul_rn(r4[u].y, sc)), __NV_SATFINITE, __NV_E4M3);
            const uint32_t hi = __nv_cvt_float2_to_fp8x2(
                make_float2(__fmul_rn(r4[u].z, sc), __fmul_rn(r4[u].w, sc)), __NV_SATFINITE, __NV_E4M3);
            reinterpret_cast<uint32_t *>(o)[j4] = (lo & 0xffffu) | (hi << 16);
        }
        return;
    }
    for (int j = lane; j < d; j += 32) {
        const float r = __fsub_rn(qr[j], cl[j]);
        ss = fmaf(r, r, ss);
        mx = fmaxf(mx, fabsf(r));
    }
    ss = warp_sum(ss);
    for (int o2 = 16; o2 > 0; o2 >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    const float sc = mx > 0.f ? 448.f / (2.f * mx) : 1.f;
    if (lane == 0) {
        qn[e] = ss;
        qsc[e] = sc;
    }
    for (int j = 2 * lane; j < d; j += 64) {
        const float2 p = make_float2(__fmul_rn(__fsub_rn(qr[j], cl[j]), sc),
                                     __fmul_rn(__fsub_rn(qr[j + 1], cl[j + 1]), sc));
        const uint32_t two = __nv_cvt_float2_to_fp8x2(p, __NV_SATFINITE, __NV_E4M3);
        o[j] = (unsigned char)(two & 0xffu);
        o[j + 1] = (unsigned char)(two >> 8);
    }
}

void pair_prep(sivf_index *ix, const float *q, int64_t nq, int P, const int32_t *probes,
               float *qn, float *qsc, unsigned char *qcast, cudaStream_t st)
{
    ix->launches += 1;
    const int64_t np = nq * P;
    launch_pdl(k_pair_prep, (unsigned)((np * 32 + 255) / 256), 256, 0, st, q, np, P, ix->d,
               ix->nlist, probes, ix->cent, qn, qsc, qcast);
}

// global slots -> labels (padding stays -1)
__global__ void k_slots_to_ids(int64_t *v, int64_t n, const int64_t *__restrict__ ids)
{
    pdl_begin();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (v[i] >= 0) v[i] = ids[v[i]];
}

void slots_to_ids(sivf_index *ix, int64_t *v, int64_t n, cudaStream_t st)
{
    ix->launches += 1;
    launch_pdl(k_slots_to_ids, (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0,
               st, v, n, ix->ids);
}

// --------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool tc_make_maps(sivf_index *ix)
{
    auto enc = tmap_encode_fn();
    if (!enc) return false;
    const cuuint64_t rows = (cuuint64_t)ix->n_slabs * ix->C;
    if (ix->xb16) {
        cuuint64_t dims[2] = {(cuuint64_t)ix->d, rows};
        cuuint64_t strides[1] = {(cuuint64_t)ix->d * 2};
        cuuint32_t box[2] = {64, (cuuint32_t)ix->C};
        cuuint32_t es[2] = {1, 1};
        if (enc(reinterpret_cast<CUtensorMap *>(ix->tmap_bf16), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                ix->xb16, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    if (ix->x8) {
        cuuint64_t dims[2] = {(cuuint64_t)ix->d, rows};
        cuuint64_t strides[1] = {(cuuint64_t)ix->d};
        cuuint32_t box[2] = {128, (cuuint32_t)ix->C};
        cuuint32_t es[2] = {1, 1};
        if (enc(reinterpret_cast<CUtensorMap *>(ix->tmap_fp8), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                ix->x8, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    // 128-row boxes for tiles whose slabs are consecutive in the pool
    ix->tmap_tile_ok = false;
    if (ix->C < TC_M && TC_M % ix->C == 0) {
        bool ok = true;
        if (ix->xb16) {
            cuuint64_t dims[2] = {(cuuint64_t)ix->d, rows};
            cuuint64_t strides[1] = {(cuuint64_t)ix->d * 2};
            cuuint32_t box[2] = {64, (cuuint32_t)TC_M};
            cuuint32_t es[2] = {1, 1};
            ok = ok && enc(reinterpret_cast<CUtensorMap *>(ix->tmap_bf16_t),
                           CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->xb16, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        }
        if (ix->x8) {
            cuuint64_t dims[2] = {(cuuint64_t)ix->d, rows};
            cuuint64_t strides[1] = {(cuuint64_t)ix->d};
            cuuint32_t box[2] = {128, (cuuint32_t)TC_M};
            cuuint32_t es[2] = {1, 1};
            ok = ok && enc(reinterpret_cast<CUtensorMap *>(ix->tmap_fp8_t),
                           CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ix->x8, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        }
        ix->tmap_tile_ok = ok;
    }
    return qt_make_maps(ix, enc);
}

// a row's run and held set: K' plus the room an approximate reduction may
// keep beyond it (a quarter of K', at least 32), a multiple of 8
int tc_run_len(int K) { return (K + max(32, K / 4) + 7) / 8 * 8; }

// a row's candidate buffer: its held set plus room for `tiles` tiles of
// candidates (TC_M each)
static int tc_buf_len(int K, int tiles) { return tc_run_len(K) + tiles * TC_M; }

// queries per tile of the reduced-precision scan for K' candidates
int tc_tile_queries(int Kc)
{
    return Kc <= TcShape<48>::KMAX ? 48 : Kc <= TcShape<32>::KMAX ? 32 : 16;
}

// dynamic shared memory one CTA may take (the kernel's static arrays aside)
constexpr size_t kTcSmemMax = 227 * 1024 - 4096;

template <int TN>
static int tc_stages(int KC, int M)
{
    int nst = TC_MAXST;
    while (nst > 2 && tc_smem<TN>(KC, M, nst).total > kTcSmemMax) --nst;
    return nst;
}

static size_t tc_total(int tn, int KC, int M, int nst)
{
    switch (tn) {
    case 48: return tc_smem<48>(KC, M, nst).total;
    case 32: return tc_smem<32>(KC, M, nst).total;
    default: return tc_smem<16>(KC, M, nst).total;
    }
}

// Entries of a row's candidate buffer.  A row folds its pending candidates
// into its best K' once more than (room - 1) tiles of them wait (for
// K' <= 128 also past 224), so with room for one tile any candidate at all
// costs a fold per tile; the default takes room for three tiles (K' > 128)
// or two where three A stages still fit beside it, else one.  sel > 0 asks
// for sel tiles of room.
int tc_buf_entries(const sivf_index *ix, int dtype, int Kc, int sel)
{
    if (sel > 0) return tc_buf_len(Kc, sel);
    const int esz = dtype == SIVF_BF16 ? 2 : 1;
    const int KC = (ix->d * esz + 127) / 128;
    const int tn = tc_tile_queries(Kc);
    // K' > 128: three tiles of room where they fit, so a fold (dominated by
    // the held K') comes every third tile while no bound prunes
    if (Kc > 128 && tc_total(tn, KC, tc_buf_len(Kc, 3), 3) <= kTcSmemMax)
        return tc_buf_len(Kc, 3);
    if (tc_total(tn, KC, tc_buf_len(Kc, 2), 3) <= kTcSmemMax) return tc_buf_len(Kc, 2);
    return tc_buf_len(Kc, 1);
}

// a buffer of M entries fits beside two A stages
bool tc_buf_fits(const sivf_index *ix, int dtype, int Kc, int M)
{
    const int esz = dtype == SIVF_BF16 ? 2 : 1;
    const int KC = (ix->d * esz + 127) / 128;
    const int tn = tc_tile_queries(Kc);
    return (tn != 16 || Kc <= TcShape<16>::KMAX) && tc_total(tn, KC, M, 2) <= kTcSmemMax;
}

int tc_wide_entries(const sivf_index *ix, int dtype, int Kc)
{
    if (Kc <= TcShape<32>::KMAX || Kc > TcShape<16>::KMAX) return 0;
    const int esz = dtype == SIVF_BF16 ? 2 : 1;
    const int KC = (ix->d * esz + 127) / 128;
    const int M = tc_buf_len(Kc, 1);
    return tc_smem<32>(KC, M, 2).total <= kTcSmemMax ? M : 0;
}

bool tc_fits(const sivf_index *ix, int Kc)
{
    const int esz = 2;  // the larger of the two formats
    const int KC = (ix->d * esz + 127) / 128;
    const int M = tc_buf_len(Kc, 1);
    switch (tc_tile_queries(Kc)) {
    case 48: return tc_smem<48>(KC, M, 2).total <= kTcSmemMax;
    case 32: return tc_smem<32>(KC, M, 2).total <= kTcSmemMax;
    default: return Kc <= TcShape<16>::KMAX && tc_smem<16>(KC, M, 2).total <= kTcSmemMax;
    }
}

template <int DT, int TN>
static void launch_tc(const unsigned char *tmap, const unsigned char *tmap_t, TcArgs a,
                      cudaStream_t st)
{
    a.nst = tc_stages<TN>(a.KC, a.M);
    const size_t smem = tc_smem<TN>(a.KC, a.M, a.nst).total;
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_scan_tc<DT, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = smem;
    }
    launch_pdl(k_scan_tc<DT, TN>, 152, TcShape<TN>::NT, smem, st,
               *reinterpret_cast<const CUtensorMap *>(tmap),
               *reinterpret_cast<const CUtensorMap *>(tmap_t), a);
}

void scan_lists_tc(sivf_index *ix, int dtype, const float *q, int64_t nq, int P, int Kc,
                   const SearchPlan &pl, const SearchScratch &s, cudaStream_t st, int seed_slabs)
{
    TcArgs a;
    a.q = q;
    a.nq = nq;
    a.P = P;
    a.K = Kc;
    a.M = pl.M;
    a.prun = s.prun;
    a.qlist = s.qlist;
    a.loff = s.loff;
    a.lcnt = s.lcnt;
    a.ibase = s.ibase;
    a.nch = s.nch;
    a.part_d = s.part_d;
    a.part_i = s.part_i;
    a.part_n = s.part_n;
    a.RK = pl.RK;
    a.thr = s.thr;
    a.items = s.items;
    a.per_pair = dtype == SIVF_FP8E4M3;
    a.qn = a.per_pair ? s.pqn : s.qn;
    a.qsc = a.per_pair ? s.pqsc : s.qsc;
    a.qcast = s.qcast;
    a.xnorm = a.per_pair ? ix->rnorm : ix->xnorm;
    a.bits = ix->bits;
    a.nslabs = ix->nslabs;
    a.dir = ix->dir;
    a.inv_scale8 = ix->inv_scale8;
    a.n_slabs = ix->n_slabs;
    a.dir_cap = ix->dir_cap;
    a.L = ix->nlist;
    a.d = ix->d;
    a.C = ix->C;
    const int esz = dtype == SIVF_BF16 ? 2 : 1;
    a.pay = dtype == SIVF_BF16 ? reinterpret_cast<const unsigned char *>(ix->xb16) : ix->x8;
    a.KC = (ix->d * esz + 127) / 128;
    a.nst = 2;
    a.pf_tiles = std::max(2, TC_PF_BYTES / (TC_M * ix->d * esz));
    a.tile_box = ix->tmap_tile_ok ? 1 : 0;
    a.ctl = ix->ctl;
    a.err = ix->err;
    a.seed_slabs = seed_slabs;
    a.wait_ns = ix->wait_ns;
    const int tn = pl.tq;  // the plan's tile: 48 / 32 / 16 (tc_tile_queries), 32 wide
    const int tok = prof_begin(ix, PROF_SCAN, 1, st);
    if (dtype == SIVF_BF16) {
        if (tn == 48) launch_tc<0, 48>(ix->tmap_bf16, ix->tmap_bf16_t, a, st);
        else if (tn == 32) launch_tc<0, 32>(ix->tmap_bf16, ix->tmap_bf16_t, a, st);
        else launch_tc<0, 16>(ix->tmap_bf16, ix->tmap_bf16_t, a, st);
    } else {
        if (tn == 48) launch_tc<1, 48>(ix->tmap_fp8, ix->tmap_fp8_t, a, st);
        else if (tn == 32) launch_tc<1, 32>(ix->tmap_fp8, ix->tmap_fp8_t, a, st);
        else launch_tc<1, 16>(ix->tmap_fp8, ix->tmap_fp8_t, a, st);
    }
    prof_end(ix, tok, st);
}

// merge and re-rank of a search: fused for K' <= 128 (d <= 256), else the
// merge into cand_d / cand_s followed by the wide re-rank
void merge_rerank(sivf_index *ix, const float *q, int64_t nq, int nphase,
                  const SearchScratch &s, int Kc, int RK, int k, float *cand_d,
                  int64_t *cand_s, float *dist, int64_t *labels, cudaStream_t st)
{
    if (Kc > 128) {
        merge_tc(ix, nq, nphase, s, Kc, RK, cand_d, cand_s, st);
        rerank(ix, q, nq, Kc, cand_d, cand_s, k, dist, labels, st);
        return;
    }
    const unsigned blocks = (unsigned)((nq * 32 + MT_NT - 1) / MT_NT);
    const int tok = prof_begin(ix, PROF_RERANK, 1, st);
#define SIVF_MRR(E_, NQ_)                                                                          \
    launch_pdl(k_merge_rerank<E_, NQ_>, blocks, MT_NT, 0, st, s.qrun, nq, nphase, Kc, RK,          \
               s.part_n, s.part_d, s.part_i, q, ix->d, ix->x32, ix->ids, k, dist,                  \
               labels)
    const bool wide = ix->d > 128;
    if (Kc <= 32) {
        if (wide) SIVF_MRR(1, 8);
        else SIVF_MRR(1, 4);
    } else if (Kc <= 64) {
        if (wide) SIVF_MRR(2, 8);
        else SIVF_MRR(2, 4);
    } else {
        if (wide) SIVF_MRR(4, 8);
        else SIVF_MRR(4, 4);
    }
#undef SIVF_MRR
    prof_end(ix, tok, st);
}

void rerank(sivf_index *ix, const float *q, int64_t nq, int Kc, const float *cand_d,
            const int64_t *cand_s, int k, float *dist, int64_t *labels, cudaStream_t st)
{
    const int64_t blocks = (nq * 32 + RK_NT - 1) / RK_NT;
    const int tok = prof_begin(ix, PROF_RERANK, 1, st);
#define SIVF_RERANK(E_, NQ_)                                                                       \
    launch_pdl(k_rerank<E_, NQ_>, (unsigned)blocks, RK_NT, 0, st, q, nq, ix->d, Kc, cand_d,        \
               cand_s, ix->x32, ix->ids, k, dist, labels)
    const bool wide = ix->d > 128;  // chunks per lane: 4 (d <= 128) or 8 (d <= 256)
    if (Kc <= 32) {
        if (wide) SIVF_RERANK(1, 8);
        else SIVF_RERANK(1, 4);
    } else if (Kc <= 64) {
        if (wide) SIVF_RERANK(2, 8);
        else SIVF_RERANK(2, 4);
    } else if (Kc <= 128) {
        if (wide) SIVF_RERANK(4, 8);
        else SIVF_RERANK(4, 4);
    } else {
        if (ix->d > 128)
            launch_pdl(k_rerank_wide<8>, (unsigned)nq, RR_NT, 0, st, q, nq, ix->d, Kc, cand_d,
                       cand_s, ix->x32, ix->ids, k, dist, labels);
        else
            launch_pdl(k_rerank_wide<4>, (unsigned)nq, RR_NT, 0, st, q, nq, ix->d, Kc, cand_d,
                       cand_s, ix->x32, ix->ids, k, dist, labels);
    }
#undef SIVF_RERANK
    prof_end(ix, tok, st);
}

}  // namespace sivf
