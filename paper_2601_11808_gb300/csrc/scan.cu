// List scan and top-k of the search (Algorithm 3, redone list-centrically).
//
// Algorithm 3 gives one warp to one query and walks each probed list's slab
// chain.  Here the (query, list) pairs of a whole batch are first grouped by
// list, and one CTA scans one list for a tile of up to TQ queries: every slab
// of the list is read from HBM once per tile instead of once per query, and
// the list's slabs come from its directory, so the next slabs are fetched
// (whole, by one bulk copy each, into shared memory) while the current one
// is being scored.  Distances are the direct form sum_j (q_j - x_j)^2 in
// FP32 (the paper's metric, squared L2).  A slot is read only when its
// validity bit is set (Theorem 2).  Each (query, list tile) keeps its best K
// (distance, id) pairs; a final merge per query keeps the best k of all
// probed lists, ties to the lower id, padded with (+inf, -1).
#include <math.h>

#include <cmath>

#include "device_utils.cuh"
#include "kernels.cuh"

namespace sivf {

// ------------------------------------------------------ grouping by list
// pairs (q, p) with p in [p0, p1): rank of each pair inside its list group
__global__ void k_srch_hist(const int32_t *__restrict__ probes, int64_t nq, int P, int p0,
                            int p1, int L, bool dedupe, int32_t *__restrict__ lcnt,
                            int32_t *__restrict__ prank)
{
    pdl_begin();
    const int np = p1 - p0;
    const int64_t n = nq * np;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = (t / np) * P + p0 + t % np;
        const int l = probes[e];
        bool ok = l >= 0 && l < L;
        if (ok && dedupe) {
            const int64_t q0 = (e / P) * P;
            for (int64_t f = q0; f < e; ++f)
                if (probes[f] == l) {
                    ok = false;
                    break;
                }
        }
        prank[e] = ok ? atomicAdd(&lcnt[l], 1) : -1;
    }
}

// One block.  Chunking: a list is cut into slab chunks so that no work item
// is longer than 1 / (ips * 152) of the launch's whole work W (query tiles x
// slabs summed over the probed lists) and no chunk is shorter than `spc`
// slabs, at most `chmax` chunks per list; a heavy list (a skewed
// distribution puts most vectors in a few lists) is spread over many SMs
// instead of holding one SM for the length of the launch.  With
// target = max(spc, ceil(W / (ips * 152))) the chunks beyond the first of
// every list add at most ips * 152 items, and at most tq * ips * 152 output
// runs, to one tile per pair: the scratch is sized from that bound.  Then
// exclusive scans over the lists of the pair counts and of the work items.
__global__ __launch_bounds__(1024) void k_srch_plan(const int32_t *__restrict__ lcnt,
                                                    const int32_t *__restrict__ nslabs,
                                                    const int32_t *__restrict__ list_live,
                                                    int L, int tq, int chmax, int spc, int ips,
                                                    int64_t item_cap, int64_t slab_bytes,
                                                    int32_t *__restrict__ loff,
                                                    int32_t *__restrict__ ibase,
                                                    int32_t *__restrict__ nch,
                                                    int2 *__restrict__ items, Ctl *ctl,
                                                    int64_t *stat, uint32_t *err)
{
    pdl_begin();
    __shared__ int32_t sa[1024], sb[1024];
    __shared__ unsigned long long sw[32];
    const int tid = threadIdx.x;
    const int per = (L + 1023) / 1024;
    const int b0 = tid * per, b1 = min(L, b0 + per);
    unsigned long long wsum = 0;
    for (int l = b0; l < b1; ++l) {
        const int m = lcnt[l], ns = nslabs[l];
        if (m > 0 && ns > 0) wsum += (unsigned long long)((m + tq - 1) / tq) * ns;
    }
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if ((tid & 31) == 0) sw[tid >> 5] = wsum;
    __syncthreads();
    unsigned long long W = 0;
    for (int i = 0; i < 32; ++i) W += sw[i];
    const unsigned long long slots = (unsigned long long)ips * 152;
    const unsigned long long share = (W + slots - 1) / slots;
    const int target = (int)min(max((unsigned long long)spc, share), 1ull << 30);
    int32_t ca = 0, cb = 0;
    unsigned long long pairs = 0, bytes = 0, ubytes = 0;
    for (int l = b0; l < b1; ++l) {
        int m = lcnt[l], ns = nslabs[l];
        int nt = (m + tq - 1) / tq;
        int c = (m > 0 && ns > 0) ? min(chmax, max(1, (ns + target - 1) / target)) : 0;
        c = min(c, ns);
        nch[l] = c;
        ca += m;
        cb += nt * c;
        if (c) {
            pairs += (unsigned long long)m * (unsigned long long)max(list_live[l], 0);
            bytes += (unsigned long long)nt * ns * slab_bytes;
            ubytes += (unsigned long long)ns * slab_bytes;
        }
    }
    if (stat && pairs) atomicAdd(reinterpret_cast<unsigned long long *>(stat + 1), pairs);
    if (stat && bytes) atomicAdd(reinterpret_cast<unsigned long long *>(stat + 2), bytes);
    if (stat && ubytes) atomicAdd(reinterpret_cast<unsigned long long *>(stat + 3), ubytes);
    sa[tid] = ca;
    sb[tid] = cb;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int32_t va = tid >= o ? sa[tid - o] : 0, vb = tid >= o ? sb[tid - o] : 0;
        __syncthreads();
        sa[tid] += va;
        sb[tid] += vb;
        __syncthreads();
    }
    int32_t ea = sa[tid] - ca, eb = sb[tid] - cb;
    for (int l = b0; l < b1; ++l) {
        const int m = lcnt[l], c = nch[l], nt = (m + tq - 1) / tq;
        loff[l] = ea;
        ibase[l] = eb;
        // work items of list l: (list, tile << 8 | chunk)
        for (int t = 0; t < nt * c; ++t) {
            if (eb + t < item_cap) items[eb + t] = make_int2(l, ((t / c) << 8) | (t % c));
        }
        ea += m;
        eb += nt * c;
    }
    if (tid == 1023) {
        loff[L] = sa[1023];
        ibase[L] = sb[1023];
        if (sb[1023] > item_cap) atomicOr(err, ERR_PLAN);
        ctl->nitems = (int32_t)min((int64_t)sb[1023], item_cap);
        ctl->nscan = sa[1023];
        ctl->next_item = 0;
    }
}

// One thread per query, whole warps together: each pair goes to its list's
// group (qlist), and the query's pairs of this phase reserve consecutive
// output runs (one per slab chunk of the pair's list; one atomic per warp).
__global__ void k_srch_scatter_t(const int32_t *__restrict__ probes, int64_t nq, int P, int p0,
                                 int p1, const int32_t *__restrict__ prank,
                                 const int32_t *__restrict__ loff, const int32_t *__restrict__ nch,
                                 int32_t *__restrict__ qlist, int32_t *__restrict__ prun,
                                 int2 *__restrict__ qrun, Ctl *ctl, int64_t run_cap,
                                 uint32_t *err)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); q0 < nq;
         q0 += stride) {
        const int64_t q = q0 + lane;
        int cnt = 0;
        if (q < nq)
            for (int p = p0; p < p1; ++p) {
                const int64_t e = q * P + p;
                const int r = prank[e];
                int c = 0;
                if (r >= 0) {
                    const int l = probes[e];
                    qlist[loff[l] + r] = (int32_t)e;
                    c = nch[l];
                }
                prun[e] = c;
                cnt += c;
            }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int base = 0;
        if (lane == 31) base = atomicAdd(&ctl->nruns, incl);
        base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
        if (q < nq) {
            const bool fits = base >= 0 && (int64_t)base + cnt <= run_cap;
            if (!fits) atomicOr(err, ERR_PLAN);
            int run = base;
            for (int p = p0; p < p1; ++p) {
                const int64_t e = q * P + p;
                const int c = prun[e];
                prun[e] = (c > 0 && fits) ? run : -1;
                run += c;
            }
            qrun[(p0 > 0 ? nq : 0) + q] = fits ? make_int2(base, cnt) : make_int2(0, 0);
        }
    }
}

// The same with one warp per query, SC_Q queries per block, for phases of
// many probes: the warp's lanes take the probes p0 + lane + 32 j, runs are
// assigned in probe order (one atomic per block).
// prun = the pair's first run (-1: not scanned); qrun[phase][q] = (first
// run, runs) of the query.  A reservation past run_cap (the plan's bound
// makes this impossible) sets ERR_PLAN and leaves the query's runs out.
constexpr int SC_Q = 8;
__global__ __launch_bounds__(SC_Q * 32) void k_srch_scatter(
    const int32_t *__restrict__ probes, int64_t nq, int P, int p0, int p1,
    const int32_t *__restrict__ prank, const int32_t *__restrict__ loff,
    const int32_t *__restrict__ nch, int32_t *__restrict__ qlist, int32_t *__restrict__ prun,
    int2 *__restrict__ qrun, Ctl *ctl, int64_t run_cap, uint32_t *err)
{
    pdl_begin();
    __shared__ int s_cnt[SC_Q];
    __shared__ int s_base;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t qb = (int64_t)blockIdx.x * SC_Q; qb < nq; qb += (int64_t)gridDim.x * SC_Q) {
        const int64_t q = qb + w;
        int cnt = 0;
        if (q < nq)
            for (int p = p0 + lane; p < p1; p += 32) {
                const int64_t e = q * P + p;
                const int r = prank[e];
                int c = 0;
                if (r >= 0) {
                    const int l = probes[e];
                    qlist[loff[l] + r] = (int32_t)e;
                    c = nch[l];
                }
                prun[e] = c;
                cnt += c;
            }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) s_cnt[w] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < SC_Q; ++k) tot += s_cnt[k];
            s_base = atomicAdd(&ctl->nruns, tot);
        }
        __syncthreads();
        int base = s_base;
        for (int k = 0; k < w; ++k) base += s_cnt[k];
        if (q < nq) {
            const bool fits = base >= 0 && (int64_t)base + cnt <= run_cap;
            if (!fits && lane == 0) atomicOr(err, ERR_PLAN);
            int run = base;
            for (int pb = p0; pb < p1; pb += 32) {  // warp-uniform
                const int p = pb + lane;
                const int64_t e = q * P + p;
                const int c = p < p1 ? prun[e] : 0;  // this lane's own count from above
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (p < p1) prun[e] = (c > 0 && fits) ? run + incl - c : -1;
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) qrun[(p0 > 0 ? nq : 0) + q] = fits ? make_int2(base, cnt) : make_int2(0, 0);
        }
        __syncthreads();  // s_cnt and s_base are reused by the next queries
    }
}

// ------------------------------------------------------------ the scan
constexpr int SCAN_NT = 256;
constexpr int NST = 2;  // slab stages in flight

struct ScanArgs {
    const float *q;
    int64_t nq;
    int P, K, M;
    const int32_t *qlist, *loff, *lcnt, *ibase, *nch;
    const int32_t *prun;  // first output run of each pair
    const int2 *items;
    float *part_d;
    int64_t *part_i;
    float *thr;          // [nq] shared upper bound of each query's k-th distance
    // index
    const float *x32;
    const int64_t *ids;
    const uint32_t *bits;
    const SlabMeta *meta;
    const int32_t *nslabs, *dir;
    int64_t n_slabs, dir_cap;
    int L, d;
    Ctl *ctl;
    uint32_t *err;
};

__host__ __device__ constexpr int scan_next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Entries per row of the best-K + candidate buffer: the best K, then room
// for two slabs of candidates (merged by rank, at most 256 entries); for
// larger K a power of two that the bitonic fallback can sort.
__host__ __device__ constexpr int scan_buf_len(int K, int C)
{
    return K + 2 * C <= 256 ? ((K + 2 * C + 15) & ~15) : scan_next_pow2(K + C);
}

// shared memory carve-up, identical on host and device
struct ScanSmem {
    size_t qs, xs, idb, bd, bi, misc, total;
};
__host__ __device__ inline ScanSmem scan_smem(int TQ, int C, int d, int M)
{
    ScanSmem s;
    const size_t DP = d + 4;
    s.qs = 0;
    s.xs = s.qs + (size_t)TQ * DP * 4;
    s.idb = s.xs + (size_t)NST * C * d * 4;
    s.bd = s.idb + (size_t)NST * C * 8;
    s.bi = s.bd + (size_t)TQ * M * 4;
    s.bi = (s.bi + 15) & ~(size_t)15;
    s.misc = s.bi + (size_t)TQ * M * 8;
    s.total = s.misc + 256;
    return s;
}

// Merge one query's candidates into its best list (one warp).  Every
// element of the union finds its rank by counting the elements that precede
// it in (distance, id) order -- candidates by a broadcast scan, best entries
// by binary search -- and then all elements land at once.  best[0, nb) is
// sorted, cand[K, K + nc) is not; ids are distinct, so ranks are too.
template <int EPL>
__device__ __forceinline__ void warp_rank_merge(float *bd, int64_t *bi, int K, int nb, int nc,
                                                int lane)
{
    const int n = nb + nc;
    float vd[EPL];
    int64_t vi[EPL];
    int pos[EPL];
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
        const int e = lane + 32 * t;
        pos[t] = K;
        if (e >= n) continue;
        const int src = e < nb ? e : K + (e - nb);
        const float dv = bd[src];
        const int64_t iv = bi[src];
        vd[t] = dv;
        vi[t] = iv;
        int r = 0;
        for (int j = 0; j < nc; ++j) r += dk_less(bd[K + j], bi[K + j], dv, iv);
        if (e < nb) {
            r += e;
        } else {
            int lo = 0, hi = nb;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (dk_less(bd[mid], bi[mid], dv, iv)) lo = mid + 1;
                else hi = mid;
            }
            r += lo;
        }
        pos[t] = r;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < EPL; ++t)
        if (pos[t] < K) {
            bd[pos[t]] = vd[t];
            bi[pos[t]] = vi[t];
        }
    __syncwarp();
}

// Fallback for large buffers: bitonic sort of all M entries (pads first).
__device__ void warp_bitonic_merge(float *bd, int64_t *bi, int K, int nb, int nc, int M,
                                   int lane)
{
    for (int e = nb + lane; e < K; e += 32) {
        bd[e] = INFINITY;
        bi[e] = -1;
    }
    for (int e = K + nc + lane; e < M; e += 32) {
        bd[e] = INFINITY;
        bi[e] = -1;
    }
    __syncwarp();
    for (int size = 2; size <= M; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < M / 2; t += 32) {
                const int pos = 2 * t - (t & (stride - 1));
                const int par = pos + stride;
                const bool up = (pos & size) == 0;
                const float d0 = bd[pos], d1 = bd[par];
                const int64_t i0 = bi[pos], i1 = bi[par];
                // pads (id -1) sort after every real entry
                const bool lt = (i1 >= 0 && i0 < 0) ||
                                (i1 >= 0 && i0 >= 0 && dk_less(d1, i1, d0, i0));
                if (lt == up) {
                    bd[pos] = d1;
                    bd[par] = d0;
                    bi[pos] = i1;
                    bi[par] = i0;
                }
            }
            __syncwarp();
        }
}

// Direct-form distances of the first RQA row groups of a thread's tile:
// acc[i][r] = sum_j (q_{i}[j] - x_{r}[j])^2, FP32, j in steps of 4.
template <int RQA, int RQ, int RX>
__device__ __forceinline__ void dist_tile(float (&acc)[RQ][RX], const float *__restrict__ qrow,
                                          const float *__restrict__ xrow, int d, int DP)
{
#pragma unroll
    for (int i = 0; i < RQA; ++i)
#pragma unroll
        for (int r = 0; r < RX; ++r) acc[i][r] = 0.f;
#pragma unroll 2
    for (int j = 0; j < d; j += 4) {
        float4 qv[RQA], xv[RX];
#pragma unroll
        for (int i = 0; i < RQA; ++i)
            qv[i] = *reinterpret_cast<const float4 *>(qrow + (size_t)i * 8 * DP + j);
#pragma unroll
        for (int r = 0; r < RX; ++r)
            xv[r] = *reinterpret_cast<const float4 *>(xrow + (size_t)r * 4 * d + j);
#pragma unroll
        for (int i = 0; i < RQA; ++i)
#pragma unroll
            for (int r = 0; r < RX; ++r) {
                const float t0 = qv[i].x - xv[r].x, t1 = qv[i].y - xv[r].y;
                const float t2 = qv[i].z - xv[r].z, t3 = qv[i].w - xv[r].w;
                float v = acc[i][r];
                v = fmaf(t0, t0, v);
                v = fmaf(t1, t1, v);
                v = fmaf(t2, t2, v);
                v = fmaf(t3, t3, v);
                acc[i][r] = v;
            }
    }
}

template <int TQ, int C>
__global__ __launch_bounds__(SCAN_NT, 1) void k_scan(ScanArgs a)
{
    pdl_begin();
    constexpr int QW = TQ >= 32 ? TQ / 32 : 1;
    constexpr int SW = 8 / QW;
    constexpr int RQ = TQ / (8 * QW);
    constexpr int RX = C / (4 * SW);
    constexpr int W = C / 32;
    static_assert(RQ >= 1 && RX >= 1, "tile shape");

    extern __shared__ __align__(128) unsigned char smem[];
    const int d = a.d, DP = d + 4, M = a.M, K = a.K;
    const int CB = M - K;  // candidate buffer capacity (>= C)
    const ScanSmem L = scan_smem(TQ, C, d, M);
    float *Qs = reinterpret_cast<float *>(smem + L.qs);
    float *Xs = reinterpret_cast<float *>(smem + L.xs);
    int64_t *IDs = reinterpret_cast<int64_t *>(smem + L.idb);
    float *BD = reinterpret_cast<float *>(smem + L.bd);
    int64_t *BI = reinterpret_cast<int64_t *>(smem + L.bi);
    unsigned char *misc = smem + L.misc;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(misc);  // [NST]
    int *s_item = reinterpret_cast<int *>(misc + 8 * NST);
    int *s_abort = s_item + 1;
    int *stage_slab = s_item + 2;                         // [NST]
    __shared__ int32_t s_qpair[TQ];   // (query, probe) pair of each row
    __shared__ int s_cc[TQ];          // candidates waiting per row
    __shared__ int s_nb[TQ];          // valid best entries per row
    __shared__ float s_kd[TQ];        // admission threshold per row
    __shared__ int64_t s_ki[TQ];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wq = warp % QW, ws = warp / QW;
    const int qy = lane & 7, sx = lane >> 3;
    const int64_t NOID = 0x7fffffffffffffffLL;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&mbar[s], 1);
        fence_mbar_init();
        *s_abort = 0;
    }
    __syncthreads();

    const uint32_t slab_bytes = (uint32_t)(C * d * 4);
    uint32_t g_cons = 0, g_issue = 0;  // slabs consumed / issued by this CTA

    auto issue = [&](int stage, int s) {
        // called by thread 0 only
        bool ok = s >= 0 && s < a.n_slabs;
        if (!ok) atomicOr(a.err, ERR_BAD_SLAB);
        stage_slab[stage] = ok ? s : -1;
        if (ok) {
            mbar_arrive_expect_tx(&mbar[stage], slab_bytes + C * 8);
            bulk_g2s(Xs + (size_t)stage * C * d, a.x32 + (size_t)s * C * d, slab_bytes,
                     &mbar[stage]);
            bulk_g2s(IDs + (size_t)stage * C, a.ids + (size_t)s * C, C * 8, &mbar[stage]);
        } else {
            mbar_arrive(&mbar[stage]);
        }
    };

    // merge the waiting candidates of row qr (one warp), then refresh the
    // row's threshold from its own K-th entry and the query's shared bound
    auto merge_row = [&](int qr) {
        float *bd = BD + (size_t)qr * M;
        int64_t *bi = BI + (size_t)qr * M;
        const int nb = s_nb[qr], nc = s_cc[qr];
        if (nc > 0) {
            if (nb + nc <= 128) warp_rank_merge<4>(bd, bi, K, nb, nc, lane);
            else if (nb + nc <= 256) warp_rank_merge<8>(bd, bi, K, nb, nc, lane);
            else warp_bitonic_merge(bd, bi, K, nb, nc, M, lane);
        }
        const int nb2 = min(K, nb + nc);
        if (lane == 0) {
            s_nb[qr] = nb2;
            s_cc[qr] = 0;
            float kd = s_kd[qr];
            int64_t ki = s_ki[qr];
            const int q = s_qpair[qr] / a.P;
            if (nb2 == K && dk_less(bd[K - 1], bi[K - 1], kd, ki)) {
                kd = bd[K - 1];
                ki = bi[K - 1];
                atomicMin(reinterpret_cast<int *>(a.thr) + q, __float_as_int(kd));
            }
            const float g = __ldcg(a.thr + q);
            if (g < kd) {
                kd = g;
                ki = NOID;
            }
            s_kd[qr] = kd;
            s_ki[qr] = ki;
        }
        __syncwarp();
    };

    for (;;) {
        if (tid == 0) *s_item = atomicAdd(&a.ctl->next_item, 1);
        __syncthreads();
        const int item = *s_item;
        if (item >= a.ctl->nitems || *s_abort) break;

        // item -> list, query tile, slab chunk
        const int2 it = a.items[item];
        const int l = it.x;
        const int nc_l = a.nch[l];
        const int tile = it.y >> 8, chunk = it.y & 255;
        const int mcount = a.lcnt[l];
        const int r0 = tile * TQ;                     // tiles filled from the front;
        const int m = min(TQ, mcount - r0);           // the last one skips empty groups
        int ns_total = a.nslabs[l];
        if (ns_total > a.dir_cap) {
            if (tid == 0) atomicOr(a.err, ERR_DIR_BOUND);
            ns_total = (int)a.dir_cap;
        }
        const int s0 = (int)((int64_t)ns_total * chunk / nc_l);
        const int s1 = (int)((int64_t)ns_total * (chunk + 1) / nc_l);
        const int ns = s1 - s0;
        const int32_t *dirl = a.dir + (size_t)l * a.dir_cap;

        // stage the first slabs while the query tile is gathered
        if (tid == 0) {
            for (int t = 0; t < NST && t < ns; ++t) {
                issue((g_issue % NST), dirl[s0 + t]);
                ++g_issue;
            }
        }
        const int qb = a.loff[l] + r0;
        for (int r = tid; r < TQ; r += SCAN_NT) {
            const int pr = r < m ? a.qlist[qb + r] : -1;
            s_qpair[r] = pr;
            s_cc[r] = 0;
            s_nb[r] = 0;
            s_kd[r] = pr >= 0 ? __ldcg(a.thr + pr / a.P) : INFINITY;
            s_ki[r] = NOID;
        }
        __syncthreads();
        for (int e = tid; e < TQ * (d / 4); e += SCAN_NT) {
            const int r = e / (d / 4), j4 = e % (d / 4);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const int pr = s_qpair[r];
            if (pr >= 0)
                v = *reinterpret_cast<const float4 *>(a.q + (size_t)(pr / a.P) * d + 4 * j4);
            *reinterpret_cast<float4 *>(Qs + (size_t)r * DP + 4 * j4) = v;
        }
        __syncthreads();

        const bool warp_active = wq * 8 * RQ < m;  // some row of this warp is real
        for (int idx = 0; idx < ns; ++idx) {
            const int stage = g_cons % NST;
            const uint32_t parity = (g_cons / NST) & 1u;
            if (!mbar_wait_bounded(&mbar[stage], parity, a.err)) *s_abort = 1;
            ++g_cons;
            const int s = stage_slab[stage];
            if (s >= 0 && warp_active && !*s_abort) {
                const float *xs = Xs + (size_t)stage * C * d;
                const int64_t *ib = IDs + (size_t)stage * C;
                float acc[RQ][RX];
                const float *qrow = Qs + (size_t)(wq * 8 * RQ + qy) * DP;
                const float *xrow = xs + (size_t)(ws * 4 * RX + sx) * d;
                // only the row groups that hold queries are computed
                const int nact = min(RQ, (m - wq * 8 * RQ + 7) / 8);
                if (nact >= RQ) dist_tile<RQ, RQ, RX>(acc, qrow, xrow, d, DP);
                else if (nact == 1) dist_tile<1, RQ, RX>(acc, qrow, xrow, d, DP);
                else if (nact == 2) dist_tile<(RQ >= 2 ? 2 : 1), RQ, RX>(acc, qrow, xrow, d, DP);
                else dist_tile<(RQ >= 3 ? 3 : 1), RQ, RX>(acc, qrow, xrow, d, DP);
                uint32_t bw[W];
#pragma unroll
                for (int w = 0; w < W; ++w) bw[w] = __ldg(a.bits + (size_t)s * W + w);
                if (idx == 0) {
                    // first slab of the tile: every distance goes to the row's
                    // candidate area, indexed by slot (sorted below)
#pragma unroll
                    for (int i = 0; i < RQ; ++i) {
                        const int qr = wq * 8 * RQ + qy + 8 * i;
                        if (qr >= m) continue;
#pragma unroll
                        for (int r = 0; r < RX; ++r) {
                            const int slot = ws * 4 * RX + sx + 4 * r;
                            const bool live = (bw[slot >> 5] >> (slot & 31)) & 1u;
                            BD[(size_t)qr * M + K + slot] = live ? acc[i][r] : INFINITY;
                            BI[(size_t)qr * M + K + slot] = live ? ib[slot] : -1;
                        }
                    }
                } else {
#pragma unroll
                for (int i = 0; i < RQ; ++i) {
                    const int qr = wq * 8 * RQ + qy + 8 * i;
                    if (qr >= m) continue;
                    const float kd = s_kd[qr];
                    const int64_t ki = s_ki[qr];
#pragma unroll
                    for (int r = 0; r < RX; ++r) {
                        const int slot = ws * 4 * RX + sx + 4 * r;
                        if (!((bw[slot >> 5] >> (slot & 31)) & 1u)) continue;
                        const float dd = acc[i][r];
                        if (dd < kd || (dd == kd && ib[slot] < ki)) {
                            const int pos = atomicAdd(&s_cc[qr], 1);
                            BD[(size_t)qr * M + K + pos] = dd;
                            BI[(size_t)qr * M + K + pos] = ib[slot];
                        }
                    }
                }
                }
            } else if (idx == 0) {
                // an inactive warp or a skipped slab leaves its rows empty
#pragma unroll
                for (int i = 0; i < RQ; ++i) {
                    const int qr = wq * 8 * RQ + qy + 8 * i;
                    if (qr >= m) continue;
#pragma unroll
                    for (int r = 0; r < RX; ++r) {
                        BD[(size_t)qr * M + K + ws * 4 * RX + sx + 4 * r] = INFINITY;
                        BI[(size_t)qr * M + K + ws * 4 * RX + sx + 4 * r] = -1;
                    }
                }
            }
            __syncthreads();
            // the stage is free: fetch the slab NST ahead into it
            if (tid == 0 && idx + NST < ns && !*s_abort) {
                fence_proxy_async_smem();
                issue(g_issue % NST, dirl[s0 + idx + NST]);
                ++g_issue;
            }
            const bool last = idx + 1 == ns;
            if (idx == 0) {
                // exact best K of the first slab of every row: one warp per
                // row sorts the row's C distances in registers (the slab's
                // stage is already being refilled: ids come from the row)
                constexpr int E = C / 32;
                for (int qr = warp; qr < m; qr += SCAN_NT / 32) {
                    float v[E];
                    int64_t id[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int slot = lane + 32 * e;
                        v[e] = BD[(size_t)qr * M + K + slot];
                        id[e] = BI[(size_t)qr * M + K + slot];
                    }
                    warp_bitonic_sort<E>(v, id, lane);
                    const float kd0 = s_kd[qr];
                    const int64_t ki0 = s_ki[qr];
                    int nb = 0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int i = lane + 32 * e;
                        const bool keep = id[e] >= 0 && i < K && dk_less(v[e], id[e], kd0, ki0);
                        nb += __popc(__ballot_sync(0xffffffffu, keep));
                        if (keep) {
                            BD[(size_t)qr * M + i] = v[e];
                            BI[(size_t)qr * M + i] = id[e];
                        }
                    }
                    __syncwarp();
                    if (lane == 0) {
                        s_nb[qr] = nb;
                        s_cc[qr] = 0;
                    }
                    __syncwarp();
                    merge_row(qr);  // nothing to merge: refreshes the threshold
                }
            } else {
                // merge rows whose buffer could overflow on the next slab (all
                // rows after the last slab)
                for (int qr = warp; qr < m; qr += SCAN_NT / 32)
                    if (s_cc[qr] > 0 && (last || s_cc[qr] > CB - C)) merge_row(qr);
            }
            __syncthreads();
        }

        // the best K of each row of the tile (padded with (+inf, -1))
        for (int e = tid; e < m * K; e += SCAN_NT) {
            const int r = e / K, j = e % K;
            const int run = a.prun[s_qpair[r]];
            if (run < 0) continue;
            const int64_t base = ((int64_t)run + chunk) * K;
            const bool ok = j < s_nb[r];
            a.part_d[base + j] = ok ? BD[(size_t)r * M + j] : INFINITY;
            a.part_i[base + j] = ok ? BI[(size_t)r * M + j] : -1;
        }
        __syncthreads();
    }
    // after an abort, give copies still in flight a bounded chance to land
    // before the CTA (and its shared memory) goes away
    if (tid == 0)
        while (g_cons < g_issue) {
            mbar_wait_bounded(&mbar[g_cons % NST], (g_cons / NST) & 1u, a.err, 100000u);
            ++g_cons;
        }
}

// ------------------------------------------------------- per-query merge
constexpr int MERGE_NT = 128;
constexpr int MERGE_RUNS_PER_LANE = 64;

__global__ __launch_bounds__(MERGE_NT) void k_merge(const int2 *__restrict__ qrun, int64_t nq,
                                                    int K, int k,
                                                    const float *__restrict__ part_d,
                                                    const int64_t *__restrict__ part_i,
                                                    float *__restrict__ dist,
                                                    int64_t *__restrict__ labels)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)MERGE_NT + threadIdx.x) >> 5;
    if (q >= nq) return;
    // the query's runs (sorted, padded with (+inf, -1)) are contiguous:
    // r = lane, lane + 32, ... of them, cursor per run kept in local memory
    const int2 qr = qrun[q];
    int cur[MERGE_RUNS_PER_LANE];
    int nrun = 0;
    for (int r = lane; r < qr.y && nrun < MERGE_RUNS_PER_LANE; r += 32) cur[nrun++] = 0;
    auto head = [&](int j, float &hd, int64_t &hi) {
        int r = lane + 32 * j;
        if (cur[j] >= K) {
            hd = INFINITY;
            hi = -1;
            return;
        }
        int64_t e = ((int64_t)qr.x + r) * K + cur[j];
        hd = part_d[e];
        hi = part_i[e];
        if (hi < 0) hd = INFINITY;
    };
    float bd = INFINITY;
    int64_t bi = -1;
    int bj = -1;
    auto rescan = [&]() {
        bd = INFINITY;
        bi = -1;
        bj = -1;
        for (int j = 0; j < nrun; ++j) {
            float hd;
            int64_t hi;
            head(j, hd, hi);
            if (hi >= 0 && (bj < 0 || dk_less(hd, hi, bd, bi))) {
                bd = hd;
                bi = hi;
                bj = j;
            }
        }
    };
    rescan();
    for (int o = 0; o < k; ++o) {
        float wd = bd;
        int64_t wi = bi;
        int wl = bj >= 0 ? lane : 32;
        for (int s = 16; s > 0; s >>= 1) {
            float od = __shfl_xor_sync(0xffffffffu, wd, s);
            int64_t oi = __shfl_xor_sync(0xffffffffu, wi, s);
            int ol = __shfl_xor_sync(0xffffffffu, wl, s);
            bool take = ol < 32 && (wl >= 32 || dk_less(od, oi, wd, wi));
            if (take) {
                wd = od;
                wi = oi;
                wl = ol;
            }
        }
        if (lane == 0) {
            dist[q * k + o] = wl < 32 ? wd : INFINITY;
            labels[q * k + o] = wl < 32 ? wi : -1;
        }
        if (wl == lane) {
            ++cur[bj];
            rescan();
        }
    }
}

// --------------------------------------------------------------- drivers
template <int TQ, int C>
static void launch_scan(sivf_index *ix, const ScanArgs &a, size_t smem, int grid,
                        cudaStream_t st)
{
    static size_t attr = 48 * 1024;
    if (smem > attr) {
        cudaFuncSetAttribute(k_scan<TQ, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = smem;
    }
    const int tok = prof_begin(ix, PROF_SCAN, 1, st);
    launch_pdl(k_scan<TQ, C>, grid, SCAN_NT, smem, st, a);
    prof_end(ix, tok, st);
}

int tune_bucket(const sivf_index *ix, int64_t nq, int P)
{
    const double r = std::max((double)nq * P / ix->nlist, 1.0 / 256);
    const int b = (int)std::floor(std::log2(r)) + 8;
    return std::min(std::max(b, 0), kTuneB - 1);
}

int tune_kbucket(int K) { return K <= 16 ? 0 : K <= 64 ? 1 : K <= 256 ? 2 : 3; }

// k-select buffer of the FP32 scan: the best K plus `slabs` slabs of
// candidates, beyond 256 entries a power of two (bitonic fallback);
// slabs = 0 is the built-in width
static int fp32_width(int K, int C, int slabs)
{
    if (slabs == 0) return scan_buf_len(K, C);
    const int v = K + slabs * C;
    return v <= 256 ? ((v + 15) & ~15) : scan_next_pow2(v);
}

sivf_tile default_tile(const sivf_index *ix, int dtype, int64_t nq, int P, int K)
{
    sivf_tile t;
    if (dtype == SIVF_FP32) {
        const double ppl = (double)nq * P / ix->nlist;
        t.queries_per_tile = ppl >= 48 ? 64 : ppl >= 24 ? 32 : ppl >= 12 ? 16 : 8;
        while (t.queries_per_tile > 8 &&
               scan_smem(t.queries_per_tile, ix->C, ix->d, scan_buf_len(K, ix->C)).total >
                   220 * 1024)
            t.queries_per_tile >>= 1;
        t.slabs_per_chunk = 2;
        t.items_per_sm = 4;
        t.select_slabs = 0;
        t.nearest_first = 0;
    } else {
        // the vector-row scan (the query-row scan, 128, is a tile option)
        t.queries_per_tile = 64;
        t.slabs_per_chunk = 4;
        t.items_per_sm = 4;
        t.select_slabs = 0;
        t.nearest_first = 1;
    }
    return t;
}

bool tile_valid(const sivf_index *ix, int dtype, const sivf_tile &t, int K)
{
    if (t.slabs_per_chunk < 1 || t.slabs_per_chunk > 16 || t.items_per_sm < 1 ||
        t.items_per_sm > 16)
        return false;
    if (dtype == SIVF_FP32) {
        const int tq = t.queries_per_tile;
        if (!(tq == 8 || tq == 16 || tq == 32 || tq == 64)) return false;
        if (t.select_slabs < 0 || t.select_slabs > 8) return false;
        return scan_smem(tq, ix->C, ix->d, fp32_width(K, ix->C, t.select_slabs)).total <=
               220 * 1024;
    }
    if (t.nearest_first < 0 || t.nearest_first > 2) return false;
    if (t.queries_per_tile == 128)
        return t.select_slabs >= 0 && t.select_slabs <= 3 && qt_shape(ix, dtype, K).ok;
    if (t.queries_per_tile != 64) return false;
    if (t.select_slabs < 0 || t.select_slabs > 3) return false;
    return tc_buf_fits(ix, dtype, K, tc_buf_entries(ix, dtype, K, t.select_slabs));
}

sivf_tile current_tile(const sivf_index *ix, int dtype, int64_t nq, int P, int K)
{
    const TileChoice &c = ix->tune[dtype][tune_bucket(ix, nq, P)][tune_kbucket(K)];
    if (c.set && tile_valid(ix, dtype, c.t, K)) return c.t;
    return default_tile(ix, dtype, nq, P, K);
}

SearchPlan plan_from_tile(const sivf_index *ix, int dtype, int64_t nq, int P, int K,
                          const sivf_tile &t)
{
    SearchPlan pl;
    const bool fp32 = dtype == SIVF_FP32;
    pl.qt = !fp32 && t.queries_per_tile == 128;
    pl.tq = fp32 ? t.queries_per_tile : pl.qt ? 128 : tc_tile_queries(K);
    pl.K = K;
    pl.M = fp32  ? fp32_width(K, ix->C, t.select_slabs)
           : pl.qt ? qt_shape(ix, dtype, K).ME
                   : tc_buf_entries(ix, dtype, K, t.select_slabs);
    pl.split = fp32 ? 0 : t.nearest_first;
    pl.sel = t.select_slabs;
    pl.RK = (fp32 || pl.qt) ? K : tc_run_len(K);
    // slab chunks: a list is split when its items would be long against the
    // launch's work per SM (decided on the device from the grouped pairs);
    // at most 2048 runs per query reach the merge
    pl.ch = std::max(1, std::min(kMaxChunks, 2048 / std::max(P, 1)));
    pl.slabs_per_chunk = t.slabs_per_chunk;
    pl.ips = t.items_per_sm;
    // the other lists of split 1 run under the bounds of the nearest, so few
    // rows reach a buffer: K' > 128 takes 32-query tiles with one tile of
    // room there (half the tiles of 16)
    pl.tq2 = pl.tq;
    pl.M2 = pl.M;
    if (!fp32 && !pl.qt && pl.split == 1 && P > 1) {
        const int m2 = tc_wide_entries(ix, dtype, K);
        if (m2 > 0) {
            pl.tq2 = 32;
            pl.M2 = m2;
        }
    }
    pl.run_cap = plan_run_cap(nq, P, std::max(pl.tq, pl.tq2), pl.ips);
    pl.item_cap = plan_item_cap(nq, P, ix->nlist, pl.ips);
    return pl;
}

int64_t plan_run_cap(int64_t nq, int P, int tq, int ips)
{
    // a run per scanned pair, plus per scan phase (at most two) the chunks
    // past the first: at most tq * ips * 152
    return nq * P + 2 * (int64_t)tq * ips * 152;
}

int64_t plan_item_cap(int64_t nq, int P, int L, int ips)
{
    // a tile per (list, up to tq pairs), plus at most ips * 152 extra chunks
    return nq * P + L + (int64_t)ips * 152;
}

SearchPlan plan_search(const sivf_index *ix, int64_t nq, int P, int K)
{
    return plan_from_tile(ix, SIVF_FP32, nq, P, K, current_tile(ix, SIVF_FP32, nq, P, K));
}

bool scan_fits(const sivf_index *ix, int K)
{
    return scan_smem(8, ix->C, ix->d, scan_buf_len(K, ix->C)).total <= 220 * 1024;
}

void group_pairs(sivf_index *ix, int64_t nq, int P, int p0, int p1, const int32_t *probes,
                 bool dedupe, const SearchPlan &pl, const SearchScratch &s, int64_t slab_bytes,
                 cudaStream_t st, bool stats)
{
    const int L = ix->nlist;
    cudaMemsetAsync(s.lcnt, 0, sizeof(int32_t) * L, st);
    const int64_t n = nq * (p1 - p0);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
    const int tg = prof_begin(ix, PROF_GROUP, 3, st);
    launch_pdl(k_srch_hist, g, 256, 0, st, probes, nq, P, p0, p1, L, dedupe, s.lcnt, s.prank);
    launch_pdl(k_srch_plan, 1, 1024, 0, st, s.lcnt, ix->nslabs, ix->list_live, L, pl.tq, pl.ch,
               pl.slabs_per_chunk, pl.ips, pl.item_cap, slab_bytes, s.loff, s.ibase, s.nch, s.items,
               ix->ctl, stats ? ix->stat : nullptr, ix->err);
    if (p1 - p0 >= 8) {
        const int gs = (int)std::max<int64_t>(1, std::min<int64_t>((nq + SC_Q - 1) / SC_Q, 152 * 16));
        launch_pdl(k_srch_scatter, gs, SC_Q * 32, 0, st, probes, nq, P, p0, p1, s.prank, s.loff,
                   s.nch, s.qlist, s.prun, s.qrun, ix->ctl, pl.run_cap, ix->err);
    } else {
        const int gq = (int)std::max<int64_t>(1, std::min<int64_t>((nq + 255) / 256, 152 * 16));
        launch_pdl(k_srch_scatter_t, gq, 256, 0, st, probes, nq, P, p0, p1, s.prank, s.loff, s.nch,
                   s.qlist, s.prun, s.qrun, ix->ctl, pl.run_cap, ix->err);
    }
    prof_end(ix, tg, st);
}

void scan_lists(sivf_index *ix, const float *q, int64_t nq, int P, const int32_t *probes,
                bool dedupe, const SearchPlan &pl, const SearchScratch &s, cudaStream_t st)
{
    const int L = ix->nlist;
    cudaMemsetAsync(s.thr, 0x7f, sizeof(float) * nq, st);  // 3.4e38: no bound yet
    group_pairs(ix, nq, P, 0, P, probes, dedupe, pl, s,
                (int64_t)ix->C * (ix->d * 4 + 8) + ix->C / 8, st);

    ScanArgs a;
    a.q = q;
    a.nq = nq;
    a.P = P;
    a.K = pl.K;
    a.M = pl.M;
    a.prun = s.prun;
    a.qlist = s.qlist;
    a.loff = s.loff;
    a.lcnt = s.lcnt;
    a.ibase = s.ibase;
    a.nch = s.nch;
    a.part_d = s.part_d;
    a.part_i = s.part_i;
    a.thr = s.thr;
    a.items = s.items;
    a.x32 = ix->x32;
    a.ids = ix->ids;
    a.bits = ix->bits;
    a.meta = ix->meta;
    a.nslabs = ix->nslabs;
    a.dir = ix->dir;
    a.n_slabs = ix->n_slabs;
    a.dir_cap = ix->dir_cap;
    a.L = L;
    a.d = ix->d;
    a.ctl = ix->ctl;
    a.err = ix->err;
    const size_t smem = scan_smem(pl.tq, ix->C, ix->d, a.M).total;
    const int grid = 152;  // persistent: one CTA per SM
#define SIVF_SCAN_CASE(TQ_, C_) \
    if (pl.tq == TQ_ && ix->C == C_) return launch_scan<TQ_, C_>(ix, a, smem, grid, st);
    SIVF_SCAN_CASE(8, 32) SIVF_SCAN_CASE(16, 32) SIVF_SCAN_CASE(32, 32) SIVF_SCAN_CASE(64, 32)
    SIVF_SCAN_CASE(8, 64) SIVF_SCAN_CASE(16, 64) SIVF_SCAN_CASE(32, 64) SIVF_SCAN_CASE(64, 64)
    SIVF_SCAN_CASE(8, 128) SIVF_SCAN_CASE(16, 128) SIVF_SCAN_CASE(32, 128)
    SIVF_SCAN_CASE(64, 128)
#undef SIVF_SCAN_CASE
}

void merge_topk(sivf_index *ix, int64_t nq, int P, const int32_t *probes,
                const SearchPlan &pl, const SearchScratch &s, int k, float *dist,
                int64_t *labels, cudaStream_t st)
{
    int64_t warps = nq;
    int64_t blocks = (warps * 32 + MERGE_NT - 1) / MERGE_NT;
    const int tok = prof_begin(ix, PROF_MERGE, 1, st);
    launch_pdl(k_merge, (unsigned)blocks, MERGE_NT, 0, st, s.qrun, nq, pl.K, k, s.part_d, s.part_i,
               dist, labels);
    prof_end(ix, tok, st);
}

}  // namespace sivf
