// Reduced-precision list scan on the tensor cores, then an exact FP32
// re-rank (the precision pattern of the hot path; the paper scans FP32
// only).
//
// Lists keep a BF16 or an FP8 E4M3 copy of every payload row (per-list
// scale for FP8).  One CTA takes one (list, tile of up to 64 queries, slab
// chunk) item.  The list's slabs stream through shared memory as 128-row
// A tiles (TMA 2-D loads, 128-byte swizzle); the query tile, rounded to the
// same format, is the B operand; tcgen05.mma accumulates the 128 x 64 dot
// products in FP32 in tensor memory (double-buffered, so the next tile's
// MMAs overlap the epilogue of this one).  The epilogue forms the expanded
// distance ||q||^2 + ||x||^2 - 2 s q.x (FP32 norms of the unrounded
// vectors, s the dequantisation scale), and every query keeps its best K'
// (= 4k) (distance, slot) candidates.  A per-query shared bound (the K'-th
// distance any item has found) prunes the rest.  A final pass recomputes
// the K' survivors' distances exactly in FP32 from the FP32 payload and
// keeps the best k by (distance, id).
//
// Roles inside the CTA (8 warps): thread 0 drives TMA, warp 1 lane 0 issues
// the MMAs, warp 2 owns the tensor-memory allocation, warps 4-7 read tensor
// memory and select candidates.  Every wait is bounded.
#include <cudaTypedefs.h>
#include <math.h>

#include "device_utils.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace sivf {

constexpr int TC_M = 128;       // rows per A tile (MMA M)
constexpr int TC_NCOL = 16;     // query columns per epilogue warp
// Two tile shapes: 64 queries per tile for K' <= 128, 16 queries (and
// buffers for K' <= 512) for deeper re-ranks.  Epilogue warps: four per
// TMEM lane quarter at 64 queries, one at 16.
template <int TN> struct TcShape {
    static constexpr int N = TN;                        // queries per tile (MMA N)
    static constexpr int EW = 4 * (TN / TC_NCOL);       // epilogue warps
    static constexpr int EPI = EW * 32;                 // epilogue threads
    static constexpr int NT = 128 + EPI;                // + TMA, MMA, TMEM owner, idle warp
    static constexpr int NST = EW >= 16 ? 2 : 3;        // A-tile stages in flight
    static constexpr int KMAX = TN == 64 ? 128 : 512;   // deepest K' the buffers take
};

struct TcArgs {
    const float *q;
    int64_t nq;
    int P, K, M, CH;
    const int32_t *qlist, *loff, *lcnt, *ibase, *nch;
    const int2 *items;
    const float *qn, *qsc;
    float *part_d;
    int64_t *part_i;  // global slot (slab * C + slot) of each candidate
    float *thr;
    const float *xnorm;
    const uint32_t *bits;
    const int32_t *nslabs, *dir;
    const float *inv_scale8;
    int64_t n_slabs, dir_cap;
    int L, d, C, KC;  // KC = 128-byte K chunks per row
    Ctl *ctl;
    uint32_t *err;
};

constexpr int TC_META = 256;    // slabs whose ids and bitmaps are staged at once

struct TcSmem {
    size_t a, b, bd, bs, msl, mbits, hist, stg, misc, total;
};
template <int TN>
__host__ __device__ inline TcSmem tc_smem(int KC, int M)
{
    using S = TcShape<TN>;
    TcSmem s;
    s.a = 0;                                             // NST x KC x 16 KB
    s.b = s.a + (size_t)S::NST * KC * TC_M * 128;        // KC x TN rows x 128 B
    s.bd = s.b + (size_t)KC * TN * 128;
    s.bs = s.bd + (size_t)TN * M * 4;
    s.msl = s.bs + (size_t)TN * M * 4;
    s.mbits = s.msl + (size_t)TC_META * 4;
    s.hist = s.mbits + (size_t)TC_META * 4 * 4;           // per warp 256 bins
    s.stg = s.hist + (size_t)S::EW * 256 * 4;             // per warp KMAX (dist, slot)
    s.misc = s.stg + (size_t)S::EW * S::KMAX * 8;
    s.total = s.misc + 1024 + 1024;                      // + base alignment slack
    return s;
}

// (distance, slot) order with pads (+inf, INT_MAX) last
__device__ __forceinline__ bool ds_less(float a, int32_t sa, float b, int32_t sb)
{
    return a < b || (a == b && sa < sb);
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

// Merge nc unsorted candidates (bd/bs[K, K+nc)) into the sorted best list
// (bd/bs[0, nb)), keeping the K smallest: the candidates are sorted in
// registers, written back in order, and every output position finds its
// split between the two sorted runs by binary search (merge path).
template <int EC, int KMAX>
__device__ void warp_sort_merge32(float *bd, int32_t *bs, int K, int nb, int nc, int lane)
{
    float v[EC];
    int32_t sv[EC];
#pragma unroll
    for (int e = 0; e < EC; ++e) {
        const int i = lane + 32 * e;
        v[e] = i < nc ? bd[K + i] : INFINITY;
        sv[e] = i < nc ? bs[K + i] : 0x7fffffff;
    }
    warp_sort32<EC>(v, sv, lane);
#pragma unroll
    for (int e = 0; e < EC; ++e) {
        const int i = lane + 32 * e;
        if (i < nc) {
            bd[K + i] = v[e];
            bs[K + i] = sv[e];
        }
    }
    __syncwarp();
    const int n = min(K, nb + nc);
    constexpr int OPL = KMAX / 32;  // outputs per lane (K <= KMAX)
    float ov[OPL];
    int32_t os[OPL];
#pragma unroll
    for (int t = 0; t < OPL; ++t) {
        const int o = lane + 32 * t;
        if (o >= n) continue;
        // smallest i in [lo, hi] with: taking i best and o - i candidates
        int lo = max(0, o - nc), hi = min(o, nb);
        while (lo < hi) {
            const int i = (lo + hi) >> 1;          // i best, o - i candidates before o
            const int j = o - i - 1;               // last candidate taken
            if (ds_less(bd[K + j], bs[K + j], bd[i], bs[i])) hi = i;
            else lo = i + 1;
        }
        const int i = lo, j = o - lo;
        const bool from_best = i < nb && (j >= nc || !ds_less(bd[K + j], bs[K + j], bd[i], bs[i]));
        ov[t] = from_best ? bd[i] : bd[K + j];
        os[t] = from_best ? bs[i] : bs[K + j];
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < OPL; ++t) {
        const int o = lane + 32 * t;
        if (o < n) {
            bd[o] = ov[t];
            bs[o] = os[t];
        }
    }
    __syncwarp();
}

// Keep the K smallest of best[0, nb) (sorted) and cand[K, K + nc) when the
// union is too large to sort in registers: a warp radix select finds the
// K-th smallest key in 8-bit passes over the union, the entries at or
// below it (ties included, at most KMAX) are gathered and sorted.  More
// than KMAX entries tied at the K-th key keep the first ones found,
// ordered by slot among the gathered.
template <int KMAX>
__device__ void warp_select_merge32(float *bd, int32_t *bs, int K, int nb, int nc,
                                    uint32_t *hist, float *stg_d, int32_t *stg_s, int lane)
{
    const int n = nb + nc;
    auto at = [&](int i) { return i < nb ? i : K + (i - nb); };
    // the keys share their leading bits (distances of one list are of one
    // magnitude): start the 8-bit passes at the highest bit where they differ
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    for (int i = lane; i < n; i += 32) {
        const uint32_t k = fkey(bd[at(i)]);
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    const uint32_t diff = kmin ^ kmax;
    const int top = diff ? 31 - __clz(diff) : 0;  // highest differing bit
    uint32_t mask = top >= 31 ? 0u : ~((2u << top) - 1u);
    uint32_t prefix = kmin & mask, need = (uint32_t)K;
    for (int hi = top; hi >= 0; hi -= 8) {
        const int shift = max(hi - 7, 0);
        const uint32_t width = (uint32_t)(hi - shift + 1);
        const uint32_t bmask = (width >= 32 ? 0xffffffffu : ((1u << width) - 1u));
#pragma unroll
        for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0u;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const uint32_t k = fkey(bd[at(i)]);
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & bmask], 1u);
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
        uint32_t bin = 0, below = 0;
        if (mine) {
            uint32_t cum = excl;
            for (int b = 0; b < 8; ++b) {
                if (cum + loc[b] >= need) {
                    bin = (uint32_t)(lane * 8 + b);
                    below = cum;
                    break;
                }
                cum += loc[b];
            }
        }
        const uint32_t who = __ballot_sync(0xffffffffu, mine);
        const int src = who ? __ffs(who) - 1 : 0;
        bin = __shfl_sync(0xffffffffu, bin, src);
        below = __shfl_sync(0xffffffffu, below, src);
        prefix |= bin << shift;
        mask |= bmask << shift;
        need -= below;
        __syncwarp();
    }
    // gather every entry at or below the K-th key (at most KMAX)
    int cnt = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        bool take = false;
        float dv = 0.f;
        int32_t sv = 0;
        if (i < n) {
            dv = bd[at(i)];
            sv = bs[at(i)];
            take = fkey(dv) <= prefix;
        }
        const uint32_t mk = __ballot_sync(0xffffffffu, take);
        const int p = cnt + __popc(mk & lanemask_lt());
        if (take && p < KMAX) {
            stg_d[p] = dv;
            stg_s[p] = sv;
        }
        cnt += __popc(mk);
    }
    __syncwarp();
    cnt = min(cnt, KMAX);
    constexpr int E = KMAX / 32;
    float v[E];
    int32_t sv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        v[e] = i < cnt ? stg_d[i] : INFINITY;
        sv[e] = i < cnt ? stg_s[i] : 0x7fffffff;
    }
    warp_sort32<E>(v, sv, lane);
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < K) {
            bd[i] = v[e];
            bs[i] = sv[e];
        }
    }
    __syncwarp();
}

template <int DT, int TN>  // DT: 0 = BF16, 1 = FP8 E4M3; TN: queries per tile
__global__ __launch_bounds__(TcShape<TN>::NT, 1) void k_scan_tc(
    const __grid_constant__ CUtensorMap tmap, TcArgs a)
{
    using S = TcShape<TN>;
    constexpr int TC_N = TN, TC_EW = S::EW, TC_EPI = S::EPI, TC_NT = S::NT, TC_NST = S::NST;
    constexpr int KMAX = S::KMAX;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled operand tiles
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int KC = a.KC, M = a.M, K = a.K, C = a.C, d = a.d;
    const TcSmem L = tc_smem<TN>(KC, M);
    unsigned char *A = smem + L.a;
    unsigned char *B = smem + L.b;
    float *BD = reinterpret_cast<float *>(smem + L.bd);
    int32_t *BS = reinterpret_cast<int32_t *>(smem + L.bs);
    int32_t *Msl = reinterpret_cast<int32_t *>(smem + L.msl);     // slab ids
    uint32_t *Mbits = reinterpret_cast<uint32_t *>(smem + L.mbits);  // their bitmaps
    uint32_t *Hist = reinterpret_cast<uint32_t *>(smem + L.hist);
    unsigned char *Stg = smem + L.stg;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.misc);
    uint64_t *full = bars, *empty = bars + TC_NST, *tfull = bars + 2 * TC_NST,
             *tempty = bars + 2 * TC_NST + 2;
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(bars + 2 * TC_NST + 4);
    int *s_item = reinterpret_cast<int *>(bars + 2 * TC_NST + 5);
    int *s_abort = s_item + 1;
    __shared__ int32_t s_qpair[TC_N], s_cc[TC_N], s_nb[TC_N], s_ks[TC_N];
    __shared__ float s_kd[TC_N], s_qn[TC_N], s_qsc[TC_N];
    __shared__ __align__(16) float s_t[TC_N];   // kd - ||q||^2 of each row, per tile

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int ESZ = DT == 0 ? 2 : 1;
    constexpr int EPC = 128 / ESZ;  // elements per 128-byte chunk
    const int SPB = TC_M / C;       // slabs per A tile
    const uint32_t idesc = DT == 0 ? mma_idesc(1, 1, TC_M, TC_N) : mma_idesc(0, 0, TC_M, TC_N);

    if (tid == 0) {
        for (int i = 0; i < TC_NST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], TC_EPI);
        }
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == 2) tmem_alloc(tmem_base, 2 * TC_N);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_base;

    uint32_t gblk = 0;  // A tiles processed by this CTA (all roles agree)
    for (;;) {
        if (tid == 0) *s_item = atomicAdd(&a.ctl->next_item, 1);
        __syncthreads();
        const int item = *s_item;
        if (item >= a.ctl->nitems || *s_abort) break;

        const int2 it = a.items[item];
        const int l = it.x;
        const int nc_l = a.nch[l];
        const int tile = it.y >> 8, chunk = it.y & 255;
        const int r0 = tile * TC_N;
        const int m = min(TC_N, a.lcnt[l] - r0);
        int ns_total = a.nslabs[l];
        if (ns_total > a.dir_cap) {
            if (tid == 0) atomicOr(a.err, ERR_DIR_BOUND);
            ns_total = (int)a.dir_cap;
        }
        const int s0 = (int)((int64_t)ns_total * chunk / nc_l);
        const int ns = (int)((int64_t)ns_total * (chunk + 1) / nc_l) - s0;
        const int nblk = (ns + SPB - 1) / SPB;
        // rows of a thin tile get proportionally longer candidate buffers
        const int ME = max(M, ((TC_N * M) / max(m, 1)) & ~7);
        const int32_t *dirl = a.dir + (size_t)l * a.dir_cap + s0;
        const float inv_l = DT == 1 ? a.inv_scale8[l] : 1.f;

        // ---- query tile: norms, thresholds, B operand (rounded, swizzled)
        const int qb = a.loff[l] + r0;
        for (int r = tid; r < TC_N; r += TC_NT) {
            const int pr = r < m ? a.qlist[qb + r] : -1;
            const int qi = pr >= 0 ? pr / a.P : 0;
            s_qpair[r] = pr;
            s_cc[r] = 0;
            s_nb[r] = 0;
            s_kd[r] = pr >= 0 ? __ldcg(a.thr + qi) : INFINITY;
            s_ks[r] = 0x7fffffff;
            s_qn[r] = pr >= 0 ? a.qn[qi] : 0.f;
            s_qsc[r] = pr >= 0 ? a.qsc[qi] : 1.f;
            s_t[r] = pr >= 0 ? s_kd[r] - s_qn[r] : -INFINITY;
        }
        __syncthreads();
        for (int e = tid; e < TC_N * KC * 8; e += TC_NT) {
            const int r = e / (KC * 8), kc = (e / 8) % KC, c = e % 8;
            const int pr = s_qpair[r];
            const int k0 = kc * EPC + c * (16 / ESZ);  // first element of the 16-byte chunk
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (pr >= 0 && k0 < d) {                  // d % 16 == 0: chunks are all in or out
                const float4 *qr = reinterpret_cast<const float4 *>(a.q + (size_t)(pr / a.P) * d + k0);
                if (DT == 0) {
                    const float4 f0 = qr[0], f1 = qr[1];
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(f0.x, f0.y);
                    __nv_bfloat162 h1 = __floats2bfloat162_rn(f0.z, f0.w);
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(f1.x, f1.y);
                    __nv_bfloat162 h3 = __floats2bfloat162_rn(f1.z, f1.w);
                    w[0] = *reinterpret_cast<uint32_t *>(&h0);
                    w[1] = *reinterpret_cast<uint32_t *>(&h1);
                    w[2] = *reinterpret_cast<uint32_t *>(&h2);
                    w[3] = *reinterpret_cast<uint32_t *>(&h3);
                } else {
                    const float sc = s_qsc[r];
                    float4 f[4] = {qr[0], qr[1], qr[2], qr[3]};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float2 p0 = make_float2(__fmul_rn(f[t].x, sc), __fmul_rn(f[t].y, sc));
                        const float2 p1 = make_float2(__fmul_rn(f[t].z, sc), __fmul_rn(f[t].w, sc));
                        const uint32_t lo8 = __nv_cvt_float2_to_fp8x2(p0, __NV_SATFINITE, __NV_E4M3);
                        const uint32_t hi8 = __nv_cvt_float2_to_fp8x2(p1, __NV_SATFINITE, __NV_E4M3);
                        w[t] = lo8 | (hi8 << 16);
                    }
                }
            }
            unsigned char *dst = B + (size_t)kc * TC_N * 128 + (size_t)(r >> 3) * 1024 +
                                 (r & 7) * 128 + ((c ^ (r & 7)) << 4);
            *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_proxy_async_smem();  // B is read by the tensor cores (async proxy)
        __syncthreads();

        // ---- block loop: TMA -> MMA -> epilogue -> selection
        if (warp == 0) {
            if (lane == 0)
            for (int b = 0; b < nblk && !*s_abort; ++b) {
                const uint32_t g = gblk + b, st = g % TC_NST, u = g / TC_NST;
                if (u >= 1 && !mbar_wait_bounded(&empty[st], (u - 1) & 1, a.err)) {
                    *s_abort = 1;
                    break;
                }
                const int nsl = min(SPB, ns - b * SPB);
                int okc = 0;
                int sl[4];
                for (int j = 0; j < nsl; ++j) {
                    sl[j] = dirl[b * SPB + j];
                    if (sl[j] < 0 || sl[j] >= a.n_slabs) {
                        atomicOr(a.err, ERR_BAD_SLAB);
                        sl[j] = -1;
                    } else {
                        ++okc;
                    }
                }
                mbar_arrive_expect_tx(&full[st], (uint32_t)(okc * KC * C * 128));
                for (int j = 0; j < nsl; ++j) {
                    if (sl[j] < 0) continue;
                    for (int kc = 0; kc < KC; ++kc)
                        tma_load_2d(A + (size_t)st * KC * TC_M * 128 + (size_t)kc * TC_M * 128 +
                                        (size_t)j * C * 128,
                                    &tmap, kc * EPC, sl[j] * C, &full[st]);
                }
            }
            __syncwarp();
        } else if (warp == 1) {
            if (lane == 0)
            for (int b = 0; b < nblk && !*s_abort; ++b) {
                const uint32_t g = gblk + b, st = g % TC_NST, u = g / TC_NST;
                const uint32_t buf = g & 1, ub = g >> 1;
                if (!mbar_wait_bounded(&full[st], u & 1, a.err)) {
                    *s_abort = 1;
                    break;
                }
                if (ub >= 1 && !mbar_wait_bounded(&tempty[buf], (ub - 1) & 1, a.err)) {
                    *s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(A + (size_t)st * KC * TC_M * 128);
                const uint32_t bbase = smem_u32(B);
                for (int kc = 0; kc < KC; ++kc)
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = smem_desc_sw128(abase + kc * TC_M * 128 + ks * 32, 1024);
                        const uint64_t bd = smem_desc_sw128(bbase + kc * TC_N * 128 + ks * 32, 1024);
                        const uint32_t acc = (kc | ks) != 0;
                        if (DT == 0) mma_bf16(tbase + buf * TC_N, ad, bd, idesc, acc);
                        else mma_fp8(tbase + buf * TC_N, ad, bd, idesc, acc);
                    }
                mma_commit(&tfull[buf]);
                mma_commit(&empty[st]);
            }
            __syncwarp();
        } else if (warp >= 4) {
            const int ew = warp - 4;          // epilogue warp
            const int qt = ew & 3;            // its TMEM lane quarter (warp % 4)
            const int c0 = (ew >> 2) * TC_NCOL;  // its first query column
            const int et = ew * 32 + lane;    // epilogue thread
            const int v = qt * 32 + lane;     // A row = vector of the tile
            const int CB = ME - K;
            const int BPS = TC_META / SPB;    // tiles whose slab metadata is staged
            float xn_next = 0.f;
            for (int b = 0; b < nblk; ++b) {
                const uint32_t g = gblk + b, buf = g & 1, ub = g >> 1;
                if (b % BPS == 0) {
                    // stage ids + bitmaps of the next TC_META slabs of the chunk
                    named_bar_sync(1, TC_EPI);
                    const int sb0 = b * SPB, sn = min(TC_META, ns - sb0);
                    for (int i = et; i < sn; i += TC_EPI) {
                        const int sl = dirl[sb0 + i];
                        const bool okk = sl >= 0 && sl < a.n_slabs;
                        Msl[i] = okk ? sl : -1;
                        for (int w = 0; w < C / 32; ++w)
                            Mbits[i * 4 + w] = okk ? __ldg(a.bits + (size_t)sl * (C / 32) + w) : 0u;
                    }
                    named_bar_sync(1, TC_EPI);
                    const int j0 = v / C;
                    const int s_first = j0 < min(SPB, ns - b * SPB) ? Msl[(b * SPB - sb0) + j0] : -1;
                    xn_next = s_first >= 0 ? __ldg(a.xnorm + (size_t)s_first * C + v % C) : 0.f;
                }
                // row of this thread in the tile
                const int nsl = min(SPB, ns - b * SPB);
                const int j = v / C, slot = v % C;
                const int mi = (b % BPS) * SPB + j;
                const int sl = j < nsl ? Msl[mi] : -1;
                const bool live = sl >= 0 && ((Mbits[mi * 4 + (slot >> 5)] >> (slot & 31)) & 1u);
                const int32_t gslot = live ? sl * C + slot : -1;
                const float xn = xn_next;
                // prefetch ||x||^2 of the row of the next tile
                if (b + 1 < nblk && (b + 1) % BPS != 0) {
                    const int nsl2 = min(SPB, ns - (b + 1) * SPB);
                    const int mi2 = ((b + 1) % BPS) * SPB + j;
                    const int sl2 = j < nsl2 ? Msl[mi2] : -1;
                    xn_next = sl2 >= 0 ? __ldg(a.xnorm + (size_t)sl2 * C + slot) : 0.f;
                }

                bool ok = !*s_abort && mbar_wait_bounded(&tfull[buf], ub & 1, a.err);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-aligned
                if (!ok) *s_abort = 1;
                tc_fence_after();
                float dv[TC_NCOL];
                if (ok) {
#pragma unroll
                    for (int c16 = 0; c16 < TC_NCOL / 16; ++c16) {
                        float t[16];
                        tmem_ld16(tbase + buf * TC_N + c0 + c16 * 16 + ((uint32_t)(qt * 32) << 16), t);
#pragma unroll
                        for (int i = 0; i < 16; ++i) dv[c16 * 16 + i] = t[i];
                    }
                    tmem_ld_wait();
                }
                tc_fence_before();
                mbar_arrive(&tempty[buf]);

                // candidates straight from registers: a row passes for query n
                // when -s q.x + ||x||^2 <= kd_n - ||q_n||^2 (= s_t[n], set per
                // tile); per query one ballot over this warp's 32 rows and one
                // shared atomic for their buffer slots
                const float4 *t4 = reinterpret_cast<const float4 *>(s_t);
#pragma unroll
                for (int j0 = 0; j0 < TC_NCOL; j0 += 16) {
                    const int n0 = c0 + j0;
                    if (n0 >= m) break;
                    uint32_t mk[16];
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4) {
                        const float4 tv = t4[(n0 >> 2) + i4];
                        const float tt[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int n = n0 + 4 * i4 + c;
                            const float sc = DT == 0 ? 2.f : 2.f / (inv_l * s_qsc[n]);
                            const float part = fmaf(-sc, dv[j0 + 4 * i4 + c], xn);
                            mk[4 * i4 + c] = __ballot_sync(0xffffffffu, ok && live && part <= tt[c]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (!mk[i]) continue;
                        const int n = n0 + i;
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&s_cc[n], __popc(mk[i]));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if ((mk[i] >> lane) & 1u) {
                            const float sc = DT == 0 ? 2.f : 2.f / (inv_l * s_qsc[n]);
                            const int p = K + base + __popc(mk[i] & lanemask_lt());
                            BD[(size_t)n * ME + p] = fmaf(-sc, dv[j0 + i], s_qn[n] + xn);
                            BS[(size_t)n * ME + p] = gslot;
                        }
                    }
                }
                named_bar_sync(1, TC_EPI);
                // merges: warp ew takes rows n = ew, ew + TC_EW, ...
                const bool last = b + 1 == nblk;
                for (int n = ew; n < m; n += TC_EW) {
                    const int cc = s_cc[n];
                    if (cc == 0 || !(last || cc > CB - TC_M)) continue;
                    float *bd = BD + (size_t)n * ME;
                    int32_t *bs = BS + (size_t)n * ME;
                    const int nb = s_nb[n];
                    if (cc <= 32) warp_sort_merge32<1, KMAX>(bd, bs, K, nb, cc, lane);
                    else if (cc <= 64) warp_sort_merge32<2, KMAX>(bd, bs, K, nb, cc, lane);
                    else if (cc <= 128) warp_sort_merge32<4, KMAX>(bd, bs, K, nb, cc, lane);
                    else
                        warp_select_merge32<KMAX>(
                            bd, bs, K, nb, cc, Hist + ew * 256,
                            reinterpret_cast<float *>(Stg + (size_t)ew * KMAX * 8),
                            reinterpret_cast<int32_t *>(Stg + (size_t)ew * KMAX * 8 + KMAX * 4), lane);
                    const int nb2 = min(K, nb + cc);
                    if (lane == 0) {
                        s_nb[n] = nb2;
                        s_cc[n] = 0;
                        if (nb2 == K && bd[K - 1] < s_kd[n]) {
                            s_kd[n] = bd[K - 1];
                            s_t[n] = s_kd[n] - s_qn[n];
                        }
                    }
                    __syncwarp();
                }
                named_bar_sync(1, TC_EPI);
            }
        }
        gblk += nblk;
        __syncthreads();

        // ---- publish each row's K'-th distance as its query's shared bound
        const int MEo = max(M, ((TC_N * M) / max(m, 1)) & ~7);
        for (int r = tid; r < m; r += TC_NT)
            if (s_nb[r] == K && BD[(size_t)r * MEo + K - 1] >= 0.f)
                atomicMin(reinterpret_cast<int *>(a.thr) + s_qpair[r] / a.P,
                          __float_as_int(BD[(size_t)r * MEo + K - 1]));
        // ---- the best K' of each row (padded with (+inf, -1))
        for (int e = tid; e < m * K; e += TC_NT) {
            const int r = e / K, jj = e % K;
            const int64_t base = ((int64_t)s_qpair[r] * a.CH + chunk) * K;
            const bool ok = jj < s_nb[r];
            a.part_d[base + jj] = ok ? BD[(size_t)r * MEo + jj] : INFINITY;
            a.part_i[base + jj] = ok ? (int64_t)BS[(size_t)r * MEo + jj] : -1;
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tbase, 2 * TC_N);
}

// ---------------------------------------------------------------- re-rank
// One warp per query: exact FP32 direct-form distances of the K' merged
// candidates (global slots) from the FP32 payload, then the best k by
// (distance, id).
template <int E>
__global__ __launch_bounds__(128) void k_rerank(const float *__restrict__ q, int64_t nq, int d,
                                                int Kc, const float *__restrict__ cand_d,
                                                const int64_t *__restrict__ cand_s,
                                                const float *__restrict__ x32,
                                                const int64_t *__restrict__ ids, int k,
                                                float *__restrict__ dist, int64_t *__restrict__ labels)
{
    const int lane = threadIdx.x & 31;
    const int64_t qi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (qi >= nq) return;
    const float *qr = q + (size_t)qi * d;
    float v[E];
    int64_t id[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        v[e] = INFINITY;
        id[e] = -1;
    }
    for (int c = 0; c < Kc; ++c) {
        const int64_t gs = cand_s[qi * Kc + c];
        if (gs < 0 || !(cand_d[qi * Kc + c] < INFINITY)) continue;
        const float *xr = x32 + (size_t)gs * d;
        float acc = 0.f;
        for (int j = lane; j < d; j += 32) {
            const float t = qr[j] - xr[j];
            acc = fmaf(t, t, acc);
        }
        acc = warp_sum(acc);
        const int64_t lab = ids[gs];
        // candidate c lives in register e = c / 32 of lane c % 32
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (c / 32 == e && lane == c % 32) {
                v[e] = acc;
                id[e] = lab;
            }
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
// candidates' exact FP32 direct-form distances into shared memory, then
// the block sorts them by (distance, id) with a bitonic network and writes
// the best k.
constexpr int RR_NT = 256;
constexpr int RR_MAX = 512;
__global__ __launch_bounds__(RR_NT) void k_rerank_wide(const float *__restrict__ q, int64_t nq,
                                                       int d, int Kc,
                                                       const float *__restrict__ cand_d,
                                                       const int64_t *__restrict__ cand_s,
                                                       const float *__restrict__ x32,
                                                       const int64_t *__restrict__ ids, int k,
                                                       float *__restrict__ dist,
                                                       int64_t *__restrict__ labels)
{
    __shared__ float sd[RR_MAX];
    __shared__ int64_t si[RR_MAX];
    const int64_t qi = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t PAD = 0x7fffffffffffffffLL;  // pads sort after every id
    int N = 32;
    while (N < Kc) N <<= 1;
    const float *qr = q + (size_t)qi * d;
    for (int c = warp; c < N; c += RR_NT / 32) {
        float acc = INFINITY;
        int64_t lab = PAD;
        if (c < Kc) {
            const int64_t gs = cand_s[qi * Kc + c];
            if (gs >= 0 && cand_d[qi * Kc + c] < INFINITY) {
                const float *xr = x32 + (size_t)gs * d;
                float a = 0.f;
                for (int j = lane; j < d; j += 32) {
                    const float t = qr[j] - xr[j];
                    a = fmaf(t, t, a);
                }
                acc = warp_sum(a);
                lab = ids[gs];
            }
        }
        if (lane == 0) {
            sd[c] = acc;
            si[c] = lab;
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

// per query: FP32 ||q||^2 and the FP8 inverse scale 448 / (2 max_j |q_j|)
__global__ void k_query_prep(const float *__restrict__ q, int64_t nq, int d,
                             float *__restrict__ qn, float *__restrict__ qsc)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= nq) return;
    const float *qr = q + (size_t)i * d;
    float ss = 0.f, mx = 0.f;
    for (int j = lane; j < d; j += 32) {
        const float v = qr[j];
        ss = fmaf(v, v, ss);
        mx = fmaxf(mx, fabsf(v));
    }
    ss = warp_sum(ss);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        qn[i] = ss;
        qsc[i] = mx > 0.f ? 448.f / (2.f * mx) : 1.f;
    }
}

void query_prep(sivf_index *ix, const float *q, int64_t nq, float *qn, float *qsc,
                cudaStream_t st)
{
    ix->launches += 1;
    k_query_prep<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, st>>>(q, nq, ix->d, qn, qsc);
}

// global slots -> labels (padding stays -1)
__global__ void k_slots_to_ids(int64_t *v, int64_t n, const int64_t *__restrict__ ids)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (v[i] >= 0) v[i] = ids[v[i]];
}

void slots_to_ids(sivf_index *ix, int64_t *v, int64_t n, cudaStream_t st)
{
    ix->launches += 1;
    k_slots_to_ids<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(v, n, ix->ids);
}

// --------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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
    auto enc = encode_fn();
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
    return true;
}

// best K' entries + room for one more tile of candidates
int tc_buf_len(int K) { return (K + TC_M + 7) / 8 * 8; }

// queries per tile of the reduced-precision scan for K' candidates
int tc_tile_queries(int Kc) { return Kc <= TcShape<64>::KMAX ? 64 : 16; }

bool tc_fits(const sivf_index *ix, int Kc)
{
    const int esz = 2;  // the larger of the two formats
    const int KC = (ix->d * esz + 127) / 128;
    if (Kc <= TcShape<64>::KMAX) return tc_smem<64>(KC, tc_buf_len(Kc)).total <= 227 * 1024 - 1024;
    return Kc <= TcShape<16>::KMAX && tc_smem<16>(KC, tc_buf_len(Kc)).total <= 227 * 1024 - 1024;
}

template <int DT, int TN>
static void launch_tc(const unsigned char *tmap, const TcArgs &a, cudaStream_t st)
{
    const size_t smem = tc_smem<TN>(a.KC, a.M).total;
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_scan_tc<DT, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = smem;
    }
    k_scan_tc<DT, TN><<<152, TcShape<TN>::NT, smem, st>>>(
        *reinterpret_cast<const CUtensorMap *>(tmap), a);
}

void scan_lists_tc(sivf_index *ix, int dtype, const float *q, int64_t nq, int P, int Kc,
                   const SearchPlan &pl, const SearchScratch &s, cudaStream_t st)
{
    TcArgs a;
    a.q = q;
    a.nq = nq;
    a.P = P;
    a.K = Kc;
    a.M = tc_buf_len(Kc);
    a.CH = pl.ch;
    a.qlist = s.qlist;
    a.loff = s.loff;
    a.lcnt = s.lcnt;
    a.ibase = s.ibase;
    a.nch = s.nch;
    a.part_d = s.part_d;
    a.part_i = s.part_i;
    a.thr = s.thr;
    a.items = s.items;
    a.qn = s.qn;
    a.qsc = s.qsc;
    a.xnorm = ix->xnorm;
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
    a.KC = (ix->d * esz + 127) / 128;
    a.ctl = ix->ctl;
    a.err = ix->err;
    const bool wide = tc_tile_queries(Kc) == 64;
    const int tok = prof_begin(ix, PROF_SCAN, 1, st);
    if (dtype == SIVF_BF16) {
        if (wide) launch_tc<0, 64>(ix->tmap_bf16, a, st);
        else launch_tc<0, 16>(ix->tmap_bf16, a, st);
    } else {
        if (wide) launch_tc<1, 64>(ix->tmap_fp8, a, st);
        else launch_tc<1, 16>(ix->tmap_fp8, a, st);
    }
    prof_end(ix, tok, st);
}

void rerank(sivf_index *ix, const float *q, int64_t nq, int Kc, const float *cand_d,
            const int64_t *cand_s, int k, float *dist, int64_t *labels, cudaStream_t st)
{
    const int64_t blocks = (nq * 32 + 127) / 128;
    const int tok = prof_begin(ix, PROF_RERANK, 1, st);
#define SIVF_RERANK(E_)                                                                  \
    k_rerank<E_><<<(unsigned)blocks, 128, 0, st>>>(q, nq, ix->d, Kc, cand_d, cand_s, ix->x32, \
                                                   ix->ids, k, dist, labels)
    if (Kc <= 32) SIVF_RERANK(1);
    else if (Kc <= 64) SIVF_RERANK(2);
    else if (Kc <= 128) SIVF_RERANK(4);
    else
        k_rerank_wide<<<(unsigned)nq, RR_NT, 0, st>>>(q, nq, ix->d, Kc, cand_d, cand_s, ix->x32,
                                                      ix->ids, k, dist, labels);
#undef SIVF_RERANK
    prof_end(ix, tok, st);
}

}  // namespace sivf
