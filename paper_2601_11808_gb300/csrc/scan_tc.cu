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

constexpr int TC_N = 64;        // queries per tile (MMA N)
constexpr int TC_M = 128;       // rows per A tile (MMA M)
constexpr int TC_NT = 256;
constexpr int TC_DMP = TC_M + 4;  // padded row of the distance matrix

struct TcArgs {
    const float *q;
    int64_t nq;
    int P, K, M, CH;
    const int32_t *qlist, *loff, *lcnt, *ibase, *nch;
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

struct TcSmem {
    size_t a, b, dm, bd, bs, gs, misc, total;
};
__host__ __device__ inline TcSmem tc_smem(int KC, int M)
{
    TcSmem s;
    s.a = 0;                                            // 2 stages x KC x 16 KB
    s.b = s.a + (size_t)2 * KC * TC_M * 128;            // KC x 64 rows x 128 B
    s.dm = s.b + (size_t)KC * TC_N * 128;
    s.bd = s.dm + (size_t)TC_N * TC_DMP * 4;
    s.bs = s.bd + (size_t)TC_N * M * 4;
    s.gs = s.bs + (size_t)TC_N * M * 4;
    s.misc = s.gs + (size_t)TC_M * 4;
    s.total = s.misc + 1024 + 1024;                     // + base alignment slack
    return s;
}

// rank merge for (distance, 32-bit slot) entries, as warp_rank_merge
template <int EPL>
__device__ __forceinline__ void rank_merge32(float *bd, int32_t *bs, int K, int nb, int nc,
                                             int lane)
{
    const int n = nb + nc;
    float vd[EPL];
    int32_t vs[EPL];
    int pos[EPL];
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
        const int e = lane + 32 * t;
        pos[t] = K;
        if (e >= n) continue;
        const int src = e < nb ? e : K + (e - nb);
        const float dv = bd[src];
        const int32_t sv = bs[src];
        vd[t] = dv;
        vs[t] = sv;
        int r = 0;
        for (int j = 0; j < nc; ++j) {
            const float cd = bd[K + j];
            r += cd < dv || (cd == dv && bs[K + j] < sv);
        }
        if (e < nb) {
            r += e;
        } else {
            int lo = 0, hi = nb;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (bd[mid] < dv || (bd[mid] == dv && bs[mid] < sv)) lo = mid + 1;
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
            bs[pos[t]] = vs[t];
        }
    __syncwarp();
}

template <int DT>  // 0 = BF16, 1 = FP8 E4M3
__global__ __launch_bounds__(TC_NT, 1) void k_scan_tc(const __grid_constant__ CUtensorMap tmap,
                                                      TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled operand tiles
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int KC = a.KC, M = a.M, K = a.K, C = a.C, d = a.d;
    const TcSmem L = tc_smem(KC, M);
    unsigned char *A = smem + L.a;
    unsigned char *B = smem + L.b;
    float *Dm = reinterpret_cast<float *>(smem + L.dm);
    float *BD = reinterpret_cast<float *>(smem + L.bd);
    int32_t *BS = reinterpret_cast<int32_t *>(smem + L.bs);
    int32_t *Gs = reinterpret_cast<int32_t *>(smem + L.gs);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.misc);
    uint64_t *full = bars, *empty = bars + 2, *tfull = bars + 4, *tempty = bars + 6;
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(bars + 8);
    int *s_item = reinterpret_cast<int *>(bars + 9);
    int *s_abort = s_item + 1;
    __shared__ int32_t s_qpair[TC_N], s_cc[TC_N], s_nb[TC_N], s_ks[TC_N];
    __shared__ float s_kd[TC_N], s_qn[TC_N], s_qsc[TC_N];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int ESZ = DT == 0 ? 2 : 1;
    constexpr int EPC = 128 / ESZ;  // elements per 128-byte chunk
    const int SPB = TC_M / C;       // slabs per A tile
    const uint32_t idesc = DT == 0 ? mma_idesc(1, 1, TC_M, TC_N) : mma_idesc(0, 0, TC_M, TC_N);

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 128);
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

        int lo = 0, hi = a.L;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.ibase[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int l = lo;
        const int nc_l = a.nch[l];
        const int rel = item - a.ibase[l];
        const int tile = rel / nc_l, chunk = rel % nc_l;
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
        const int32_t *dirl = a.dir + (size_t)l * a.dir_cap + s0;
        const float inv_l = DT == 1 ? a.inv_scale8[l] : 1.f;

        // ---- query tile: norms, thresholds, B operand (rounded, swizzled)
        const int qb = a.loff[l] + r0;
        for (int r = tid; r < TC_N; r += TC_NT) {
            const int pr = r < m ? a.qlist[qb + r] : -1;
            s_qpair[r] = pr;
            s_cc[r] = 0;
            s_nb[r] = 0;
            s_kd[r] = pr >= 0 ? __ldcg(a.thr + pr / a.P) : INFINITY;
            s_ks[r] = 0x7fffffff;
        }
        __syncthreads();
        // one warp per row: FP32 norm and (FP8) the query's inverse scale
        for (int r = warp; r < TC_N; r += TC_NT / 32) {
            const int pr = s_qpair[r];
            float ss = 0.f, mx = 0.f;
            if (pr >= 0) {
                const float *qr = a.q + (size_t)(pr / a.P) * d;
                for (int j = lane; j < d; j += 32) {
                    const float v = qr[j];
                    ss = fmaf(v, v, ss);
                    mx = fmaxf(mx, fabsf(v));
                }
            }
            ss = warp_sum(ss);
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) {
                s_qn[r] = ss;
                s_qsc[r] = mx > 0.f ? 448.f / (2.f * mx) : 1.f;
            }
        }
        __syncthreads();
        for (int e = tid; e < TC_N * KC * 8; e += TC_NT) {
            const int r = e / (KC * 8), kc = (e / 8) % KC, c = e % 8;
            const int pr = s_qpair[r];
            const int k0 = kc * EPC + c * (16 / ESZ);
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (pr >= 0) {
                const float *qr = a.q + (size_t)(pr / a.P) * d;
                if (DT == 0) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int k = k0 + 2 * t;
                        const float x0 = k < d ? qr[k] : 0.f, x1 = k + 1 < d ? qr[k + 1] : 0.f;
                        __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                        w[t] = *reinterpret_cast<uint32_t *>(&h);
                    }
                } else {
                    const float sc = s_qsc[r];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int k = k0 + 4 * t;
                        float2 p0 = make_float2(k < d ? __fmul_rn(qr[k], sc) : 0.f,
                                                k + 1 < d ? __fmul_rn(qr[k + 1], sc) : 0.f);
                        float2 p1 = make_float2(k + 2 < d ? __fmul_rn(qr[k + 2], sc) : 0.f,
                                                k + 3 < d ? __fmul_rn(qr[k + 3], sc) : 0.f);
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
                const uint32_t g = gblk + b, st = g & 1, u = g >> 1;
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
                const uint32_t g = gblk + b, st = g & 1, buf = g & 1, u = g >> 1;
                if (!mbar_wait_bounded(&full[st], u & 1, a.err)) {
                    *s_abort = 1;
                    break;
                }
                if (u >= 1 && !mbar_wait_bounded(&tempty[buf], (u - 1) & 1, a.err)) {
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
            const int ew = warp - 4;          // epilogue warp = TMEM lane quarter
            const int v = ew * 32 + lane;     // A row = vector of the tile
            for (int b = 0; b < nblk; ++b) {
                const uint32_t g = gblk + b, buf = g & 1, u = g >> 1;
                bool ok = !*s_abort && mbar_wait_bounded(&tfull[buf], u & 1, a.err);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-aligned
                if (!ok) *s_abort = 1;
                tc_fence_after();
                float dv[TC_N];
                if (ok) {
#pragma unroll
                    for (int c16 = 0; c16 < TC_N / 16; ++c16) {
                        float t[16];
                        tmem_ld16(tbase + buf * TC_N + c16 * 16 + ((uint32_t)(ew * 32) << 16), t);
#pragma unroll
                        for (int i = 0; i < 16; ++i) dv[c16 * 16 + i] = t[i];
                    }
                    tmem_ld_wait();
                }
                tc_fence_before();
                mbar_arrive(&tempty[buf]);
                // row metadata
                const int nsl = min(SPB, ns - b * SPB);
                const int j = v / C, slot = v % C;
                int s = -1;
                bool live = false;
                if (ok && j < nsl) {
                    s = dirl[b * SPB + j];
                    if (s >= 0 && s < a.n_slabs)
                        live = (__ldg(a.bits + (size_t)s * (C / 32) + (slot >> 5)) >> (slot & 31)) & 1u;
                }
                const float xn = live ? __ldg(a.xnorm + (size_t)s * C + slot) : 0.f;
                Gs[v] = live ? s * C + slot : -1;
#pragma unroll
                for (int n = 0; n < TC_N; ++n) {
                    float dist = INFINITY;
                    if (live) {
                        const float sc = DT == 0 ? 2.f : 2.f / (inv_l * s_qsc[n]);
                        dist = fmaf(-sc, dv[n], s_qn[n] + xn);
                    }
                    Dm[n * TC_DMP + v] = dist;
                }
                named_bar_sync(1, 128);
                // selection: warp ew takes rows n = ew, ew + 4, ...
                const bool last = b + 1 == nblk;
                const int CB = M - K;
                for (int n = ew; n < m; n += 4) {
                    const float kd = s_kd[n];
                    const int32_t ks = s_ks[n];
                    float *bd = BD + (size_t)n * M;
                    int32_t *bs = BS + (size_t)n * M;
                    int cc = s_cc[n];
#pragma unroll
                    for (int t = 0; t < TC_M / 32; ++t) {
                        const int row = lane + 32 * t;
                        const float dd = Dm[n * TC_DMP + row];
                        const int32_t gs = Gs[row];
                        const bool take = gs >= 0 && (dd < kd || (dd == kd && gs < ks));
                        const uint32_t mk = __ballot_sync(0xffffffffu, take);
                        if (take) {
                            const int p = cc + __popc(mk & lanemask_lt());
                            bd[K + p] = dd;
                            bs[K + p] = gs;
                        }
                        cc += __popc(mk);
                    }
                    __syncwarp();
                    if (cc > 0 && (last || cc > CB - TC_M)) {
                        const int nb = s_nb[n];
                        if (nb + cc <= 128) rank_merge32<4>(bd, bs, K, nb, cc, lane);
                        else rank_merge32<8>(bd, bs, K, nb, cc, lane);
                        const int nb2 = min(K, nb + cc);
                        cc = 0;
                        if (lane == 0) {
                            s_nb[n] = nb2;
                            float nkd = kd;
                            int32_t nks = ks;
                            const int q = s_qpair[n] / a.P;
                            if (nb2 == K && (bd[K - 1] < nkd || (bd[K - 1] == nkd && bs[K - 1] < nks))) {
                                nkd = bd[K - 1];
                                nks = bs[K - 1];
                                if (nkd >= 0.f)
                                    atomicMin(reinterpret_cast<int *>(a.thr) + q, __float_as_int(nkd));
                            }
                            const float gthr = __ldcg(a.thr + q);
                            if (gthr < nkd) {
                                nkd = gthr;
                                nks = 0x7fffffff;
                            }
                            s_kd[n] = nkd;
                            s_ks[n] = nks;
                        }
                    }
                    if (lane == 0) s_cc[n] = cc;
                    __syncwarp();
                }
                named_bar_sync(1, 128);
            }
        }
        gblk += nblk;
        __syncthreads();

        // ---- the best K' of each row (padded with (+inf, -1))
        for (int e = tid; e < m * K; e += TC_NT) {
            const int r = e / K, jj = e % K;
            const int64_t base = ((int64_t)s_qpair[r] * a.CH + chunk) * K;
            const bool ok = jj < s_nb[r];
            a.part_d[base + jj] = ok ? BD[(size_t)r * M + jj] : INFINITY;
            a.part_i[base + jj] = ok ? (int64_t)BS[(size_t)r * M + jj] : -1;
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

// best K' entries + room for one more tile of candidates, at most 256 (the
// rank merge's capacity) for K' <= 128
int tc_buf_len(int K) { return (K + TC_M + 63) / 64 * 64; }

bool tc_fits(const sivf_index *ix, int Kc)
{
    const int esz = 2;  // the larger of the two formats
    const int KC = (ix->d * esz + 127) / 128;
    return Kc <= 128 && tc_smem(KC, tc_buf_len(Kc)).total <= 227 * 1024 - 1024;
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
    const size_t smem = tc_smem(a.KC, a.M).total;
    const int tok = prof_begin(ix, PROF_SCAN, 1, st);
    if (dtype == SIVF_BF16) {
        static size_t attr = 0;
        if (smem > attr) {
            cudaFuncSetAttribute(k_scan_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = smem;
        }
        k_scan_tc<0><<<152, TC_NT, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(ix->tmap_bf16), a);
    } else {
        static size_t attr = 0;
        if (smem > attr) {
            cudaFuncSetAttribute(k_scan_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = smem;
        }
        k_scan_tc<1><<<152, TC_NT, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(ix->tmap_fp8), a);
    }
    prof_end(ix, tok, st);
}

void rerank(sivf_index *ix, const float *q, int64_t nq, int Kc, const float *cand_d,
            const int64_t *cand_s, int k, float *dist, int64_t *labels, cudaStream_t st)
{
    const int64_t blocks = (nq * 32 + 127) / 128;
    const int tok = prof_begin(ix, PROF_RERANK, 1, st);
    if (Kc <= 32)
        k_rerank<1><<<(unsigned)blocks, 128, 0, st>>>(q, nq, ix->d, Kc, cand_d, cand_s, ix->x32,
                                                      ix->ids, k, dist, labels);
    else if (Kc <= 64)
        k_rerank<2><<<(unsigned)blocks, 128, 0, st>>>(q, nq, ix->d, Kc, cand_d, cand_s, ix->x32,
                                                      ix->ids, k, dist, labels);
    else
        k_rerank<4><<<(unsigned)blocks, 128, 0, st>>>(q, nq, ix->d, Kc, cand_d, cand_s, ix->x32,
                                                      ix->ids, k, dist, labels);
    prof_end(ix, tok, st);
}

}  // namespace sivf
