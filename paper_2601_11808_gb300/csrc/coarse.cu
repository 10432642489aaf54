// Coarse quantizer of the index (Sec. 3.3, "the coarse lists returned by
// the quantizer"): nearest centroid for insert (A1) and the nprobe nearest
// centroids for search (A4).
//
// The result must equal the FP64 definition  argmin_c sum_j (x_j - c_j)^2
// (ties to the lowest index) bit for bit.  The fast part is an FP32 GEMM
//     Dt[i][c] = fl(||c||^2 - 2 x_i.c)
// which differs from the exact  Q = ||c||^2 - 2 x.c  (= D - ||x||^2) by at
// most
//     E = 2 * ( u (fl||c||^2 + |Dt|) + 2 gamma_d ||x|| ||c|| )
// (u = 2^-24, gamma_d = d u / (1 - d u); the dot product error of any
// summation order is gamma_d sum_j |x_j c_j| <= gamma_d ||x|| ||c||; the
// factor 2 covers the roundings of the bound arithmetic itself).  The
// selection then works on intervals [Dt - E, Dt + E]:
//   T  = the P-th smallest upper bound,
//   S  = { c : lower bound <= T }         (contains the whole top-P set),
//   c in S is *sure* when UB_c <= T and fewer than P others have a lower
//   bound <= UB_c; the remaining places go to the best of the other members
//   of S by their FP64 distance, computed in the same order and with the
//   same roundings as the definition (no fused multiply-add).
// Only near-ties ever reach the FP64 step.
//
// For assignment (P = 1) with d % 16 == 0 the distances of the first stage
// come from a BF16 tensor-core GEMM instead (tcgen05.mma, FP32
// accumulation): the same
// selection then runs twice.  With the bound of the BF16 stage (rounding of
// x and c to BF16 plus the accumulation) it keeps the lists S_b that can
// still be among the top P; their distances are recomputed in FP32 and the
// selection above runs on S_b with the FP32 bound.  Lists outside S_b have
// exact distances above the P-th smallest, so the result is the same set.
#include <float.h>
#include <math.h>

#include <cmath>

#include "device_utils.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace sivf {

// ------------------------------------------------------------ centroid prep
__global__ void k_centroid_norms(const float *__restrict__ cent, int L, int d,
                                 float *__restrict__ cn, float *__restrict__ cnrm_up,
                                 float *__restrict__ inv_scale8, uint16_t *__restrict__ cb,
                                 uint16_t *__restrict__ clo)
{
    pdl_begin();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L) return;
    const float *v = cent + (size_t)c * d;
    double s = 0.0, mx = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)v[j];
        s = __dadd_rn(s, __dmul_rn(t, t));
        mx = fmax(mx, fabs(t));
    }
    cn[c] = __double2float_rn(s);
    cnrm_up[c] = __double2float_ru(sqrt(s) * (1.0 + 1e-12));
    if (cb)
        for (int j = 0; j < d; ++j) {
            const __nv_bfloat16 h = __float2bfloat16_rn(v[j]);
            cb[(size_t)c * d + j] = *reinterpret_cast<const uint16_t *>(&h);
            if (clo) {
                const __nv_bfloat16 l = __float2bfloat16_rn(v[j] - __bfloat162float(h));
                clo[(size_t)c * d + j] = *reinterpret_cast<const uint16_t *>(&l);
            }
        }
    (void)mx;
}

// ----------------------------------------------------- FP32 tile GEMM (SIMT)
// out[i][c] = fl(cn[c] - 2 * sum_j x[i][j] * cent[c][j]) for i < m, c < L.
// 128 x 128 tiles, 256 threads, 8 x 8 outputs per thread, k-tiles of 16.
constexpr int GBM = 128, GBN = 128, GBK = 16;

__global__ __launch_bounds__(256) void k_coarse_gemm(const float *__restrict__ x, int m,
                                                     int d, const float *__restrict__ cent,
                                                     const float *__restrict__ cn, int L,
                                                     float *__restrict__ out)
{
    pdl_begin();
    __shared__ __align__(16) float As[GBK][GBM];
    __shared__ __align__(16) float Bs[GBK][GBN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * GBM, col0 = blockIdx.x * GBN;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < d; k0 += GBK) {
        for (int e = tid; e < GBM * GBK / 4; e += 256) {
            int r = e / (GBK / 4), c4 = e % (GBK / 4);
            int gk = k0 + c4 * 4;
            int gr = row0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < m && gk < d) v = *reinterpret_cast<const float4 *>(x + (size_t)gr * d + gk);
            As[c4 * 4 + 0][r] = v.x;
            As[c4 * 4 + 1][r] = v.y;
            As[c4 * 4 + 2][r] = v.z;
            As[c4 * 4 + 3][r] = v.w;
            int gc = col0 + r;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gc < L && gk < d) w = *reinterpret_cast<const float4 *>(cent + (size_t)gc * d + gk);
            Bs[c4 * 4 + 0][r] = w.x;
            Bs[c4 * 4 + 1][r] = w.y;
            Bs[c4 * 4 + 2][r] = w.z;
            Bs[c4 * 4 + 3][r] = w.w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
            float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int c = col0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
            if (c < L) out[(size_t)r * L + c] = fmaf(-2.f, acc[i][j], cn[c]);
        }
    }
}

// ------------------------------------------------------- exact selection
constexpr int SEL_NT = 256;
constexpr int SEL_SCAP = 1024;   // candidate capacity before the slow path

struct SelArgs {
    const float *D;        // [m, L] approximate distances (row stride L)
    int m, L, P, d;
    const float *x;        // [m, d] rows being assigned / queries
    const float *cent;     // [L, d]
    const float *cn;       // [L]
    const float *cnrm_up;  // [L]
    float gamma2;          // 2 * gamma_d
    float gamma2_first;    // the same factor for the first-stage distances D
    int two_level;         // D is the BF16 tensor-core stage: recheck S in FP32
    const int32_t *S;      // instead of D: per-row candidate lists of the fused
    int s_stride;          // first stage ([n, lists...], n = -1: redo the row)
    const int32_t *hard;   // the rows the fused first stage left undecided
    const int *nhard;      // (their number, on the device)
    int32_t *out;          // [m, P]
    uint32_t *err;
};

// FP64 distance in the order and with the roundings of the definition
__device__ __forceinline__ double exact_dist(const float *__restrict__ a,
                                             const float *__restrict__ b, int d)
{
    double acc = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = __dsub_rn((double)a[j], (double)b[j]);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    return acc;
}

// Bound E of |Dt - Q|.  Written with explicit-rounding intrinsics so that
// every evaluation for the same inputs gives the same bits (no contraction).
__device__ __forceinline__ float bound_of(float Dt, float cnc, float cnrm, float xn,
                                          float gamma2)
{
    const float u = 5.9604645e-08f;  // 2^-24
    float t1 = __fmul_rn(u, __fadd_rn(cnc, fabsf(Dt)));
    float t2 = __fmul_rn(__fmul_rn(gamma2, xn), cnrm);
    return __fadd_rn(__fmul_rn(2.f, __fadd_rn(t1, t2)), 1e-30f);
}
__device__ __forceinline__ float upper_of(float Dt, float E) { return __fadd_rn(Dt, E); }
__device__ __forceinline__ float lower_of(float Dt, float E) { return __fsub_rn(Dt, E); }

// block-wide helpers for SEL_NT threads
__device__ float block_min(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < SEL_NT / 32 ? red[l] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    float r = red[0];
    __syncthreads();
    return r;
}

__global__ __launch_bounds__(SEL_NT) void k_coarse_select(SelArgs a)
{
    pdl_begin();
    const int row = blockIdx.x;
    if (row >= a.m) return;
    const int tid = threadIdx.x;
    const float *Dr = a.D + (size_t)row * a.L;
    const float *xr = a.x + (size_t)row * a.d;

    __shared__ float red[32];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_rank;
    __shared__ int s_ns, s_nsel;
    __shared__ float sLB[SEL_SCAP], sUB[SEL_SCAP];
    __shared__ int sIdx[SEL_SCAP];
    __shared__ unsigned char sSure[SEL_SCAP];
    __shared__ double sDx[SEL_SCAP];
    __shared__ int sSel[kMaxK];

    // ||x|| upper bound from an FP64 sum
    double part = 0.0;
    for (int j = tid; j < a.d; j += SEL_NT) part += (double)xr[j] * (double)xr[j];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __shared__ double dred[SEL_NT / 32];
    if ((tid & 31) == 0) dred[tid >> 5] = part;
    __syncthreads();
    double xs = 0.0;
    for (int w = 0; w < SEL_NT / 32; ++w) xs += dred[w];
    const float xn = __double2float_ru(sqrt(xs) * (1.0 + 1e-12));

    // T = P-th smallest upper bound
    float T;
    if (a.P == 1) {
        float v = INFINITY;
        for (int c = tid; c < a.L; c += SEL_NT) {
            float Dt = Dr[c];
            v = fminf(v, upper_of(Dt, bound_of(Dt, a.cn[c], a.cnrm_up[c], xn, a.gamma2)));
        }
        T = block_min(v, red);
    } else {
        if (tid == 0) {
            s_prefix = 0;
            s_rank = (uint32_t)a.P;
        }
        uint32_t mask = 0;
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 24 - 8 * pass;
            hist[tid] = 0;  // SEL_NT == 256 bins
            __syncthreads();
            const uint32_t prefix = s_prefix;
            for (int c = tid; c < a.L; c += SEL_NT) {
                float Dt = Dr[c];
                uint32_t k = fkey(upper_of(Dt, bound_of(Dt, a.cn[c], a.cnrm_up[c], xn, a.gamma2)));
                if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid < 32) {
                // lane l owns bins 8l .. 8l+7
                uint32_t loc[8], s = 0;
                for (int b = 0; b < 8; ++b) {
                    loc[b] = hist[tid * 8 + b];
                    s += loc[b];
                }
                uint32_t incl = s;
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (tid >= o) incl += t;
                }
                uint32_t excl = incl - s, need = s_rank;
                bool mine = excl < need && incl >= need;
                if (mine) {
                    uint32_t cum = excl;
                    for (int b = 0; b < 8; ++b) {
                        if (cum + loc[b] >= need) {
                            s_prefix = prefix | ((uint32_t)(tid * 8 + b) << shift);
                            s_rank = need - cum;
                            break;
                        }
                        cum += loc[b];
                    }
                }
            }
            mask |= 255u << shift;
            __syncthreads();
        }
        T = fkey_inv(s_prefix);
    }

    // candidate set S
    if (tid == 0) {
        s_ns = 0;
        s_nsel = 0;
    }
    __syncthreads();
    for (int c = tid; c < a.L; c += SEL_NT) {
        float Dt = Dr[c];
        float E = bound_of(Dt, a.cn[c], a.cnrm_up[c], xn, a.gamma2);
        if (lower_of(Dt, E) <= T) {
            int p = atomicAdd(&s_ns, 1);
            if (p < SEL_SCAP) {
                sLB[p] = lower_of(Dt, E);
                sUB[p] = upper_of(Dt, E);
                sIdx[p] = c;
            }
        }
    }
    __syncthreads();
    const int ns = s_ns;
    int32_t *outr = a.out + (size_t)row * a.P;

    if (ns <= SEL_SCAP) {
        // sure members
        for (int p = tid; p < ns; p += SEL_NT) {
            float ub = sUB[p];
            int cnt = 0;
            for (int q = 0; q < ns; ++q) cnt += (q != p && sLB[q] <= ub);
            bool sure = ub <= T && cnt < a.P;
            sSure[p] = sure;
            if (sure) {
                int s = atomicAdd(&s_nsel, 1);
                if (s < kMaxK) sSel[s] = sIdx[p];
            }
        }
        __syncthreads();
        const int nsure = s_nsel;
        const int r = a.P - nsure;
        if (r > 0) {
            // boundary members: exact FP64 distances, then rank among them
            const int nb = ns - nsure;
            if (nb > r) {
                for (int p = tid; p < ns; p += SEL_NT)
                    if (!sSure[p]) sDx[p] = exact_dist(xr, a.cent + (size_t)sIdx[p] * a.d, a.d);
                __syncthreads();
            }
            for (int p = tid; p < ns; p += SEL_NT) {
                if (sSure[p]) continue;
                bool take = true;
                if (nb > r) {
                    const double Dc = sDx[p];
                    const int c = sIdx[p];
                    int rank = 0;
                    for (int q = 0; q < ns; ++q) {
                        if (q == p || sSure[q]) continue;
                        rank += (sDx[q] < Dc || (sDx[q] == Dc && sIdx[q] < c));
                    }
                    take = rank < r;
                }
                if (take) {
                    int s = atomicAdd(&s_nsel, 1);
                    if (s < kMaxK) sSel[s] = sIdx[p];
                }
            }
        }
        __syncthreads();
    } else if (tid == 0) {
        // pathological: more than SEL_SCAP candidates (e.g. many identical
        // centroids).  Exact FP64 selection by insertion into a sorted
        // array of P (distance, index) pairs, scanning lists in index order.
        double *hd = sDx;  // P <= SEL_SCAP entries
        int n = 0;
        for (int c = 0; c < a.L; ++c) {
            float Dt = Dr[c];
            float E = bound_of(Dt, a.cn[c], a.cnrm_up[c], xn, a.gamma2);
            if (lower_of(Dt, E) > T) continue;
            double Dc = exact_dist(xr, a.cent + (size_t)c * a.d, a.d);
            if (n == a.P && !(Dc < hd[n - 1])) continue;  // index order keeps ties
            int pos = n < a.P ? n : a.P - 1;
            while (pos > 0 && Dc < hd[pos - 1]) {
                hd[pos] = hd[pos - 1];
                sSel[pos] = sSel[pos - 1];
                --pos;
            }
            hd[pos] = Dc;
            sSel[pos] = c;
            if (n < a.P) ++n;
        }
        s_nsel = n;
    }
    __syncthreads();

    // write the selected set nearest first: ascending approximate distance,
    // ties to the lower list index (the set itself is the exact one)
    const int nsel = min(s_nsel, a.P);
    if (s_nsel != a.P && tid == 0) atomicOr(a.err, ERR_SELECT);
    for (int s = tid; s < a.P; s += SEL_NT) {
        if (s >= nsel) {
            outr[s] = -1;
            continue;
        }
        const int c = sSel[s];
        const float dc = Dr[c];
        int pos = 0;
        for (int q = 0; q < nsel; ++q) {
            const int c2 = sSel[q];
            const float d2 = Dr[c2];
            pos += d2 < dc || (d2 == dc && c2 < c);
        }
        outr[pos] = c;
    }
}

// ------------------------------------------ BF16 tensor-core first stage
// out[i][c] = fl(cn[c] - 2 * acc[i][c]) with, accumulated in FP32 by
// tcgen05.mma,
//   SPLIT = 1:  acc = sum_j bf16(x_ij) bf16(c_cj)
//   SPLIT = 3:  acc = sum_j xh xh' ... the three leading products of
//               x = xh + xl, c = ch + cl (xh = bf16(x), xl = bf16(x - xh),
//               likewise c): xh ch + xh cl + xl ch.
// One CTA: 128 rows of x (rounded, split and swizzled by its threads)
// against 256 centroids (BF16 rows copied with cp.async), K = d (d % 16 ==
// 0), accumulator in 256 TMEM columns; four warps read their TMEM lane
// quarter back.
constexpr int CT_M = 128, CT_N = 256;
constexpr int CT_NT = 256;  // threads: 8 warps, two per TMEM lane quarter in the epilogue
constexpr int CT_AU = 4;    // A chunks each thread loads before converting

__host__ __device__ inline size_t coarse_tc_smem(int d, int split)
{
    const int KC = (d * 2 + 127) / 128;
    return (size_t)(split == 3 ? 2 : 1) * KC * (CT_M + CT_N) * 128 + 1024;
}

__device__ __forceinline__ void cp_async16_c(void *dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

template <int SPLIT>
__global__ __launch_bounds__(CT_NT, 1) void k_coarse_tc(const float *__restrict__ x, int m, int d,
                                                        const uint16_t *__restrict__ cb,
                                                        const uint16_t *__restrict__ clo,
                                                        const float *__restrict__ cn, int L,
                                                        float *__restrict__ out, uint32_t *err)
{
    pdl_begin();
    constexpr int NP = SPLIT == 3 ? 2 : 1;  // hi (and lo) parts
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int KC = (d * 2 + 127) / 128;
    unsigned char *A = smem;                                // NP x KC x 128 rows x 128 B
    unsigned char *B = smem + (size_t)NP * KC * CT_M * 128;  // NP x KC x 256 rows x 128 B
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * CT_M, col0 = blockIdx.y * CT_N;
    const int ncol = min(CT_N, L - col0);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, CT_N);
    // B: BF16 centroid rows; chunks past L or d are zero
    for (int pp = 0; pp < NP; ++pp) {
        const uint16_t *src0 = pp ? clo : cb;
        unsigned char *Bp = B + (size_t)pp * KC * CT_N * 128;
        for (int e = tid; e < CT_N * KC * 8; e += CT_NT) {
            const int r = e / (KC * 8), kc = (e >> 3) % KC, c = e & 7;
            const int k0 = kc * 64 + c * 8;  // first element of the 16-byte chunk
            const bool in = col0 + r < L && k0 < d;
            cp_async16_c(Bp + (size_t)kc * CT_N * 128 + (size_t)(r >> 3) * 1024 + (r & 7) * 128 +
                             ((c ^ (r & 7)) << 4),
                         in ? (const void *)(src0 + (size_t)(col0 + r) * d + k0) : (const void *)src0,
                         in ? 16u : 0u);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // A: rows of x rounded to BF16 (round to nearest even); zero past m or d.
    // Each thread loads CT_AU chunks before converting any (loads in flight)
    const int nA = CT_M * KC * 8;
    for (int e0 = tid; e0 < nA; e0 += CT_NT * CT_AU) {
        float4 f0[CT_AU], f1[CT_AU];
#pragma unroll
        for (int u = 0; u < CT_AU; ++u) {
            const int e = e0 + u * CT_NT;
            const int r = e / (KC * 8), kc = (e >> 3) % KC, c = e & 7;
            const int k0 = kc * 64 + c * 8;
            f0[u] = f1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < nA && row0 + r < m && k0 < d) {
                const float4 *xr = reinterpret_cast<const float4 *>(x + (size_t)(row0 + r) * d + k0);
                f0[u] = __ldg(xr);
                f1[u] = __ldg(xr + 1);
            }
        }
#pragma unroll
        for (int u = 0; u < CT_AU; ++u) {
            const int e = e0 + u * CT_NT;
            if (e >= nA) break;
            const int r = e / (KC * 8), kc = (e >> 3) % KC, c = e & 7;
            const float f[8] = {f0[u].x, f0[u].y, f0[u].z, f0[u].w,
                                f1[u].x, f1[u].y, f1[u].z, f1[u].w};
            uint32_t w[4], wl[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * t], f[2 * t + 1]);
                w[t] = *reinterpret_cast<uint32_t *>(&h);
                if (NP == 2) {
                    __nv_bfloat162 l = __floats2bfloat162_rn(f[2 * t] - __low2float(h),
                                                             f[2 * t + 1] - __high2float(h));
                    wl[t] = *reinterpret_cast<uint32_t *>(&l);
                }
            }
            const size_t off = (size_t)kc * CT_M * 128 + (size_t)(r >> 3) * 1024 + (r & 7) * 128 +
                               ((c ^ (r & 7)) << 4);
            *reinterpret_cast<uint4 *>(A + off) = make_uint4(w[0], w[1], w[2], w[3]);
            if (NP == 2)
                *reinterpret_cast<uint4 *>(A + (size_t)KC * CT_M * 128 + off) =
                    make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;
    if (tid == 0) {
        const uint32_t idesc = mma_idesc(1, 1, CT_M, CT_N);
        // products: (x hi, c hi), then for the split (x hi, c lo), (x lo, c hi)
        constexpr int NPROD = SPLIT == 3 ? 3 : 1;
        for (int pr = 0; pr < NPROD; ++pr) {
            const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
            const uint32_t abase = smem_u32(A + (size_t)pa * KC * CT_M * 128);
            const uint32_t bbase = smem_u32(B + (size_t)pb * KC * CT_N * 128);
            for (int kc = 0; kc < KC; ++kc)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_bf16(tbase, smem_desc_sw128(abase + kc * CT_M * 128 + ks * 32, 1024),
                             smem_desc_sw128(bbase + kc * CT_N * 128 + ks * 32, 1024), idesc,
                             (pr | kc | ks) != 0);
        }
        mma_commit(&bar);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar, 0, err));
    tc_fence_after();
    // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +31 (its lane
    // quarter) and every other group of 16 columns, starting at w div 4
    const int q = warp & 3, half = warp >> 2;
    const int r = row0 + q * 32 + lane;
    const bool vec = (L & 3) == 0;
    for (int c16 = half; c16 * 16 < ncol; c16 += CT_NT / 128) {  // warp-uniform
        float v[16];
        if (ok) {
            tmem_ld16(tbase + c16 * 16 + ((uint32_t)(q * 32) << 16), v);
            tmem_ld_wait();
        }
        if (!ok || r >= m) continue;
        const int cb0 = col0 + c16 * 16;
        float *o = out + (size_t)r * L + cb0;
        if (vec && c16 * 16 + 16 <= ncol) {
#pragma unroll
            for (int i4 = 0; i4 < 4; ++i4) {
                const float4 cv = __ldg(reinterpret_cast<const float4 *>(cn + cb0) + i4);
                reinterpret_cast<float4 *>(o)[i4] =
                    make_float4(fmaf(-2.f, v[4 * i4], cv.x), fmaf(-2.f, v[4 * i4 + 1], cv.y),
                                fmaf(-2.f, v[4 * i4 + 2], cv.z), fmaf(-2.f, v[4 * i4 + 3], cv.w));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (c16 * 16 + i < ncol) o[i] = fmaf(-2.f, v[i], __ldg(cn + cb0 + i));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, CT_N);
}

// ------------------------------- fused BF16 first stage for assignment
// P = 1, one CTA per 128 rows of x against ALL centroids, without writing
// the distance matrix.  The BF16 centroids pass in chunks of CT_N = 256 rows
// (TMA boxes of 64 columns x 256 rows, 128-byte swizzle, into two buffers),
// one tcgen05.mma group per chunk into one of two 256-column TMEM buffers,
// so that the MMA of the next step and the copy of the one after run under
// each epilogue.  The chunks pass twice (recomputing a chunk's products
// costs far less than keeping them):
//   pass 1: per row Dmin = min_c Dt_c and A = max_c |Dt_c|.  With
//           Ebig >= E_c for every c (the bound of the selection evaluated
//           at max ||c||^2, A and max ||c||, rounded up), T = Dmin + Ebig
//           (rounded up) is >= the smallest upper bound Dt_c + E_c;
//   pass 2: the lists with lower bound Dt_c - E_c <= T, a superset of the
//           selection's set S.  A list with Dt_c above thr = T + Ebig plus
//           one unit in the last place of T (rounded up) cannot qualify and
//           is rejected by one comparison; the rest take the exact test.
// Pass 1 also keeps the row's second smallest Dt: when it is above thr only
// the argmin can qualify, so the argmin is the answer; a tile whose rows
// are all decided that way skips pass 2.
// A row left with one list has its answer (S holds the nearest list): it
// is written to `out1` directly.  Any other row is appended to `hard` and
// leaves [n, list_0 .. list_{n-1}] for the finishing selection, n = -1 when
// one of its four threads had more than CF_CAP lists (the row is then
// redone from all lists).  ||x|| is bounded from the FP32 sum of squares
// s of the tile's rows (relative error <= d u) as RU(sqrt(RU(s (1 + 4 d u)))).
// One thread issues the copies and MMAs and waits for them; a block barrier
// per step releases the others.
constexpr int CF_CAP = 8;                   // lists per thread
constexpr int CF_SUB = 4;                   // threads per row
constexpr int CF_STRIDE = CF_SUB * CF_CAP + 1;  // ints per row of the output
constexpr int CF_NT = 128 * CF_SUB;

__host__ __device__ inline size_t coarse_fused_smem(int d)
{
    const int KC = (d * 2 + 127) / 128;
    return (size_t)KC * (CT_M + 2 * CT_N) * 128 + (size_t)CF_CAP * CF_NT * 4 + 1024;
}

template <int KC>
__global__ __launch_bounds__(CF_NT, 1) void k_coarse_fused1(
    const __grid_constant__ CUtensorMap tmB, const float *__restrict__ x, int m, int d,
    const float *__restrict__ cn, const float *__restrict__ cnrm_up, int L, float g1,
    int32_t *__restrict__ out1, int32_t *__restrict__ outS, int32_t *__restrict__ hard,
    int *nhard, uint32_t *err)
{
    pdl_begin();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    __shared__ uint64_t fullb[2], mmab[2];
    __shared__ uint32_t tmem_base;
    __shared__ float sxn[CT_M], sMin[CF_SUB][CT_M], sSec[CF_SUB][CT_M], sMax[CF_SUB][CT_M];
    __shared__ int sn[CF_SUB][CT_M], sArg[CF_SUB][CT_M];
    __shared__ uint32_t smax[2];  // max ||c||^2, max ||c|| (bits of non-negative floats)
    constexpr uint32_t BBYTES = KC * CT_N * 128;
    unsigned char *A = smem;                                  // KC x 128 rows x 128 B
    unsigned char *B = smem + (size_t)KC * CT_M * 128;        // 2 x KC x 256 rows x 128 B
    int *rc = reinterpret_cast<int *>(B + 2 * BBYTES);        // [CF_CAP][CF_NT] lists
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, sub = warp >> 2, rloc = q * 32 + lane;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&fullb[i], 1);
            mbar_init(&mmab[i], 1);
        }
        fence_mbar_init();
        smax[0] = smax[1] = 0u;
    }
    if (warp == 0) tmem_alloc(&tmem_base, 2 * CT_N);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    {
        float a0 = 0.f, a1 = 0.f;
        for (int c = tid; c < L; c += CF_NT) {
            a0 = fmaxf(a0, __ldg(cn + c));
            a1 = fmaxf(a1, __ldg(cnrm_up + c));
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0 = fmaxf(a0, __shfl_xor_sync(0xffffffffu, a0, o));
            a1 = fmaxf(a1, __shfl_xor_sync(0xffffffffu, a1, o));
        }
        if (lane == 0) {
            atomicMax(&smax[0], __float_as_uint(a0));
            atomicMax(&smax[1], __float_as_uint(a1));
        }
    }
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = mma_idesc(1, 1, CT_M, CT_N);
    const int nch = (L + CT_N - 1) / CT_N, nsteps = 2 * nch, ntiles = (m + CT_M - 1) / CT_M;
    // thread 0's bookkeeping, bit b for buffer b: phases, and copies / MMAs
    // issued but not waited for
    uint32_t fph = 0u, mph = 0u, fpend = 0u, mpend = 0u;
    bool ok = true;

    auto load_b = [&](int j, int b) {  // chunk j -> B buffer b
        mbar_arrive_expect_tx(&fullb[b], BBYTES);
#pragma unroll
        for (int kc = 0; kc < KC; ++kc)
            tma_load_2d(B + (size_t)b * BBYTES + (size_t)kc * CT_N * 128, &tmB, kc * 64, j * CT_N,
                        &fullb[b]);
        fpend |= 1u << b;
    };
    auto wait_full = [&](int b) {
        const bool g = mbar_wait_bounded(&fullb[b], (fph >> b) & 1u, err);
        fph ^= 1u << b;
        fpend &= ~(1u << b);
        return g;
    };
    auto issue_mma = [&](int b) {  // B buffer b -> TMEM buffer b
        const uint32_t abase = smem_u32(A), bbase = smem_u32(B + (size_t)b * BBYTES);
#pragma unroll
        for (int kc = 0; kc < KC; ++kc)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(tbase + b * CT_N, smem_desc_sw128(abase + kc * CT_M * 128 + ks * 32, 1024),
                         smem_desc_sw128(bbase + kc * CT_N * 128 + ks * 32, 1024), idesc,
                         (kc | ks) != 0);
        mma_commit(&mmab[b]);
        mpend |= 1u << b;
    };
    auto wait_mma = [&](int b) {
        const bool g = mbar_wait_bounded(&mmab[b], (mph >> b) & 1u, err);
        mph ^= 1u << b;
        mpend &= ~(1u << b);
        return g;
    };

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int row0 = tile * CT_M;
        if (tid == 0) {
            load_b(0, 0);
            load_b(1 % nch, 1);
        }
        // A: the tile's rows rounded to BF16, zero past m or d.  The KC * 8
        // chunks of a row sit in consecutive lanes: their sums of squares
        // reduce by shuffles into the row's ||x|| bound
        constexpr int nA = CT_M * KC * 8, W = KC * 8;
        const float fx = 1.f + 4.f * (float)d * 5.9604645e-08f;
        static_assert(nA % CF_NT == 0 || CF_NT % nA == 0, "whole warps per A pass");
        for (int e0 = tid; e0 < nA; e0 += CF_NT * CT_AU) {
            float4 f0[CT_AU], f1[CT_AU];
#pragma unroll
            for (int u = 0; u < CT_AU; ++u) {
                const int e = e0 + u * CF_NT;
                const int r = e / W, kc = (e >> 3) % KC, c = e & 7;
                const int k0 = kc * 64 + c * 8;
                f0[u] = f1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (e < nA && row0 + r < m && k0 < d) {
                    const float4 *xr = reinterpret_cast<const float4 *>(x + (size_t)(row0 + r) * d + k0);
                    f0[u] = __ldg(xr);
                    f1[u] = __ldg(xr + 1);
                }
            }
#pragma unroll
            for (int u = 0; u < CT_AU; ++u) {
                const int e = e0 + u * CF_NT;
                if (e >= nA) break;  // warp-uniform: nA is a multiple of CF_NT / 2
                const int r = e / W, kc = (e >> 3) % KC, c = e & 7;
                const float f[8] = {f0[u].x, f0[u].y, f0[u].z, f0[u].w,
                                    f1[u].x, f1[u].y, f1[u].z, f1[u].w};
                uint32_t w[4];
                float sq = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * t], f[2 * t + 1]);
                    w[t] = *reinterpret_cast<uint32_t *>(&h);
                    sq = fmaf(f[2 * t], f[2 * t], sq);
                    sq = fmaf(f[2 * t + 1], f[2 * t + 1], sq);
                }
                *reinterpret_cast<uint4 *>(A + (size_t)kc * CT_M * 128 + (size_t)(r >> 3) * 1024 +
                                           (r & 7) * 128 + ((c ^ (r & 7)) << 4)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
                for (int o = W >> 1; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
                if ((lane & (W - 1)) == 0) sxn[r] = __fsqrt_ru(__fmul_ru(sq, fx));
            }
        }
        fence_proxy_async_smem();  // A (generic stores) is read by the MMAs
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        bool got = true;  // thread 0: every wait so far succeeded
        if (tid == 0) {
            got = wait_full(0);
            if (got) issue_mma(0);
        }
        const float xn = sxn[rloc];
        // pass 1: smallest, second smallest and largest Dt, the smallest's list
        float d1 = INFINITY, d2 = INFINITY, dmax = -INFINITY, T = INFINITY, thr = -INFINITY;
        int c1 = -1, n = 0;
        bool ovf = false, done = false;
        for (int s = 0; s < nsteps; ++s) {
            const int b = s & 1, j = s % nch;
            if (tid == 0 && got) got = wait_mma(b);
            // MMA s is done and every thread has finished epilogue s - 1
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            tc_fence_after();
            if (tid == 0) {
                if (s + 1 < nsteps) {  // TMEM buffer b ^ 1 is free: MMA s + 1 under this epilogue
                    got = wait_full(b ^ 1);
                    if (got) issue_mma(b ^ 1);
                }
                if (got && s + 2 < nsteps) load_b((s + 2) % nch, b);  // MMA s has read buffer b
            }
            for (int c16 = sub; c16 < CT_N / 16; c16 += CF_SUB) {  // warp-uniform
                const int cb0 = j * CT_N + c16 * 16;
                if (cb0 >= L) break;
                const int nv = min(16, L - cb0);
                float v[16], cv[16];
                tmem_ld16(tbase + b * CT_N + c16 * 16 + ((uint32_t)(q * 32) << 16), v);
                if (nv == 16) {
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4) {
                        const float4 t = __ldg(reinterpret_cast<const float4 *>(cn + cb0) + i4);
                        cv[4 * i4] = t.x;
                        cv[4 * i4 + 1] = t.y;
                        cv[4 * i4 + 2] = t.z;
                        cv[4 * i4 + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) cv[i] = i < nv ? __ldg(cn + cb0 + i) : 0.f;
                }
                tmem_ld_wait(v);
                if (s < nch) {
                    auto see = [&](float Dt, int c) {
                        const bool lt = Dt < d1;
                        d2 = fminf(d2, lt ? d1 : Dt);
                        c1 = lt ? c : c1;
                        d1 = fminf(d1, Dt);
                        dmax = fmaxf(dmax, Dt);
                    };
                    if (nv == 16) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) see(fmaf(-2.f, v[i], cv[i]), cb0 + i);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (i < nv) see(fmaf(-2.f, v[i], cv[i]), cb0 + i);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float Dt = fmaf(-2.f, v[i], cv[i]);
                        if (!(i < nv && Dt <= thr)) continue;
                        const int c = cb0 + i;
                        const float E = bound_of(Dt, cv[i], __ldg(cnrm_up + c), xn, g1);
                        if (!(lower_of(Dt, E) <= T)) continue;
                        if (n < CF_CAP) rc[n * CF_NT + tid] = c;
                        else ovf = true;
                        ++n;
                    }
                }
            }
            if (s == nch - 1) {  // end of pass 1: the row's T and quick-reject threshold
                sMin[sub][rloc] = d1;
                sSec[sub][rloc] = d2;
                sMax[sub][rloc] = dmax;
                sArg[sub][rloc] = c1;
                __syncthreads();
                int kmin = 0;
                float mn = sMin[0][rloc], mx = sMax[0][rloc];
#pragma unroll
                for (int k = 1; k < CF_SUB; ++k) {
                    if (sMin[k][rloc] < mn) kmin = k;
                    mn = fminf(mn, sMin[k][rloc]);
                    mx = fmaxf(mx, sMax[k][rloc]);
                }
                float second = sSec[kmin][rloc];
#pragma unroll
                for (int k = 0; k < CF_SUB; ++k)
                    if (k != kmin) second = fminf(second, sMin[k][rloc]);
                const float ab = fmaxf(fabsf(mn), fabsf(mx));
                // Ebig: the bound at the maxima, every step rounded up, times
                // 1 + 2^-10 (covers the roundings of the bound itself)
                const float t1 = __fmul_ru(5.9604645e-08f, __fadd_ru(__uint_as_float(smax[0]), ab));
                const float t2 = __fmul_ru(__fmul_ru(g1, xn), __uint_as_float(smax[1]));
                const float eb = __fadd_ru(
                    __fmul_ru(__fmul_ru(2.f, __fadd_ru(t1, t2)), 1.f + 1.f / 1024.f), 1e-30f);
                T = __fadd_ru(mn, eb);
                // RN(Dt - E) <= T needs Dt < T + E + ulp(T) <= thr
                thr = __fadd_ru(__fadd_ru(T, eb), __fadd_ru(__fmul_ru(fabsf(T), 1.2e-7f), 1e-30f));
                // decided: no list but the argmin has Dt <= thr
                const bool decided = !(second <= thr) && mn <= thr;
                if (!__syncthreads_or(!decided && row0 + rloc < m)) {
                    if (sub == 0 && row0 + rloc < m) out1[row0 + rloc] = sArg[kmin][rloc];
                    if (tid == 0)  // the pass-2 copy and MMA already issued are waited for
                        for (int i = 0; i < 2; ++i) {
                            if ((fpend >> i) & 1u) got &= wait_full(i);
                            if ((mpend >> i) & 1u) got &= wait_mma(i);
                        }
                    done = true;
                    break;
                }
            }
            tc_fence_before();
        }
        if (!ok) break;
        if (done) {
            if (__syncthreads_or(!got)) ok = false;  // a drain wait ran out
            continue;                                // sMin ... are rewritten after a barrier
        }
        sn[sub][rloc] = ovf ? -1 : n;
        __syncthreads();
        const int r = row0 + rloc;
        if (r < m) {
            int32_t *o = outS + (size_t)r * CF_STRIDE;
            int before = 0, total = 0;
            bool bad = false;
#pragma unroll
            for (int k = 0; k < CF_SUB; ++k) {
                const int nk = sn[k][rloc];
                bad |= nk < 0;
                before += k < sub ? nk : 0;
                total += nk;
            }
            if (!bad && total == 1) {
                if (n == 1) out1[r] = rc[tid];
            } else {
                if (bad) {
                    if (sub == 0) o[0] = -1;
                } else {
                    for (int k = 0; k < n; ++k) o[1 + before + k] = rc[k * CF_NT + tid];
                    if (sub == 0) o[0] = total;
                }
                if (sub == 0) hard[atomicAdd(nhard, 1)] = r;
            }
        }
        __syncthreads();  // sxn, sMin, sMax, sn, the lists and A are reused by the next tile
    }
    if (!ok) {
        // a wait ran out: thread 0 waits (bounded) for its copies and MMAs
        // still in flight; every row of this CTA's tiles goes to the full
        // selection
        if (tid == 0)
            for (int i = 0; i < 2; ++i) {
                if ((fpend >> i) & 1u) wait_full(i);
                if ((mpend >> i) & 1u) wait_mma(i);
            }
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
            for (int r = tile * CT_M + tid; r < min(m, tile * CT_M + CT_M); r += CF_NT) {
                outS[(size_t)r * CF_STRIDE] = -1;
                hard[atomicAdd(nhard, 1)] = r;
            }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, 2 * CT_N);
}

// TMA descriptor of the BF16 centroids for the fused first stage: boxes of
// 64 columns x CT_N rows, 128-byte swizzle; rows past nlist read as zero.
bool coarse_make_map(sivf_index *ix)
{
    const int d = ix->d;
    if (!ix->cent_bf16 || d < 64 || d > 128 || d % 16) return false;
    auto enc = tmap_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)ix->nlist};
    cuuint64_t strides[1] = {(cuuint64_t)d * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)CT_N};
    cuuint32_t es[2] = {1, 1};
    return enc(reinterpret_cast<CUtensorMap *>(ix->tmap_cent), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               ix->cent_bf16, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ----------------------------------------------- warp-per-row selection
// The same selection for P <= CW_PMAX with one warp per row and no block
// barriers: each lane keeps the CW_PMAX smallest upper bounds of its lists
// (sorted, in registers), the warp extracts the P-th smallest of their
// union as T, then gathers S, tests the sure members and re-decides the
// rest in FP64 exactly as above.  Rows whose S exceeds CW_SCAP take the
// serial FP64 path.  FROM_S: the candidate set comes from the fused first
// stage (a superset of S for its BF16 bound); a row it marked as overflowed
// is selected from all lists with FP32 distances computed here.
constexpr int CW_ROWS = 4;     // rows (warps) per block
constexpr int CW_PMAX = 8;
constexpr int CW_SCAP = 128;
constexpr int CW_LMAX = 4096;  // most lists for one warp per row
constexpr int CW_RG = 4;       // FP32 rechecks in flight per warp

// PM: length of each lane's sorted list (1 when P = 1, else CW_PMAX)
template <int PM, bool FROM_S>
__global__ __launch_bounds__(CW_ROWS * 32) void k_coarse_select_w(SelArgs a)
{
    pdl_begin();
    __shared__ float sLB[CW_ROWS][CW_SCAP], sUB[CW_ROWS][CW_SCAP], sDt[CW_ROWS][CW_SCAP];
    __shared__ int sIdx[CW_ROWS][CW_SCAP];
    __shared__ double sDx[CW_ROWS][CW_SCAP];
    __shared__ unsigned char sSure[CW_ROWS][CW_SCAP];
    __shared__ int sSel[CW_ROWS][CW_PMAX];
    __shared__ float sSelDt[CW_ROWS][CW_PMAX];
    __shared__ double sHd[CW_ROWS][CW_PMAX];
    __shared__ __align__(16) float sX[CW_ROWS][kMaxD];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = a.L, P = a.P;
    const int nrows = FROM_S ? *a.nhard : a.m;
    for (int it = blockIdx.x * CW_ROWS + w; it < nrows; it += gridDim.x * CW_ROWS) {  // whole warps
        const int row = FROM_S ? a.hard[it] : it;
        const float *Dr = FROM_S ? nullptr : a.D + (size_t)row * L;
        const float *xr = a.x + (size_t)row * a.d;
        int two_level = a.two_level;
        float g1 = two_level ? a.gamma2_first : a.gamma2;

        // ||x|| upper bound from an FP64 sum
        double part = 0.0;
        for (int j = lane; j < a.d; j += 32) part += (double)xr[j] * (double)xr[j];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const float xn = __double2float_ru(sqrt(part) * (1.0 + 1e-12));

        // first-stage distance of list c: the approximate matrix, or for a row
        // the fused first stage could not record, an FP32 dot product (one lane)
        int ns = 0;
        bool have_s = false;
        if (FROM_S) {
            for (int j = lane; j < a.d; j += 32) sX[w][j] = xr[j];
            const int32_t *Sr = a.S + (size_t)row * a.s_stride;
            const int n0 = Sr[0];
            if (n0 >= 0 && n0 <= CW_SCAP) {
                for (int p = lane; p < n0; p += 32) sIdx[w][p] = Sr[1 + p];
                ns = n0;
                have_s = true;
            } else {
                two_level = 0;
                g1 = a.gamma2;
            }
            __syncwarp();
        }
        auto dt_of = [&](int c) -> float {
            if (!FROM_S) return __ldg(Dr + c);
            const float4 *x4 = reinterpret_cast<const float4 *>(sX[w]);
            const float4 *c4 = reinterpret_cast<const float4 *>(a.cent + (size_t)c * a.d);
            float acc = 0.f;
            for (int j4 = 0; j4 < (a.d >> 2); ++j4) {
                const float4 xv = x4[j4], cv = __ldg(c4 + j4);
                acc = fmaf(xv.x, cv.x, acc);
                acc = fmaf(xv.y, cv.y, acc);
                acc = fmaf(xv.z, cv.z, acc);
                acc = fmaf(xv.w, cv.w, acc);
            }
            for (int j = a.d & ~3; j < a.d; ++j)
                acc = fmaf(sX[w][j], __ldg(a.cent + (size_t)c * a.d + j), acc);
            return fmaf(-2.f, acc, __ldg(a.cn + c));
        };

        // P-th smallest of the values v(i), i < n, each lane keeping its
        // CW_PMAX smallest in a sorted register list
        auto pth_smallest = [&](auto val, int n) {
            float top[PM];
#pragma unroll
            for (int k = 0; k < PM; ++k) top[k] = INFINITY;
            constexpr int CU = 8;  // values per lane loaded ahead
            for (int i0 = lane; i0 < n; i0 += 32 * CU) {
                float vv[CU];
#pragma unroll
                for (int u = 0; u < CU; ++u) vv[u] = i0 + 32 * u < n ? val(i0 + 32 * u) : INFINITY;
#pragma unroll
                for (int u = 0; u < CU; ++u) {
                    float v = vv[u];
#pragma unroll
                    for (int k = 0; k < PM; ++k) {  // insert into the sorted list
                        const float lo = fminf(top[k], v), hi = fmaxf(top[k], v);
                        top[k] = lo;
                        v = hi;
                    }
                }
            }
            float T = INFINITY;
            for (int t = 0; t < P; ++t) {
                float v = top[0];
                int who = lane;
                for (int o = 16; o > 0; o >>= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
                    const int ow = __shfl_xor_sync(0xffffffffu, who, o);
                    if (ov < v || (ov == v && ow < who)) {
                        v = ov;
                        who = ow;
                    }
                }
                T = v;
                if (lane == who) {
#pragma unroll
                    for (int k = 0; k + 1 < PM; ++k) top[k] = top[k + 1];
                    top[PM - 1] = INFINITY;
                }
            }
            return T;
        };

        // T = P-th smallest upper bound over all lists
        float T = INFINITY;
        if (!have_s) T = pth_smallest([&](int c) {
            const float Dt = dt_of(c);
            return upper_of(Dt, bound_of(Dt, __ldg(a.cn + c), __ldg(a.cnrm_up + c), xn, g1));
        }, L);

        // candidate set S = {c : lower bound <= T}
        constexpr int CU = 8;
        for (int c00 = 0; c00 < (have_s ? 0 : L); c00 += 32 * CU) {
            float lbv[CU], ubv[CU], dtv[CU];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int c = c00 + 32 * u + lane;
                lbv[u] = INFINITY;
                ubv[u] = INFINITY;
                dtv[u] = 0.f;
                if (c < L) {
                    const float Dt = dt_of(c);
                    const float E = bound_of(Dt, __ldg(a.cn + c), __ldg(a.cnrm_up + c), xn, g1);
                    lbv[u] = lower_of(Dt, E);
                    ubv[u] = upper_of(Dt, E);
                    dtv[u] = Dt;
                }
            }
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int c = c00 + 32 * u + lane;
                const bool in = c < L && lbv[u] <= T;
                const uint32_t mk = __ballot_sync(0xffffffffu, in);
                if (in) {
                    const int p = ns + __popc(mk & lanemask_lt());
                    if (p < CW_SCAP) {
                        sLB[w][p] = lbv[u];
                        sUB[w][p] = ubv[u];
                        sDt[w][p] = dtv[u];
                        sIdx[w][p] = c;
                    }
                }
                ns += __popc(mk);
            }
        }
        __syncwarp();
        if (two_level && ns <= CW_SCAP) {
            // S holds every list that can be among the top P (BF16-stage
            // bound); recompute their distances in FP32, one list per lane,
            // rebuild T and S with the FP32 bound inside S
            for (int j = lane; j < a.d; j += 32) sX[w][j] = xr[j];
            __syncwarp();
            // the warp computes CW_RG members' dot products at a time, lanes
            // over the coordinates (coalesced centroid rows), then a butterfly
            const float4 *x4 = reinterpret_cast<const float4 *>(sX[w]);
            const int n4 = a.d >> 2;
            for (int p0 = 0; p0 < ns; p0 += CW_RG) {
                float part[CW_RG];
#pragma unroll
                for (int t = 0; t < CW_RG; ++t) {
                    part[t] = 0.f;
                    if (p0 + t >= ns) continue;
                    const float4 *c4 =
                        reinterpret_cast<const float4 *>(a.cent + (size_t)sIdx[w][p0 + t] * a.d);
#pragma unroll
                    for (int u = 0; u < kMaxD / 128; ++u) {
                        const int j4 = lane + 32 * u;
                        if (j4 >= n4) break;
                        const float4 xv = x4[j4], cv = __ldg(c4 + j4);
                        part[t] = fmaf(xv.x, cv.x, part[t]);
                        part[t] = fmaf(xv.y, cv.y, part[t]);
                        part[t] = fmaf(xv.z, cv.z, part[t]);
                        part[t] = fmaf(xv.w, cv.w, part[t]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int t = 0; t < CW_RG; ++t) part[t] += __shfl_xor_sync(0xffffffffu, part[t], o);
                float acc = part[0];
#pragma unroll
                for (int t = 1; t < CW_RG; ++t)
                    if (lane == t) acc = part[t];
                const int p = p0 + lane;
                if (lane < CW_RG && p < ns) {
                    const int c = sIdx[w][p];
                    const float cnc = __ldg(a.cn + c);
                    const float Dt = fmaf(-2.f, acc, cnc);
                    const float E = bound_of(Dt, cnc, __ldg(a.cnrm_up + c), xn, a.gamma2);
                    sLB[w][p] = lower_of(Dt, E);
                    sUB[w][p] = upper_of(Dt, E);
                    sDt[w][p] = Dt;
                }
            }
            __syncwarp();
            T = pth_smallest([&](int p) { return sUB[w][p]; }, ns);
            int n2 = 0;
            for (int p0 = 0; p0 < ns; p0 += 32) {
                const int p = p0 + lane;
                const bool keep = p < ns && sLB[w][p] <= T;
                float lb = 0.f, ub = 0.f, dt = 0.f;
                int c = 0;
                if (keep) {
                    lb = sLB[w][p];
                    ub = sUB[w][p];
                    dt = sDt[w][p];
                    c = sIdx[w][p];
                }
                const uint32_t mk = __ballot_sync(0xffffffffu, keep);
                __syncwarp();
                if (keep) {  // write index <= read index
                    const int q = n2 + __popc(mk & lanemask_lt());
                    sLB[w][q] = lb;
                    sUB[w][q] = ub;
                    sDt[w][q] = dt;
                    sIdx[w][q] = c;
                }
                n2 += __popc(mk);
                __syncwarp();
            }
            ns = n2;
        }
        int32_t *outr = a.out + (size_t)row * P;
        int nsel = 0;
        if (ns <= CW_SCAP) {
            // sure members
            for (int p0 = 0; p0 < ns; p0 += 32) {
                const int p = p0 + lane;
                bool sure = false;
                if (p < ns) {
                    const float ub = sUB[w][p];
                    int cnt = 0;
                    for (int q = 0; q < ns; ++q) cnt += (q != p && sLB[w][q] <= ub);
                    sure = ub <= T && cnt < P;
                    sSure[w][p] = sure;
                }
                const uint32_t mk = __ballot_sync(0xffffffffu, sure);
                if (sure) {
                    const int s = nsel + __popc(mk & lanemask_lt());
                    if (s < CW_PMAX) {
                        sSel[w][s] = sIdx[w][p];
                        sSelDt[w][s] = sDt[w][p];
                    }
                }
                nsel += __popc(mk);
            }
            __syncwarp();
            const int r = P - nsel, nb = ns - nsel;
            if (r > 0) {
                // boundary members: exact FP64 distances, rank among them
                if (nb > r) {
                    for (int p = lane; p < ns; p += 32)
                        if (!sSure[w][p]) sDx[w][p] = exact_dist(xr, a.cent + (size_t)sIdx[w][p] * a.d, a.d);
                    __syncwarp();
                }
                for (int p0 = 0; p0 < ns; p0 += 32) {
                    const int p = p0 + lane;
                    bool take = false;
                    if (p < ns && !sSure[w][p]) {
                        take = true;
                        if (nb > r) {
                            const double Dc = sDx[w][p];
                            const int c = sIdx[w][p];
                            int rank = 0;
                            for (int q = 0; q < ns; ++q) {
                                if (q == p || sSure[w][q]) continue;
                                rank += (sDx[w][q] < Dc || (sDx[w][q] == Dc && sIdx[w][q] < c));
                            }
                            take = rank < r;
                        }
                    }
                    const uint32_t mk = __ballot_sync(0xffffffffu, take);
                    if (take) {
                        const int s = nsel + __popc(mk & lanemask_lt());
                        if (s < CW_PMAX) {
                            sSel[w][s] = sIdx[w][p];
                            sSelDt[w][s] = sDt[w][p];
                        }
                    }
                    nsel += __popc(mk);
                }
            }
        } else {
            // pathological (more than CW_SCAP candidates, e.g. many identical
            // centroids): exact FP64 insertion into a sorted array of P, lists
            // in index order (keeps the lowest index among ties)
            if (lane == 0) {
                int n = 0;
                for (int c = 0; c < L; ++c) {
                    const float Dt = dt_of(c);
                    const float E = bound_of(Dt, a.cn[c], a.cnrm_up[c], xn, g1);
                    if (lower_of(Dt, E) > T) continue;
                    const double Dc = exact_dist(xr, a.cent + (size_t)c * a.d, a.d);
                    if (n == P && !(Dc < sHd[w][n - 1])) continue;
                    int pos = n < P ? n : P - 1;
                    while (pos > 0 && Dc < sHd[w][pos - 1]) {
                        sHd[w][pos] = sHd[w][pos - 1];
                        sSel[w][pos] = sSel[w][pos - 1];
                        --pos;
                    }
                    sHd[w][pos] = Dc;
                    sSel[w][pos] = c;
                    if (n < P) ++n;
                }
                for (int i = 0; i < n; ++i) sSelDt[w][i] = (float)sHd[w][i];
                nsel = n;
            }
            nsel = __shfl_sync(0xffffffffu, nsel, 0);
        }
        __syncwarp();
        // the selected set nearest first: ascending approximate distance, ties
        // to the lower list index (the set itself is the exact one)
        if (nsel != P && lane == 0) atomicOr(a.err, ERR_SELECT);
        nsel = min(nsel, P);
        if (lane < P) {
            if (lane >= nsel) {
                outr[lane] = -1;
            } else {
                const int c = sSel[w][lane];
                const float dc = sSelDt[w][lane];
                int pos = 0;
                for (int q = 0; q < nsel; ++q) {
                    const int c2 = sSel[w][q];
                    const float d2 = sSelDt[w][q];
                    pos += d2 < dc || (d2 == dc && c2 < c);
                }
                outr[pos] = c;
            }
        }
        __syncwarp();  // the warp's shared rows are reused by its next row
    }
}

// FP8 inverse scale of each list for its residual codes x - c_l: 448 / R_l
// with R_l the distance from c_l to its nearest other centroid (FP64, the
// squared distance summed in index order, no fused multiply-add); with a
// single list or a duplicated centroid (R_l = 0) the raw-magnitude rule
// 448 / (2 max_j |c_lj|) (1 for a zero centroid).  One warp per list, its
// lanes striding over the other centroids.
__global__ void k_fp8_scales(const float *__restrict__ cent, int L, int d,
                             float *__restrict__ inv_scale8)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= L) return;
    const float *cl = cent + (size_t)l * d;
    double best = INFINITY;
    for (int o = lane; o < L; o += 32) {
        if (o == l) continue;
        const float *co = cent + (size_t)o * d;
        double s = 0.0;
        for (int j = 0; j < d; ++j) {
            const double t = __dsub_rn((double)cl[j], (double)co[j]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        best = fmin(best, s);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) {
        float inv;
        if (best > 0.0 && best < INFINITY) {
            inv = __double2float_rn(448.0 / sqrt(best));
        } else {
            double mx = 0.0;
            for (int j = 0; j < d; ++j) mx = fmax(mx, fabs((double)cl[j]));
            inv = mx > 0.0 ? __double2float_rn(448.0 / (2.0 * mx)) : 1.0f;
        }
        inv_scale8[l] = inv;
    }
}

// ------------------------------------------------------------ host drivers
void centroid_prep(sivf_index *ix, cudaStream_t st)
{
    ix->launches += 1;
    launch_pdl(k_centroid_norms, (ix->nlist + 127) / 128, 128, 0, st, ix->cent, ix->nlist, ix->d,
               ix->cnorm, ix->cnrm_up, ix->inv_scale8, ix->cent_bf16, ix->cent_lo);
    if (ix->x8) {
        ix->launches += 1;
        launch_pdl(k_fp8_scales, (ix->nlist * 32 + 127) / 128, 128, 0, st, ix->cent, ix->nlist,
                   ix->d, ix->inv_scale8);
    }
}

// Squared distance from each centroid to its nearest other centroid, FP32
// (a statistic that picks the first stage, never a result).  One warp per
// list, its lanes striding over the other centroids.
__global__ void k_cent_gap(const float *__restrict__ cent, int L, int d,
                           float *__restrict__ gap2)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= L) return;
    const float *cl = cent + (size_t)l * d;
    float best = INFINITY;
    for (int o = lane; o < L; o += 32) {
        if (o == l) continue;
        const float *co = cent + (size_t)o * d;
        float s0 = 0.f, s1 = 0.f;
        int j = 0;
        for (; j + 1 < d; j += 2) {
            const float t0 = cl[j] - co[j], t1 = cl[j + 1] - co[j + 1];
            s0 = fmaf(t0, t0, s0);
            s1 = fmaf(t1, t1, s1);
        }
        if (j < d) {
            const float t0 = cl[j] - co[j];
            s0 = fmaf(t0, t0, s0);
        }
        best = fminf(best, s0 + s1);
    }
    for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) gap2[l] = best;
}

// relative error of the BF16 first stage's dot products, |acc - x.c| /
// (||x|| ||c||): unit roundoff of BF16 ub = 2^-8; the FP32 accumulation of
// the exact BF16 products is taken as up to two ulps per addition, over d
// (single) or 3 d (split) terms.  Single: 2 ub + ub^2 (both roundings) plus
// the accumulation; split: the dropped products xl cl, and the roundings of
// xl and cl (each ub^2 relative), 3.1 ub^2 in all, plus the accumulation.
static double first_stage_rel(int d, int split)
{
    const double ub = 1.0 / 256.0;
    const double gacc = (split == 3 ? 3.0 * d : (double)d) * std::ldexp(1.0, -22);
    return split == 3 ? 3.1 * ub * ub + gacc * (1 + 2 * ub)
                      : (2 * ub + ub * ub) + gacc * (1 + ub) * (1 + ub);
}

// Which first stage nearest-list assignment takes.  The single BF16 product
// decides a row on its own when the row's second-nearest list is farther
// than its nearest by more than twice the bound the fused stage uses,
// E = 2 gamma ||x|| max ||c|| (gamma = 2 first_stage_rel, the bound on one
// distance, doubled for safety); otherwise the row's candidates are
// recorded and re-decided, and a row with more candidates than its records
// hold is redone from every list.  For a point near its centroid that gap
// is about the squared distance R^2 from the centroid to its nearest
// neighbour, so when 2 E (taken at ||x|| = max ||c||) exceeds the median
// R^2, most rows would be undecided and the split first stage (bound about
// 60x tighter) is taken instead.  Both give the same assignment.
// Synchronizes `st`.
cudaError_t assign_stage_choose(sivf_index *ix, cudaStream_t st)
{
    ix->assign_split = false;
    const int L = ix->nlist, d = ix->d;
    if (!ix->cent_bf16 || !ix->cent_lo || L < 2 || L > CW_LMAX || d % 16 || d > 128)
        return cudaSuccess;
    float *gap2 = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&gap2), sizeof(float) * L, st);
    if (e != cudaSuccess) return e;
    ix->launches += 1;
    launch_pdl(k_cent_gap, (L * 32 + 127) / 128, 128, 0, st, ix->cent, L, d, gap2);
    std::vector<float> g((size_t)L), cn((size_t)L);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.data(), gap2, sizeof(float) * L, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cn.data(), ix->cnorm, sizeof(float) * L, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(gap2, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::nth_element(g.begin(), g.begin() + L / 2, g.end());
    const double med = g[(size_t)L / 2];
    const double c2 = *std::max_element(cn.begin(), cn.end());
    const double e_max = 4.0 * first_stage_rel(d, 1) * c2;  // E at ||x|| = max ||c||
    ix->assign_split = std::isfinite(med) && 2.0 * e_max > med;
    return cudaSuccess;
}

// First stage of the selection of P lists: 1 the single BF16 product, 3
// the split BF16 products, 0 FP32.  The single product is within a few
// percent of ||x|| ||c||: tight enough to isolate the nearest centroid
// (assignment, P = 1) unless the centroids are close together against
// their norms (assign_stage_choose), but not to separate the P-th from the
// (P+1)-th of a dense shell of far centroids; probe selection takes the
// split form (three products, ~1e-4 of ||x|| ||c||), which needs twice the
// shared memory (d <= 128).  One warp per row suits up to a few thousand
// lists; beyond, the block kernel (256 threads per row) selects, from the
// FP32 first stage.
int first_stage_split(const sivf_index *ix, int P)
{
    const int d = ix->d;
    if (P > CW_PMAX || ix->nlist > CW_LMAX || d % 16) return 0;
    const bool single = P == 1 && !ix->assign_split;
    if (single) return ix->cent_bf16 && d <= kMaxD ? 1 : 0;
    return ix->cent_lo && d <= 128 ? 3 : 0;
}

// rows [0, m) of x -> out[m, P]; `Dbuf` holds at least rows_per_chunk * L
// floats.
void coarse_topP(sivf_index *ix, const float *x, int64_t m, int P, int32_t *out,
                 float *Dbuf, int64_t rows_per_chunk, cudaStream_t st)
{
    const int L = ix->nlist, d = ix->d;
    const double u = 5.9604644775390625e-08;
    const double gd = d * u / (1.0 - d * u);
    const bool warp_rows = P <= CW_PMAX && L <= CW_LMAX;
    const int split = first_stage_split(ix, P);
    const bool two = split != 0;
    const float gamma2_first = (float)(2.0 * first_stage_rel(d, split) * (1.0 + 1e-6));
    // assignment with the single BF16 product: the fused first stage keeps
    // only each row's candidate lists (needs CF_STRIDE ints per row of the
    // distance buffer, and d <= 128 for its shared memory)
    const bool fused = split == 1 && ix->tmap_cent_ok &&
                       (size_t)32 + (size_t)rows_per_chunk * (CF_STRIDE + 1) <=
                           (size_t)rows_per_chunk * L;
    int nsm = 0;
    if (fused) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        nsm = std::max(nsm, 1);
    }
    for (int64_t r0 = 0; r0 < m; r0 += rows_per_chunk) {
        int mc = (int)std::min<int64_t>(rows_per_chunk, m - r0);
        const int tok = prof_begin(ix, PROF_COARSE, 2, st);
        if (fused) {
            const size_t smem = coarse_fused_smem(d);
            // the distance buffer holds the undecided-row count, the
            // undecided rows and the candidate lists
            int32_t *nh = reinterpret_cast<int32_t *>(Dbuf);
            cudaMemsetAsync(nh, 0, sizeof(int32_t), st);
            const int nt = (mc + CT_M - 1) / CT_M;
            const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(ix->tmap_cent);
            // shared memory opted in once per instantiation (index KC - 1)
            static size_t attr[2] = {0, 0};
            auto go = [&](auto kern, int kc) {
                if (smem > attr[kc - 1]) {
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
                    attr[kc - 1] = smem;
                }
                launch_pdl(kern, std::min(nt, nsm), CF_NT, smem, st, tm, x + r0 * d, mc, d,
                           ix->cnorm, ix->cnrm_up, L, gamma2_first, out + r0, nh + 32 + mc, nh + 32,
                           nh, ix->err);
            };
            if (d <= 64) go(k_coarse_fused1<1>, 1);
            else go(k_coarse_fused1<2>, 2);
        } else if (two) {
            const size_t smem = coarse_tc_smem(d, split);
            dim3 g((mc + CT_M - 1) / CT_M, (L + CT_N - 1) / CT_N);
            if (split == 1) {
                static size_t attr = 0;
                if (smem > attr) {
                    cudaFuncSetAttribute(k_coarse_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
                    attr = smem;
                }
                launch_pdl(k_coarse_tc<1>, g, CT_NT, smem, st, x + r0 * d, mc, d, ix->cent_bf16,
                           nullptr, ix->cnorm, L, Dbuf, ix->err);
            } else {
                static size_t attr = 0;
                if (smem > attr) {
                    cudaFuncSetAttribute(k_coarse_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
                    attr = smem;
                }
                launch_pdl(k_coarse_tc<3>, g, CT_NT, smem, st, x + r0 * d, mc, d, ix->cent_bf16,
                           ix->cent_lo, ix->cnorm, L, Dbuf, ix->err);
            }
        } else {
            dim3 g((L + GBN - 1) / GBN, (mc + GBM - 1) / GBM);
            launch_pdl(k_coarse_gemm, g, 256, 0, st, x + r0 * d, mc, d, ix->cent, ix->cnorm, L,
                       Dbuf);
        }
        SelArgs a;
        a.D = fused ? nullptr : Dbuf;
        a.S = fused ? reinterpret_cast<const int32_t *>(Dbuf) + 32 + mc : nullptr;
        a.s_stride = CF_STRIDE;
        a.hard = reinterpret_cast<const int32_t *>(Dbuf) + 32;
        a.nhard = reinterpret_cast<const int *>(Dbuf);
        a.m = mc;
        a.L = L;
        a.P = P;
        a.d = d;
        a.x = x + r0 * d;
        a.cent = ix->cent;
        a.cn = ix->cnorm;
        a.cnrm_up = ix->cnrm_up;
        a.gamma2 = (float)(2.0 * gd * (1.0 + 1e-6));
        a.gamma2_first = gamma2_first;
        a.two_level = two;
        a.out = out + r0 * P;
        a.err = ix->err;
        if (warp_rows) {
            const unsigned gw = (unsigned)((mc + CW_ROWS - 1) / CW_ROWS);
            if (fused)  // loops over the undecided rows, usually none
                launch_pdl(k_coarse_select_w<1, true>, std::min<unsigned>(gw, 2u * (unsigned)nsm),
                           CW_ROWS * 32, 0, st, a);
            else if (P == 1) launch_pdl(k_coarse_select_w<1, false>, gw, CW_ROWS * 32, 0, st, a);
            else launch_pdl(k_coarse_select_w<CW_PMAX, false>, gw, CW_ROWS * 32, 0, st, a);
        } else {
            launch_pdl(k_coarse_select, mc, SEL_NT, 0, st, a);
        }
        prof_end(ix, tok, st);
    }
}

}  // namespace sivf
