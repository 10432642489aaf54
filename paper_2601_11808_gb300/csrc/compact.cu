// Compaction of partly-live slabs.
//
// Deletes clear validity bits (Algorithm 4) and a slab returns to the pool
// only when its last live vector goes, so random deletes leave lists made of
// sparse slabs: memory held and bytes streamed by every scan of the list
// grow with the holes.  The paper leaves adaptive background compaction to
// future work (Conclusion); this pass is one reading of it.  A list whose
// live members would fit in at least `min_free` fewer slabs is rewritten
// densely in its own member order: member j (slab position, then slot)
// moves to slot j mod C of the list's (j div C)-th slab, the list keeps its
// first ceil(n / C) slabs and the rest go back on the free stack.  Lists are
// taken in index order while the running total of rewritten members stays
// within `max_moves` (the first list that would pass it ends the pass), so
// a caller bounds the work of one pass and runs passes between batches.
//
// Kernels, in stream order:
//   plan     one block: candidates, the budget prefix, offsets of the
//            selected lists' members and slabs
//   bases    one block per selected list: live members before each slab
//   gather   one warp per selected slab: live rows, in slot order, into a
//            staging buffer at their member index (the move never reads a
//            slot another move has written: all reads finish first)
//   scatter  one warp per member: staged row to its dense place, id, table
//   finish   one warp per selected list: fill/live/bitmaps of the kept
//            slabs, the rest reset and pushed on the free stack, directory
//            length and head slab
#include "device_utils.cuh"
#include "kernels.cuh"

namespace sivf {

namespace {

constexpr int CP_PLAN_NT = 1024;

__device__ __forceinline__ int32_t list_len(const CompactArgs &a, int l)
{
    int n = a.nslabs[l];
    if (n > a.dir_cap) {
        atomicOr(a.err, ERR_DIR_BOUND);
        n = (int)a.dir_cap;
    }
    return n;
}

// inclusive block scan of one int64 per thread (CP_PLAN_NT threads)
__device__ int64_t block_incl_scan(int64_t v, int64_t *sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int o = 1; o < CP_PLAN_NT; o <<= 1) {
        const int64_t t = tid >= o ? sh[tid - o] : 0;
        __syncthreads();
        sh[tid] += t;
        __syncthreads();
    }
    const int64_t r = sh[tid];
    __syncthreads();
    return r;
}

__global__ __launch_bounds__(CP_PLAN_NT) void k_cp_plan(CompactArgs a, int min_free,
                                                        int64_t max_moves)
{
    pdl_begin();
    __shared__ int64_t sh[CP_PLAN_NT];
    const int tid = threadIdx.x;
    const int per = (a.L + CP_PLAN_NT - 1) / CP_PLAN_NT;
    const int b0 = min(a.L, tid * per), b1 = min(a.L, b0 + per);
    auto cand_moves = [&](int l) -> int64_t {
        const int n = list_len(a, l), live = a.list_live[l];
        const int keep = (live + a.C - 1) / a.C;
        return n - keep >= min_free ? (int64_t)live : -1;
    };
    // members of the candidate lists, prefix over lists
    int64_t mv = 0;
    for (int l = b0; l < b1; ++l) {
        const int64_t m = cand_moves(l);
        if (m > 0) mv += m;
    }
    const int64_t run0 = block_incl_scan(mv, sh) - mv;
    // selected: candidates whose inclusive prefix stays within the budget
    int64_t nsel = 0, nsl = 0, nfree = 0, smv = 0, run = run0;
    for (int l = b0; l < b1; ++l) {
        const int64_t m = cand_moves(l);
        if (m <= 0) continue;
        run += m;
        if (run > max_moves) break;
        const int n = list_len(a, l);
        ++nsel;
        nsl += n;
        smv += m;
        nfree += n - (m + a.C - 1) / a.C;
    }
    const int64_t sel0 = block_incl_scan(nsel, sh) - nsel;
    const int64_t sl0 = block_incl_scan(nsl, sh) - nsl;
    const int64_t fr = block_incl_scan(nfree, sh);
    const int64_t mvs = block_incl_scan(smv, sh);
    int64_t k = sel0, so = sl0;
    run = run0;
    for (int l = b0; l < b1; ++l) {
        const int64_t m = cand_moves(l);
        if (m <= 0) continue;
        if (run + m > max_moves) break;
        a.sel[k] = l;
        a.voff[k] = run;
        a.soff[k] = so;
        run += m;
        so += list_len(a, l);
        ++k;
    }
    if (tid == CP_PLAN_NT - 1) {
        a.voff[k] = mvs;     // k = number of selected lists
        a.soff[k] = so;
        a.ctl->ntouched = (int32_t)k;
        a.ctl->count = mvs;  // members rewritten
        a.ctl->demand = fr;  // slabs freed
    }
}

// selected list holding entry g of an offset array (largest k: off[k] <= g)
__device__ __forceinline__ int find_run(const int64_t *off, int n, int64_t g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ __launch_bounds__(256) void k_cp_bases(CompactArgs a)
{
    pdl_begin();
    __shared__ int32_t wsum[8];
    __shared__ int32_t s_run;
    const int nsel = a.ctl->ntouched;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = blockIdx.x; k < nsel; k += gridDim.x) {
        const int l = a.sel[k];
        const int n = (int)(a.soff[k + 1] - a.soff[k]);
        const int32_t *D = a.dir + (size_t)l * a.dir_cap;
        if (tid == 0) s_run = 0;
        __syncthreads();
        for (int base = 0; base < n; base += 256) {
            const int i = base + tid;
            int live = 0;
            if (i < n) {
                const int s = D[i];
                if (s < 0 || s >= a.n_slabs) {
                    atomicOr(a.err, ERR_BAD_SLAB);
                } else {
                    for (int w = 0; w < a.W; ++w) live += __popc(a.bits[(size_t)s * a.W + w]);
                }
            }
            int incl = live;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            int before = s_run;
            for (int w = 0; w < warp; ++w) before += wsum[w];
            if (i < n) a.sb[a.soff[k] + i] = before + incl - live;
            __syncthreads();
            if (tid == 0) {
                int t = 0;
                for (int w = 0; w < 8; ++w) t += wsum[w];
                s_run += t;
            }
            __syncthreads();
        }
    }
}

// one row's FP32 payload, BF16 / E4M3 codes (d % 4 == 0): float4, 4 x bf16
// and 4 x e4m3 per lane and round, CP_RV rounds cover d <= 256
constexpr int CP_RV = 2;
constexpr int CP_U = 4;  // rows in flight per warp in the gather

struct RowRegs {
    float4 f[CP_RV];
    uint2 h[CP_RV];
    uint32_t b[CP_RV];
};

__device__ __forceinline__ void row_load(const CompactArgs &a, int64_t src, int lane, RowRegs &v)
{
    const int n4 = a.d >> 2;
#pragma unroll
    for (int t = 0; t < CP_RV; ++t) {
        const int j4 = lane + 32 * t;
        if (j4 >= n4) break;
        v.f[t] = __ldg(reinterpret_cast<const float4 *>(a.x32 + src * a.d) + j4);
        if (a.t16) v.h[t] = __ldg(reinterpret_cast<const uint2 *>(a.xb16 + src * a.d) + j4);
        if (a.t8) v.b[t] = __ldg(reinterpret_cast<const uint32_t *>(a.x8 + src * a.d) + j4);
    }
}

__device__ __forceinline__ void row_store(float *f32, __nv_bfloat16 *f16, uint8_t *f8, int64_t dst,
                                          int d, int lane, const RowRegs &v)
{
    const int n4 = d >> 2;
#pragma unroll
    for (int t = 0; t < CP_RV; ++t) {
        const int j4 = lane + 32 * t;
        if (j4 >= n4) break;
        reinterpret_cast<float4 *>(f32 + dst * d)[j4] = v.f[t];
        if (f16) reinterpret_cast<uint2 *>(f16 + dst * d)[j4] = v.h[t];
        if (f8) reinterpret_cast<uint32_t *>(f8 + dst * d)[j4] = v.b[t];
    }
}

__global__ __launch_bounds__(256) void k_cp_gather(CompactArgs a)
{
    pdl_begin();
    const int nsel = a.ctl->ntouched;
    if (nsel == 0) return;
    const int64_t total = a.soff[nsel];
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; g < total; g += nw) {
        const int k = find_run(a.soff, nsel, g);
        const int l = a.sel[k];
        const int s = a.dir[(size_t)l * a.dir_cap + (g - a.soff[k])];
        if (s < 0 || s >= a.n_slabs) continue;  // reported by k_cp_bases
        int64_t r = a.voff[k] + a.sb[g];
        const int64_t rend = a.voff[k + 1];
        for (int w = 0; w < a.W; ++w) {
            uint32_t word = a.bits[(size_t)s * a.W + w];  // the same in every lane
            while (word) {
                int slot[CP_U];
                int nb = 0;
#pragma unroll
                for (int u = 0; u < CP_U; ++u) {
                    slot[u] = -1;
                    if (word) {
                        slot[u] = 32 * w + __ffs(word) - 1;
                        word &= word - 1;
                        ++nb;
                    }
                }
                if (r + nb > rend) {  // more bits than the list's live count
                    if (lane == 0) atomicOr(a.err, ERR_BAD_SLAB);
                    word = 0;
                    break;
                }
                RowRegs v[CP_U];
#pragma unroll
                for (int u = 0; u < CP_U; ++u)
                    if (slot[u] >= 0) row_load(a, (int64_t)s * a.C + slot[u], lane, v[u]);
#pragma unroll
                for (int u = 0; u < CP_U; ++u) {
                    if (slot[u] < 0) continue;
                    const int64_t src = (int64_t)s * a.C + slot[u];
                    row_store(a.t32, a.t16, a.t8, r + u, a.d, lane, v[u]);
                    if (lane == 0) {
                        a.tn[r + u] = a.xnorm[src];
                        if (a.tr) a.tr[r + u] = a.rnorm[src];
                        a.ti[r + u] = a.ids[src];
                    }
                }
                r += nb;
            }
        }
    }
}

__global__ __launch_bounds__(256) void k_cp_scatter(CompactArgs a)
{
    pdl_begin();
    const int nsel = a.ctl->ntouched;
    if (nsel == 0) return;
    const int64_t total = a.voff[nsel];
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < total; r += nw) {
        const int k = find_run(a.voff, nsel, r);
        const int l = a.sel[k];
        const int64_t j = r - a.voff[k];
        const int s = a.dir[(size_t)l * a.dir_cap + j / a.C];
        if (s < 0 || s >= a.n_slabs) continue;
        const int slot = (int)(j % a.C);
        const int64_t dst = (int64_t)s * a.C + slot;
        RowRegs v;
        const int n4 = a.d >> 2;
#pragma unroll
        for (int t = 0; t < CP_RV; ++t) {
            const int j4 = lane + 32 * t;
            if (j4 >= n4) break;
            v.f[t] = reinterpret_cast<const float4 *>(a.t32 + r * a.d)[j4];
            if (a.t16) v.h[t] = reinterpret_cast<const uint2 *>(a.t16 + r * a.d)[j4];
            if (a.t8) v.b[t] = reinterpret_cast<const uint32_t *>(a.t8 + r * a.d)[j4];
        }
        row_store(a.x32, a.t16 ? a.xb16 : nullptr, a.t8 ? a.x8 : nullptr, dst, a.d, lane, v);
        if (lane == 0) {
            a.xnorm[dst] = a.tn[r];
            if (a.tr) a.rnorm[dst] = a.tr[r];
            const int64_t id = a.ti[r];
            a.ids[dst] = id;
            if (id >= 0 && id < a.n_max) a.att[id] = ((int64_t)s << 32) | slot;
            else atomicOr(a.err, ERR_BAD_SLAB);
        }
    }
}

__global__ __launch_bounds__(256) void k_cp_finish(CompactArgs a)
{
    pdl_begin();
    const int nsel = a.ctl->ntouched;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x / 32);
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / 32; k < nsel; k += nw) {
        const int l = a.sel[k];
        const int n = (int)(a.soff[k + 1] - a.soff[k]);
        const int64_t live = a.voff[k + 1] - a.voff[k];
        const int keep = (int)((live + a.C - 1) / a.C);
        int32_t *D = a.dir + (size_t)l * a.dir_cap;
        for (int i = lane; i < n; i += 32) {
            const int s = D[i];
            if (s < 0 || s >= a.n_slabs) continue;
            if (i < keep) {
                const int64_t rem = live - (int64_t)i * a.C;
                const int f = rem < a.C ? (int)rem : a.C;
                a.meta[s].fill = f;
                a.meta[s].live = f;
                for (int w = 0; w < a.W; ++w) {
                    const int c = f - 32 * w;
                    a.bits[(size_t)s * a.W + w] =
                        c >= 32 ? 0xffffffffu : c <= 0 ? 0u : ((1u << c) - 1u);
                }
            } else {
                a.meta[s].list = -1;
                a.meta[s].fill = 0;
                a.meta[s].live = 0;
                for (int w = 0; w < a.W; ++w) a.bits[(size_t)s * a.W + w] = 0u;
                D[i] = -1;
                const int t = atomicAdd(a.free_top, 1);
                if (t >= a.n_slabs) atomicOr(a.err, ERR_STACK);
                else a.free_list[t] = s;
            }
        }
        __syncwarp();
        if (lane == 0) {
            a.nslabs[l] = keep;
            a.head[l] = keep > 0 ? D[keep - 1] : -1;
        }
    }
}

}  // namespace

void compact_pass(sivf_index *ix, const CompactArgs &a, int min_free, int64_t max_moves,
                  cudaStream_t st)
{
    const int tok = prof_begin(ix, PROF_COMPACT, 5, st);
    launch_pdl(k_cp_plan, 1, CP_PLAN_NT, 0, st, a, min_free, max_moves);
    const int grid = 152 * 4;
    launch_pdl(k_cp_bases, grid, 256, 0, st, a);
    launch_pdl(k_cp_gather, grid, 256, 0, st, a);
    launch_pdl(k_cp_scatter, grid, 256, 0, st, a);
    launch_pdl(k_cp_finish, grid, 256, 0, st, a);
    prof_end(ix, tok, st);
}

}  // namespace sivf
