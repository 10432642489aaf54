// Batched insert (Algorithms 1-2) and delete (Algorithm 4) of the slab index.
//
// Insert.  Algorithm 2 lets every thread race on the head slab's counter
// with CAS and retry; on a batch the outcome of that race is only a
// permutation of slots.  Here the permutation is fixed in advance, so no
// thread ever retries: each kept vector gets its rank among the batch's
// vectors of the same list (stable in batch order), the list's head slab
// takes the first C - fill of them and fresh slabs popped from the free
// stack take the rest.  Payload, id and address-table entry are written
// first, then a device fence, then the validity bit (Theorem 1: the bit is
// the publication point).  Kernels, in stream order:
//   claim     last occurrence of each id wins (atomicMax into claim[id])
//   rank      per block of 1024 vectors: stable sort by list, local ranks,
//             run counts per (list, block)
//   plan      per touched list: prefix of run counts over blocks, slab demand
//   overwrite all-or-nothing admission against the free stack (derived by
//             every thread, recorded once), then delete-then-insert for kept
//             ids that are live
//   reclaim   lists that lost a slab: directory compaction, slab to the stack
//   alloc     per touched list: fill the head, pop fresh slabs
//   append    per vector: payload + copies + id + table, fence, bit
//   cleanup   reset the per-batch bookkeeping
//
// Delete.  Per id: table lookup, atomicAnd on the validity word; the thread
// that takes the bit 1 -> 0 invalidates the table entry and decrements the
// slab's live count (Theorem 3: the atomicAnd is the linearization point,
// repeats are no-ops).  The thread that takes live 1 -> 0 records the list;
// a second kernel removes the emptied slabs from the list's directory (one
// warp per list, stable compaction) and pushes them on the free stack after
// resetting their metadata.  Pushes (delete) and pops (insert) never run in
// the same kernel, so the stack needs no ABA protection.
#include "device_utils.cuh"
#include "kernels.cuh"

namespace sivf {

struct IndexView {
    int d, nlist, C, W, nblk_max;
    int64_t n_max, n_slabs, dir_cap;
    float *x32;
    __nv_bfloat16 *xb16;
    uint8_t *x8;
    float *xnorm;
    int64_t *ids;
    uint32_t *bits;
    SlabMeta *meta;
    int32_t *free_list, *free_top;
    int32_t *head, *nslabs, *dir, *list_live;
    const float *inv_scale8;
    const float *cent;  // [nlist, d] (FP8 residual codes)
    float *rnorm;       // [S, C] ||x - c_l||^2 or null
    int64_t *att;
    int32_t *claim, *list_flag, *aff_flag, *runcnt;
    Ctl *ctl;
    uint32_t *err;
    int64_t *live_total;
};

static IndexView view_of(sivf_index *ix)
{
    IndexView v;
    v.d = ix->d;
    v.nlist = ix->nlist;
    v.C = ix->C;
    v.W = ix->W;
    v.nblk_max = ix->nblk_max;
    v.n_max = ix->n_max;
    v.n_slabs = ix->n_slabs;
    v.dir_cap = ix->dir_cap;
    v.x32 = ix->x32;
    v.xb16 = ix->xb16;
    v.x8 = ix->x8;
    v.xnorm = ix->xnorm;
    v.ids = ix->ids;
    v.bits = ix->bits;
    v.meta = ix->meta;
    v.free_list = ix->free_list;
    v.free_top = ix->free_top;
    v.head = ix->head;
    v.nslabs = ix->nslabs;
    v.dir = ix->dir;
    v.list_live = ix->list_live;
    v.inv_scale8 = ix->inv_scale8;
    v.cent = ix->cent;
    v.rnorm = ix->rnorm;
    v.att = ix->att;
    v.claim = ix->claim;
    v.list_flag = ix->list_flag;
    v.aff_flag = ix->aff_flag;
    v.runcnt = ix->runcnt;
    v.ctl = ix->ctl;
    v.err = ix->err;
    v.live_total = ix->stat;
    return v;
}

#define GRID_STRIDE(i, n)                                                    \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------ delete core
__device__ __forceinline__ void delete_one(const IndexView &V, int64_t id,
                                           int32_t *affected, bool count)
{
    const int64_t coord = V.att[id];
    if (coord < 0) return;
    const int64_t s = coord >> 32;
    const int o = (int)(coord & 0xffffffff);
    if (s >= V.n_slabs || o >= V.C) {
        atomicOr(V.err, ERR_BAD_SLAB);
        return;
    }
    const uint32_t m = 1u << (o & 31);
    const uint32_t old = atomicAnd(&V.bits[s * V.W + (o >> 5)], ~m);
    if (!(old & m)) return;  // already cleared: a repeat of this id
    V.att[id] = -1;
    atomicAdd(reinterpret_cast<unsigned long long *>(V.live_total),
              (unsigned long long)(-1LL));
    if (count) atomicAdd(reinterpret_cast<unsigned long long *>(&V.ctl->count), 1ull);
    const int l = V.meta[s].list;
    if (l < 0 || l >= V.nlist) {
        atomicOr(V.err, ERR_BAD_SLAB);
        return;
    }
    atomicSub(&V.list_live[l], 1);
    if (atomicSub(&V.meta[s].live, 1) == 1) {
        if (atomicCAS(&V.aff_flag[l], 0, 1) == 0)
            affected[atomicAdd(&V.ctl->naffected, 1)] = l;
    }
}

// one warp per list that lost a slab: stable compaction of the directory,
// emptied slabs reset and pushed on the free stack
__global__ void k_reclaim(IndexView V, const int32_t *__restrict__ affected)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * blockDim.x / 32;
    const int na = V.ctl->naffected;
    for (int a = (blockIdx.x * blockDim.x + threadIdx.x) / 32; a < na; a += nw) {
        const int l = affected[a];
        int n = V.nslabs[l];
        if (n > V.dir_cap) {
            if (lane == 0) atomicOr(V.err, ERR_DIR_BOUND);
            n = (int)V.dir_cap;
        }
        int32_t *D = V.dir + (size_t)l * V.dir_cap;
        const int h = V.head[l];
        int kept = 0;
        bool hfree = false;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const int s = i < n ? D[i] : -1;
            const bool valid = s >= 0 && s < V.n_slabs;
            if (i < n && !valid) atomicOr(V.err, ERR_BAD_SLAB);
            const bool keep = valid && V.meta[s].live > 0;
            const bool drop = valid && !keep;
            const uint32_t km = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) D[kept + __popc(km & lanemask_lt())] = s;
            kept += __popc(km);
            if (drop) {
                V.meta[s].list = -1;
                V.meta[s].fill = 0;
                V.meta[s].live = 0;
                const int t = atomicAdd(V.free_top, 1);
                if (t >= V.n_slabs) atomicOr(V.err, ERR_STACK);
                else V.free_list[t] = s;
                if (s == h) hfree = true;
            }
        }
        hfree = __any_sync(0xffffffffu, hfree);
        if (lane == 0) {
            V.nslabs[l] = kept;
            if (hfree) V.head[l] = -1;
            V.aff_flag[l] = 0;
        }
    }
}

// ------------------------------------------------------------- delete
__global__ void k_rm_validate(IndexView V, const int64_t *__restrict__ ids, int64_t n)
{
    pdl_begin();
    GRID_STRIDE(i, n)
    {
        const int64_t id = ids[i];
        if (id < 0 || id >= V.n_max) atomicOr(&V.ctl->flags, FLAG_BAD_ID);
    }
}

__global__ void k_rm_phase1(IndexView V, const int64_t *__restrict__ ids, int64_t n,
                            int32_t *__restrict__ affected)
{
    pdl_begin();
    if (V.ctl->flags & FLAG_BAD_ID) return;
    GRID_STRIDE(i, n) delete_one(V, ids[i], affected, true);
}

// ------------------------------------------------------------- insert
__global__ void k_ins_claim(IndexView V, const int64_t *__restrict__ ids, int64_t n)
{
    pdl_begin();
    GRID_STRIDE(i, n)
    {
        const int64_t id = ids[i];
        if (id < 0 || id >= V.n_max) atomicOr(&V.ctl->flags, FLAG_BAD_ID);
        else atomicMax(&V.claim[id], (int)i);
    }
}

// Stable rank of each kept vector among the kept vectors of its list inside
// its block of kRankTile vectors; run lengths per (list, block).
__global__ __launch_bounds__(512) void k_ins_rank(IndexView V, const int64_t *__restrict__ ids,
                                                  const int32_t *__restrict__ lab, int64_t n,
                                                  int32_t *__restrict__ rloc,
                                                  int32_t *__restrict__ touched)
{
    pdl_begin();
    static_assert(kRankTile == 1024, "rank tile");
    __shared__ uint32_t key[1024];
    __shared__ int32_t rs[1024];
    const int tid = threadIdx.x, b = blockIdx.x;
    const int64_t base = (int64_t)b * 1024;
    const uint32_t NONE = 0xffffffffu;
    for (int e = tid; e < 1024; e += 512) {
        const int64_t i = base + e;
        uint32_t k = NONE;
        if (i < n) {
            const int64_t id = ids[i];
            const int li = lab[i];
            if (li < 0 || li >= V.nlist) atomicOr(V.err, ERR_SELECT);
            if (id >= 0 && id < V.n_max && V.claim[id] == (int)i && li >= 0 && li < V.nlist)
                k = ((uint32_t)li << 10) | (uint32_t)e;
            else
                rloc[i] = -1;
        }
        key[e] = k;
    }
    __syncthreads();
    for (int size = 2; size <= 1024; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int pos = 2 * tid - (tid & (stride - 1));
            const int par = pos + stride;
            const bool up = (pos & size) == 0;
            const uint32_t x = key[pos], y = key[par];
            if ((x > y) == up) {
                key[pos] = y;
                key[par] = x;
            }
            __syncthreads();
        }
    for (int e = tid; e < 1024; e += 512) {
        const uint32_t k = key[e];
        const bool head = k != NONE && (e == 0 || (key[e - 1] >> 10) != (k >> 10));
        rs[e] = head ? e : 0;
    }
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int a0 = tid, a1 = tid + 512;
        const int v0 = max(rs[a0], a0 >= o ? rs[a0 - o] : 0);
        const int v1 = max(rs[a1], a1 >= o ? rs[a1 - o] : 0);
        __syncthreads();
        rs[a0] = v0;
        rs[a1] = v1;
        __syncthreads();
    }
    for (int e = tid; e < 1024; e += 512) {
        const uint32_t k = key[e];
        if (k == NONE) continue;
        const int l = (int)(k >> 10);
        const int64_t i = base + (k & 1023u);
        const int r = e - rs[e];
        rloc[i] = r;
        const bool tail = e == 1023 || (key[e + 1] >> 10) != (uint32_t)l;
        if (tail) V.runcnt[(size_t)l * V.nblk_max + b] = r + 1;
        if (r == 0 && atomicCAS(&V.list_flag[l], 0, -1) == 0) {
            const int t = atomicAdd(&V.ctl->ntouched, 1);
            touched[t] = l;
            atomicExch(&V.list_flag[l], t + 1);
        }
    }
}

// one warp per touched list: exclusive scan of its run counts over the
// rank blocks (lanes over blocks), then its slab demand
__global__ void k_ins_plan(IndexView V, int nblk, const int32_t *__restrict__ touched,
                           int32_t *__restrict__ bcnt)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= V.ctl->ntouched) return;  // whole warps
    const int l = touched[t];
    int32_t *rc = V.runcnt + (size_t)l * V.nblk_max;
    int acc = 0;
    for (int b0 = 0; b0 < nblk; b0 += 32) {  // warp-uniform
        const int b = b0 + lane;
        const int c = b < nblk ? rc[b] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (b < nblk) rc[b] = acc + incl - c;
        acc += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane != 0) return;
    bcnt[t] = acc;
    const int h = V.head[l];
    const int avail = h >= 0 ? V.C - V.meta[h].fill : 0;
    const int need = acc > avail ? (acc - avail + V.C - 1) / V.C : 0;
    if ((int64_t)V.nslabs[l] + need > V.dir_cap) atomicOr(&V.ctl->flags, FLAG_DIR_FULL);
    atomicAdd(reinterpret_cast<unsigned long long *>(&V.ctl->demand), (unsigned long long)need);
    atomicAdd(reinterpret_cast<unsigned long long *>(&V.ctl->count), (unsigned long long)acc);
}

// all-or-nothing admission of the batch against the free stack, from the
// plan's totals (every thread of the overwrite kernel derives it; the
// first records it for the kernels that follow and for the host)
__device__ __forceinline__ int admission(const IndexView &V)
{
    const Ctl *c = V.ctl;
    if (c->flags & FLAG_BAD_ID) return SIVF_E_ARG;
    if ((c->flags & FLAG_DIR_FULL) || c->demand > (int64_t)*V.free_top) return SIVF_E_NOMEM;
    return SIVF_OK;
}

__global__ void k_ins_overwrite(IndexView V, const int64_t *__restrict__ ids, int64_t n,
                                const int32_t *__restrict__ rloc, int32_t *__restrict__ affected)
{
    pdl_begin();
    const int st = admission(V);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        V.ctl->status = st;
        if (st != SIVF_OK) V.ctl->count = 0;
    }
    if (st != SIVF_OK) return;
    GRID_STRIDE(i, n)
    {
        if (rloc[i] < 0) continue;
        const int64_t id = ids[i];
        if (V.att[id] >= 0) delete_one(V, id, affected, false);
    }
}

__global__ void k_ins_alloc(IndexView V, const int32_t *__restrict__ touched,
                            const int32_t *__restrict__ bcnt, PlanEntry *__restrict__ plan)
{
    pdl_begin();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (V.ctl->status != SIVF_OK || t >= V.ctl->ntouched) return;
    const int l = touched[t];
    const int cnt = bcnt[t];
    const int C = V.C;
    const int h = V.head[l];
    const int fill = h >= 0 ? V.meta[h].fill : C;
    const int avail = C - fill;
    const int a = min(cnt, avail);
    const int need = cnt > avail ? (cnt - avail + C - 1) / C : 0;
    const int pos0 = V.nslabs[l];
    PlanEntry pe;
    pe.head_old = h;
    pe.fill_old = fill;
    pe.into_head = a;
    pe.dir_pos0 = pos0;
    if (a > 0) {
        V.meta[h].fill = fill + a;
        V.meta[h].live += a;
    }
    if (need > 0) {
        const int top = atomicSub(V.free_top, need);
        if (top - need < 0 || (int64_t)pos0 + need > V.dir_cap) {
            atomicOr(V.err, ERR_STACK);
            plan[t] = pe;
            return;
        }
        const int rem = cnt - a;
        int s = -1;
        // the reserved stack entries from the top down: on a fresh pool (slab
        // 0 on top) a list receives ascending consecutive slabs, which the
        // list scan fetches as one 128-row box
        for (int j = 0; j < need; ++j) {
            s = V.free_list[top - 1 - j];
            const int f = min(C, rem - j * C);
            V.meta[s].list = l;
            V.meta[s].fill = f;
            V.meta[s].live = f;
            V.dir[(size_t)l * V.dir_cap + pos0 + j] = s;
        }
        V.nslabs[l] = pos0 + need;
        V.head[l] = s;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(V.live_total), (unsigned long long)cnt);
    V.list_live[l] += cnt;
    plan[t] = pe;
}

// sum over the 16 lanes of a half warp (every lane of the warp calls it)
__device__ __forceinline__ float half_sum(float v)
{
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// two kept vectors per warp, one per half (16 lanes of 16-byte chunks): a
// batch of 10,000 takes one wave of resident warps instead of two
__global__ void k_ins_append(IndexView V, const int64_t *__restrict__ ids,
                             const float *__restrict__ x, int64_t n,
                             const int32_t *__restrict__ lab, const int32_t *__restrict__ rloc,
                             const PlanEntry *__restrict__ plan)
{
    pdl_begin();
    if (V.ctl->status != SIVF_OK) return;
    const int lane = threadIdx.x & 31, hl = lane & 15;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    const int d = V.d, C = V.C;
    // whole warps iterate together (the half sums shuffle across the warp)
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; 2 * w < n; w += nw) {
        const int64_t i = 2 * w + (lane >> 4);
        const int r0 = i < n ? rloc[i] : -1;
        const bool on = r0 >= 0;
        int64_t s = 0;
        int slot = 0;
        float ss = 0.f, rs = 0.f;
        if (on) {
            const int l = lab[i];
            const int r = V.runcnt[(size_t)l * V.nblk_max + (i >> 10)] + r0;
            const PlanEntry pe = plan[V.list_flag[l] - 1];
            if (r < pe.into_head) {
                s = pe.head_old;
                slot = pe.fill_old + r;
            } else {
                const int q = r - pe.into_head;
                s = V.dir[(size_t)l * V.dir_cap + pe.dir_pos0 + q / C];
                slot = q % C;
            }
            const size_t row = (size_t)s * C + slot;
            const float *xi = x + (size_t)i * d;
            const float inv = V.x8 ? V.inv_scale8[l] : 1.f;
            const float *cl = V.cent + (size_t)l * d;
            for (int j = hl * 4; j < d; j += 64) {
                const float4 v = *reinterpret_cast<const float4 *>(xi + j);
                *reinterpret_cast<float4 *>(V.x32 + row * d + j) = v;
                ss = fmaf(v.x, v.x, ss);
                ss = fmaf(v.y, v.y, ss);
                ss = fmaf(v.z, v.z, ss);
                ss = fmaf(v.w, v.w, ss);
                if (V.xb16) {
                    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
                    __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
                    uint2 pk;
                    pk.x = *reinterpret_cast<uint32_t *>(&lo);
                    pk.y = *reinterpret_cast<uint32_t *>(&hi);
                    *reinterpret_cast<uint2 *>(V.xb16 + row * d + j) = pk;
                }
                if (V.x8) {
                    // residual r = fl32(x - c_l), code = E4M3(fl32(r * inv))
                    const float4 c4 = *reinterpret_cast<const float4 *>(cl + j);
                    const float4 rv = make_float4(__fsub_rn(v.x, c4.x), __fsub_rn(v.y, c4.y),
                                                  __fsub_rn(v.z, c4.z), __fsub_rn(v.w, c4.w));
                    rs = fmaf(rv.x, rv.x, rs);
                    rs = fmaf(rv.y, rv.y, rs);
                    rs = fmaf(rv.z, rv.z, rs);
                    rs = fmaf(rv.w, rv.w, rs);
                    float2 a = make_float2(__fmul_rn(rv.x, inv), __fmul_rn(rv.y, inv));
                    float2 b = make_float2(__fmul_rn(rv.z, inv), __fmul_rn(rv.w, inv));
                    __nv_fp8x2_storage_t pa =
                        __nv_cvt_float2_to_fp8x2(a, __NV_SATFINITE, __NV_E4M3);
                    __nv_fp8x2_storage_t pb =
                        __nv_cvt_float2_to_fp8x2(b, __NV_SATFINITE, __NV_E4M3);
                    *reinterpret_cast<uint32_t *>(V.x8 + row * d + j) =
                        (uint32_t)pa | ((uint32_t)pb << 16);
                }
            }
        }
        ss = half_sum(ss);
        if (V.x8) rs = half_sum(rs);
        if (on && hl == 0) {
            const size_t row = (size_t)s * C + slot;
            const int64_t id = ids[i];
            V.xnorm[row] = ss;
            if (V.rnorm) V.rnorm[row] = rs;
            V.ids[row] = id;
            V.att[id] = (s << 32) | (int64_t)slot;
        }
        // payload, id and table entry are visible before the bit (Theorem 1)
        __threadfence();
        __syncwarp();
        if (on && hl == 0) {
            __threadfence();
            atomicOr(&V.bits[s * V.W + (slot >> 5)], 1u << (slot & 31));
        }
    }
}

__global__ void k_ins_cleanup(IndexView V, const int64_t *__restrict__ ids, int64_t n, int nblk,
                              const int32_t *__restrict__ touched)
{
    pdl_begin();
    GRID_STRIDE(i, n)
    {
        const int64_t id = ids[i];
        if (id >= 0 && id < V.n_max) V.claim[id] = -1;
    }
    const int nt = V.ctl->ntouched;
    GRID_STRIDE(e, (int64_t)nt * nblk)
    {
        const int l = touched[e / nblk];
        V.runcnt[(size_t)l * V.nblk_max + e % nblk] = 0;
        if (e % nblk == 0) V.list_flag[l] = 0;
    }
}

// ---------------------------------------------------------------- drivers
static int grid_for(int64_t n, int per_block)
{
    int64_t g = (n + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

void insert_batch(sivf_index *ix, const int64_t *ids, const float *x, int64_t n,
                  const InsertScratch &s, cudaStream_t st)
{
    IndexView V = view_of(ix);
    const int nblk = (int)((n + kRankTile - 1) / kRankTile);
    const int tmax = (int)std::min<int64_t>(n, ix->nlist);
    const int tok = prof_begin(ix, PROF_INSERT, 8, st);
    launch_pdl(k_ins_claim, grid_for(n, 256), 256, 0, st, V, ids, n);
    launch_pdl(k_ins_rank, nblk, 512, 0, st, V, ids, s.lab, n, s.rloc, s.touched);
    launch_pdl(k_ins_plan, (unsigned)(((int64_t)tmax * 32 + 127) / 128), 128, 0, st, V, nblk,
               s.touched, s.bcnt);
    launch_pdl(k_ins_overwrite, grid_for(n, 256), 256, 0, st, V, ids, n, s.rloc, s.affected);
    launch_pdl(k_reclaim, grid_for((int64_t)tmax * 32, 256), 256, 0, st, V, s.affected);
    launch_pdl(k_ins_alloc, (tmax + 127) / 128, 128, 0, st, V, s.touched, s.bcnt, s.plan);
    launch_pdl(k_ins_append, grid_for(n * 16, 256), 256, 0, st, V, ids, x, n, s.lab, s.rloc,
               s.plan);
    launch_pdl(k_ins_cleanup, grid_for(std::max<int64_t>(n, (int64_t)tmax * nblk), 256), 256, 0, st,
               V, ids, n, nblk, s.touched);
    prof_end(ix, tok, st);
}

void remove_batch(sivf_index *ix, const int64_t *ids, int64_t n, int32_t *affected,
                  cudaStream_t st)
{
    IndexView V = view_of(ix);
    const int tok = prof_begin(ix, PROF_REMOVE, 3, st);
    launch_pdl(k_rm_validate, grid_for(n, 256), 256, 0, st, V, ids, n);
    launch_pdl(k_rm_phase1, grid_for(n, 256), 256, 0, st, V, ids, n, affected);
    const int amax = (int)std::min<int64_t>(n, ix->nlist);
    launch_pdl(k_reclaim, grid_for((int64_t)amax * 32, 256), 256, 0, st, V, affected);
    prof_end(ix, tok, st);
}

}  // namespace sivf
