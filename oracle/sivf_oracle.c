/*
 * SIVF oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU model of the streaming IVF-Flat index
 * of "SIVF: GPU-Resident IVF Index for Streaming Vector Search"
 * (arxiv 2601.11808).  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no code,
 * header, table or helper with the CUDA library; the product path never
 * calls it.
 *
 * Floating point: every distance is FP64, summed over coordinates in index
 * order j = 0..d-1, each term (double(a_j) - double(b_j))^2.  The file is
 * compiled with -ffp-contract=off so that a*b+c is two roundings on every
 * host (x86-64 and aarch64 give the same bits).
 *
 * What each part follows (paper sections / algorithms):
 *   - coarse assignment and probe selection: the IVF coarse quantizer of
 *     Sec. 3.3 (nearest centroid by L2; the paper is silent on ties -- ties go
 *     to the lowest centroid index);
 *   - list scan and top-k: Algorithm 3 and the search complexity of
 *     Sec. 3.5.2 (exact scan of every live member of the probed lists; the
 *     metric is squared L2; ties go to the lower id; missing results are
 *     padded with (+inf, -1));
 *   - delete-then-insert overwrite: the data model paragraph of Sec. 3;
 *   - idempotent delete: Algorithm 4 and Theorem 3;
 *   - slab bookkeeping (which slab a vector lands in, when a slab is taken
 *     from or returned to the pool): Algorithm 1 (a list fills its head slab
 *     and takes a new slab only when the head is absent or full) and
 *     Algorithm 4 (a slab whose live count reaches zero goes back to the
 *     pool).  Slab *identities* are not modelled, only per-list sequences
 *     of slab records {fill, live}, so the model is independent of how a
 *     free stack orders its slabs.
 *   - batch semantics (a reading; the paper gives per-vector operations
 *     only): add(batch) = (1) keep the last occurrence of each id, (2) all-
 *     or-nothing admission: slab demand, computed on the state before the
 *     batch, must fit in the free slabs and in each list's directory
 *     capacity, (3) remove every kept id that is currently live, (4) append
 *     the kept ids in batch order.  remove(batch) removes each live id once;
 *     absent ids are no-ops.
 *   - compaction of partly-live slabs (the adaptive background compaction
 *     the conclusion names as future work; a reading, the paper gives no
 *     algorithm): a list whose live members would fit in at least
 *     `min_free` fewer slabs is rewritten densely in its own member order
 *     -- member j goes to slot j mod C of the list's (j div C)-th slab, the
 *     list keeps its oldest ceil(n / C) slabs and the rest go back to the
 *     pool.  Lists are taken in index order while the running total of
 *     rewritten members stays within `max_moves`; the first list that would
 *     pass it ends the pass.
 *   - reduced-precision encodings used by the precision path: bfloat16 with
 *     round-to-nearest-even, and FP8 E4M3 (OCP "fn" variant: bias 7, no
 *     infinities, max finite 448) with round-to-nearest-even and saturation
 *     to +-448, applied to v = x * inv_scale rounded to FP32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { O_OK = 0, O_E_ARG = 1, O_E_NOMEM = 2, O_E_STATE = 3 };

typedef struct {
    int32_t fill; /* slots ever written in this slab (monotone until freed) */
    int32_t live; /* live vectors in this slab */
    int32_t list; /* owning list, -1 once returned to the pool */
} orec;

typedef struct {
    int64_t n, cap;  /* members, in insertion order */
    int64_t *ids;
    float *x;        /* n * d */
    int64_t *rec;    /* slab record of each member */
    int32_t *slot;   /* slot of each member inside its slab */
    int64_t nrec, reccap;
    int64_t *recs;   /* this list's slab records, oldest first; last = head */
} olist;

typedef struct oivf {
    int d, nlist, C;
    int64_t n_max, n_slabs, dir_cap;
    float *cent;
    int have_cent;
    olist *lists;
    int32_t *where;  /* id -> list, or -1 */
    orec *recs;
    int64_t nrecs, recs_cap;
    int64_t free_slabs;
    int64_t ntotal;
} oivf;

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

static double sqdist(const float *a, const float *b, int d)
{
    double acc = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)a[j] - (double)b[j];
        acc += t * t;
    }
    return acc;
}

static void *xrealloc(void *p, size_t n)
{
    void *q = realloc(p, n ? n : 1);
    if (!q) abort();
    return q;
}

typedef struct {
    double d;
    int64_t key; /* centroid index or vector id */
} dk;

static int cmp_dk(const void *a, const void *b)
{
    const dk *x = (const dk *)a, *y = (const dk *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return 0;
}

int oivf_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* lifetime                                                             */
/* ------------------------------------------------------------------ */

oivf *oivf_create(int d, int nlist, int C, int64_t n_max, int64_t n_slabs,
                  int64_t dir_cap)
{
    if (d <= 0 || nlist <= 0 || C <= 0 || n_max <= 0 || n_slabs <= 0 ||
        dir_cap <= 0)
        return NULL;
    oivf *o = (oivf *)calloc(1, sizeof(oivf));
    o->d = d;
    o->nlist = nlist;
    o->C = C;
    o->n_max = n_max;
    o->n_slabs = n_slabs;
    o->dir_cap = dir_cap;
    o->cent = (float *)calloc((size_t)nlist * d, sizeof(float));
    o->lists = (olist *)calloc((size_t)nlist, sizeof(olist));
    o->where = (int32_t *)malloc((size_t)n_max * sizeof(int32_t));
    for (int64_t i = 0; i < n_max; ++i) o->where[i] = -1;
    o->free_slabs = n_slabs;
    return o;
}

void oivf_destroy(oivf *o)
{
    if (!o) return;
    for (int l = 0; l < o->nlist; ++l) {
        olist *L = &o->lists[l];
        free(L->ids);
        free(L->x);
        free(L->rec);
        free(L->slot);
        free(L->recs);
    }
    free(o->lists);
    free(o->cent);
    free(o->where);
    free(o->recs);
    free(o);
}

int oivf_set_centroids(oivf *o, const float *c)
{
    memcpy(o->cent, c, (size_t)o->nlist * o->d * sizeof(float));
    o->have_cent = 1;
    return O_OK;
}

/* ------------------------------------------------------------------ */
/* coarse quantizer                                                     */
/* ------------------------------------------------------------------ */

/* nearest centroid; strict '<' over ascending index keeps the lowest index
 * on ties */
static int32_t nearest(const oivf *o, const float *x)
{
    int32_t best = 0;
    double bd = sqdist(x, o->cent, o->d);
    for (int c = 1; c < o->nlist; ++c) {
        double dc = sqdist(x, o->cent + (size_t)c * o->d, o->d);
        if (dc < bd) {
            bd = dc;
            best = c;
        }
    }
    return best;
}

int oivf_assign(const oivf *o, const float *x, int64_t n, int32_t *out)
{
    if (!o->have_cent) return O_E_STATE;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) out[i] = nearest(o, x + (size_t)i * o->d);
    return O_OK;
}

/* the P nearest centroids of q, ascending by (distance, index) */
static void probes_of(const oivf *o, const float *q, int P, int32_t *out,
                      dk *tmp)
{
    for (int c = 0; c < o->nlist; ++c) {
        tmp[c].d = sqdist(q, o->cent + (size_t)c * o->d, o->d);
        tmp[c].key = c;
    }
    qsort(tmp, (size_t)o->nlist, sizeof(dk), cmp_dk);
    for (int p = 0; p < P; ++p) out[p] = (int32_t)tmp[p].key;
}

int oivf_probe(const oivf *o, const float *q, int64_t nq, int P, int32_t *out)
{
    if (!o->have_cent) return O_E_STATE;
    if (P < 1 || P > o->nlist) return O_E_ARG;
#pragma omp parallel
    {
        dk *tmp = (dk *)malloc((size_t)o->nlist * sizeof(dk));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < nq; ++i)
            probes_of(o, q + (size_t)i * o->d, P, out + (size_t)i * P, tmp);
        free(tmp);
    }
    return O_OK;
}

/* ------------------------------------------------------------------ */
/* search                                                               */
/* ------------------------------------------------------------------ */

/* exact scan of every member of the given lists, then the k smallest by
 * (distance, id); fewer than k candidates are padded with (+inf, -1) */
static void scan_lists(const oivf *o, const float *q, const int32_t *probes,
                       int P, int k, double *dist, int64_t *ids)
{
    int64_t ncand = 0;
    for (int p = 0; p < P; ++p) {
        int32_t l = probes[p];
        if (l >= 0 && l < o->nlist) ncand += o->lists[l].n;
    }
    dk *cand = (dk *)malloc((size_t)(ncand ? ncand : 1) * sizeof(dk));
    int64_t m = 0;
    for (int p = 0; p < P; ++p) {
        int32_t l = probes[p];
        if (l < 0 || l >= o->nlist) continue;
        /* a list probed twice is scanned once */
        int dup = 0;
        for (int pp = 0; pp < p; ++pp)
            if (probes[pp] == l) dup = 1;
        if (dup) continue;
        const olist *L = &o->lists[l];
        for (int64_t i = 0; i < L->n; ++i) {
            cand[m].d = sqdist(q, L->x + (size_t)i * o->d, o->d);
            cand[m].key = L->ids[i];
            ++m;
        }
    }
    qsort(cand, (size_t)m, sizeof(dk), cmp_dk);
    for (int j = 0; j < k; ++j) {
        if (j < m) {
            dist[j] = cand[j].d;
            ids[j] = cand[j].key;
        } else {
            dist[j] = INFINITY;
            ids[j] = -1;
        }
    }
    free(cand);
}

int oivf_search_with_probes(const oivf *o, const float *q, int64_t nq, int k,
                            int P, const int32_t *probes, double *dist,
                            int64_t *ids)
{
    if (k < 1 || P < 1) return O_E_ARG;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i)
        scan_lists(o, q + (size_t)i * o->d, probes + (size_t)i * P, P, k,
                   dist + (size_t)i * k, ids + (size_t)i * k);
    return O_OK;
}

int oivf_search(const oivf *o, const float *q, int64_t nq, int k, int P,
                double *dist, int64_t *ids)
{
    if (!o->have_cent) return O_E_STATE;
    if (k < 1 || P < 1 || P > o->nlist) return O_E_ARG;
#pragma omp parallel
    {
        dk *tmp = (dk *)malloc((size_t)o->nlist * sizeof(dk));
        int32_t *pr = (int32_t *)malloc((size_t)P * sizeof(int32_t));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < nq; ++i) {
            const float *qi = q + (size_t)i * o->d;
            probes_of(o, qi, P, pr, tmp);
            scan_lists(o, qi, pr, P, k, dist + (size_t)i * k,
                       ids + (size_t)i * k);
        }
        free(pr);
        free(tmp);
    }
    return O_OK;
}

/* brute-force k nearest live vectors (every list scanned) */
int oivf_exact_knn(const oivf *o, const float *q, int64_t nq, int k,
                   double *dist, int64_t *ids)
{
    if (k < 1) return O_E_ARG;
    int32_t *all = (int32_t *)malloc((size_t)o->nlist * sizeof(int32_t));
    for (int l = 0; l < o->nlist; ++l) all[l] = l;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i)
        scan_lists(o, q + (size_t)i * o->d, all, o->nlist, k,
                   dist + (size_t)i * k, ids + (size_t)i * k);
    free(all);
    return O_OK;
}

/* ------------------------------------------------------------------ */
/* slab bookkeeping model (Algorithms 1 and 4)                          */
/* ------------------------------------------------------------------ */

static int64_t new_record(oivf *o, int32_t list)
{
    if (o->nrecs == o->recs_cap) {
        o->recs_cap = o->recs_cap ? 2 * o->recs_cap : 1024;
        o->recs = (orec *)xrealloc(o->recs, (size_t)o->recs_cap * sizeof(orec));
    }
    int64_t u = o->nrecs++;
    o->recs[u].fill = 0;
    o->recs[u].live = 0;
    o->recs[u].list = list;
    olist *L = &o->lists[list];
    if (L->nrec == L->reccap) {
        L->reccap = L->reccap ? 2 * L->reccap : 8;
        L->recs = (int64_t *)xrealloc(L->recs, (size_t)L->reccap * sizeof(int64_t));
    }
    L->recs[L->nrec++] = u;
    o->free_slabs -= 1;
    return u;
}

/* Algorithm 4: clear the member, decrement its slab's live count and give
 * the slab back to the pool when nothing live remains in it. */
static void erase(oivf *o, int64_t id)
{
    int32_t l = o->where[id];
    olist *L = &o->lists[l];
    int64_t p = 0;
    while (L->ids[p] != id) ++p;
    int64_t u = L->rec[p];
    int64_t tail = L->n - p - 1;
    memmove(L->ids + p, L->ids + p + 1, (size_t)tail * sizeof(int64_t));
    memmove(L->x + (size_t)p * o->d, L->x + (size_t)(p + 1) * o->d,
            (size_t)tail * o->d * sizeof(float));
    memmove(L->rec + p, L->rec + p + 1, (size_t)tail * sizeof(int64_t));
    memmove(L->slot + p, L->slot + p + 1, (size_t)tail * sizeof(int32_t));
    L->n -= 1;
    o->where[id] = -1;
    o->ntotal -= 1;
    o->recs[u].live -= 1;
    if (o->recs[u].live == 0) {
        int64_t r = 0;
        while (L->recs[r] != u) ++r;
        memmove(L->recs + r, L->recs + r + 1,
                (size_t)(L->nrec - r - 1) * sizeof(int64_t));
        L->nrec -= 1;
        o->recs[u].list = -1;
        o->free_slabs += 1;
    }
}

/* Algorithm 1 (Insert): write into the head slab while it has a free slot,
 * otherwise take a fresh slab from the pool and make it the head. */
static void append(oivf *o, int32_t l, int64_t id, const float *x)
{
    olist *L = &o->lists[l];
    int64_t u = -1;
    if (L->nrec > 0) {
        int64_t h = L->recs[L->nrec - 1];
        if (o->recs[h].fill < o->C) u = h;
    }
    if (u < 0) u = new_record(o, l);
    int32_t slot = o->recs[u].fill;
    o->recs[u].fill += 1;
    o->recs[u].live += 1;
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->ids = (int64_t *)xrealloc(L->ids, (size_t)L->cap * sizeof(int64_t));
        L->x = (float *)xrealloc(L->x, (size_t)L->cap * o->d * sizeof(float));
        L->rec = (int64_t *)xrealloc(L->rec, (size_t)L->cap * sizeof(int64_t));
        L->slot = (int32_t *)xrealloc(L->slot, (size_t)L->cap * sizeof(int32_t));
    }
    L->ids[L->n] = id;
    memcpy(L->x + (size_t)L->n * o->d, x, (size_t)o->d * sizeof(float));
    L->rec[L->n] = u;
    L->slot[L->n] = slot;
    L->n += 1;
    o->where[id] = l;
    o->ntotal += 1;
}

int oivf_add(oivf *o, const int64_t *ids, const float *x, int64_t n,
             int64_t *n_added)
{
    if (n_added) *n_added = 0;
    if (!o->have_cent) return O_E_STATE;
    if (n < 0) return O_E_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (ids[i] < 0 || ids[i] >= o->n_max) return O_E_ARG;
    if (n == 0) return O_OK;

    /* (1) the last occurrence of every id wins */
    int64_t *last = (int64_t *)malloc((size_t)o->n_max * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) last[ids[i]] = i;
    char *win = (char *)malloc((size_t)n);
    for (int64_t i = 0; i < n; ++i) win[i] = (last[ids[i]] == i);
    free(last);

    int32_t *lab = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    oivf_assign(o, x, n, lab);

    /* (2) admission on the state before the batch */
    int64_t *cnt = (int64_t *)calloc((size_t)o->nlist, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        if (win[i]) cnt[lab[i]] += 1;
    int64_t demand = 0;
    int status = O_OK;
    for (int l = 0; l < o->nlist; ++l) {
        if (!cnt[l]) continue;
        const olist *L = &o->lists[l];
        int64_t avail = 0;
        if (L->nrec > 0) avail = o->C - o->recs[L->recs[L->nrec - 1]].fill;
        int64_t need = cnt[l] > avail ? (cnt[l] - avail + o->C - 1) / o->C : 0;
        if (L->nrec + need > o->dir_cap) status = O_E_NOMEM;
        demand += need;
    }
    if (demand > o->free_slabs) status = O_E_NOMEM;
    free(cnt);
    if (status != O_OK) {
        free(win);
        free(lab);
        return status;
    }

    /* (3) delete-then-insert: every kept id that is live is removed first */
    for (int64_t i = 0; i < n; ++i)
        if (win[i] && o->where[ids[i]] >= 0) erase(o, ids[i]);

    /* (4) append in batch order */
    int64_t added = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!win[i]) continue;
        append(o, lab[i], ids[i], x + (size_t)i * o->d);
        ++added;
    }
    free(win);
    free(lab);
    if (n_added) *n_added = added;
    return O_OK;
}

int oivf_remove(oivf *o, const int64_t *ids, int64_t n, int64_t *n_removed)
{
    if (n_removed) *n_removed = 0;
    if (n < 0) return O_E_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (ids[i] < 0 || ids[i] >= o->n_max) return O_E_ARG;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (o->where[ids[i]] < 0) continue; /* absent: no-op (Theorem 3) */
        erase(o, ids[i]);
        ++cnt;
    }
    if (n_removed) *n_removed = cnt;
    return O_OK;
}

/* Compaction (see the header): rewrite list l densely in member order. */
static void compact_list(oivf *o, int l)
{
    olist *L = &o->lists[l];
    const int64_t keep = (L->n + o->C - 1) / o->C;
    for (int64_t j = 0; j < L->n; ++j) {
        L->rec[j] = L->recs[j / o->C];
        L->slot[j] = (int32_t)(j % o->C);
    }
    for (int64_t r = 0; r < L->nrec; ++r) {
        orec *R = &o->recs[L->recs[r]];
        if (r < keep) {
            int64_t f = L->n - r * o->C;
            R->fill = (int32_t)(f < o->C ? f : o->C);
            R->live = R->fill;
        } else {
            R->list = -1;
            R->fill = 0;
            R->live = 0;
        }
    }
    o->free_slabs += L->nrec - keep;
    L->nrec = keep;
}

int oivf_compact(oivf *o, int32_t min_free, int64_t max_moves, int64_t *n_freed,
                 int64_t *n_moved)
{
    if (n_freed) *n_freed = 0;
    if (n_moved) *n_moved = 0;
    if (min_free < 1 || max_moves < 1) return O_E_ARG;
    int64_t moved = 0, freed = 0;
    for (int l = 0; l < o->nlist; ++l) {
        const olist *L = &o->lists[l];
        const int64_t keep = (L->n + o->C - 1) / o->C;
        if (L->nrec - keep < min_free) continue;
        if (moved + L->n > max_moves) break;
        moved += L->n;
        freed += L->nrec - keep;
        compact_list(o, l);
    }
    if (n_freed) *n_freed = freed;
    if (n_moved) *n_moved = moved;
    return O_OK;
}

/* FP64 squared distances of q to n vectors (the definition, one by one) */
void oivf_dists(const float *q, const float *x, int64_t n, int d, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = sqdist(q, x + (size_t)i * d, d);
}

/* ------------------------------------------------------------------ */
/* introspection                                                        */
/* ------------------------------------------------------------------ */

int64_t oivf_ntotal(const oivf *o) { return o->ntotal; }
int64_t oivf_free_slabs(const oivf *o) { return o->free_slabs; }
int32_t oivf_list_of(const oivf *o, int64_t id)
{
    return (id >= 0 && id < o->n_max) ? o->where[id] : -1;
}
int64_t oivf_list_size(const oivf *o, int l) { return o->lists[l].n; }
int64_t oivf_list_nslabs(const oivf *o, int l) { return o->lists[l].nrec; }

/* members of list l in insertion order, with the slab sequence number (the
 * position of their slab in the list's slab sequence, oldest = 0) and slot */
void oivf_list_members(const oivf *o, int l, int64_t *ids, int32_t *slab_seq,
                       int32_t *slot)
{
    const olist *L = &o->lists[l];
    for (int64_t i = 0; i < L->n; ++i) {
        if (ids) ids[i] = L->ids[i];
        if (slot) slot[i] = L->slot[i];
        if (slab_seq) {
            int32_t r = 0;
            while (L->recs[r] != L->rec[i]) ++r;
            slab_seq[i] = r;
        }
    }
}

void oivf_list_vectors(const oivf *o, int l, float *x)
{
    const olist *L = &o->lists[l];
    memcpy(x, L->x, (size_t)L->n * o->d * sizeof(float));
}

/* fill and live count of each slab of list l, oldest first */
void oivf_list_slabs(const oivf *o, int l, int32_t *fill, int32_t *live)
{
    const olist *L = &o->lists[l];
    for (int64_t r = 0; r < L->nrec; ++r) {
        fill[r] = o->recs[L->recs[r]].fill;
        live[r] = o->recs[L->recs[r]].live;
    }
}

/* ------------------------------------------------------------------ */
/* reduced-precision encodings                                          */
/* ------------------------------------------------------------------ */

static uint32_t f2u(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* bfloat16: keep the top 16 bits of the FP32 pattern, rounding the dropped
 * 16 bits to nearest, ties to even; NaN stays a quiet NaN */
void oivf_to_bf16(const float *in, uint16_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = f2u(in[i]);
        if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) {
            out[i] = (uint16_t)((u >> 16) | 0x0040u);
            continue;
        }
        uint32_t upper = u >> 16, lower = u & 0xffffu;
        if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1;
        out[i] = (uint16_t)upper;
    }
}

void oivf_from_bf16(const uint16_t *in, float *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = (uint32_t)in[i] << 16;
        memcpy(&out[i], &u, 4);
    }
}

/* value of an E4M3 code: sign, 4 exponent bits (bias 7), 3 mantissa bits;
 * exponent field 0 is subnormal (m/8 * 2^-6); S.1111.111 is NaN */
static double e4m3_value(uint8_t c)
{
    int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
    double v;
    if (e == 15 && m == 7) return NAN;
    if (e == 0)
        v = ldexp((double)m / 8.0, -6);
    else
        v = ldexp(1.0 + (double)m / 8.0, e - 7);
    return s ? -v : v;
}

void oivf_from_e4m3(const uint8_t *in, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_value(in[i]);
}

/* E4M3 encoding of v = fl32(x * inv_scale): the nearest code value, ties to
 * the code with an even mantissa, |v| above the largest finite value
 * saturates to +-448.  Found by plain search over the 127 non-negative
 * finite codes (obviously correct, slow). */
void oivf_to_e4m3(const float *in, float inv_scale, uint8_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        float vf = (float)((double)in[i] * (double)inv_scale);
        double v = (double)vf;
        if (isnan(v)) {
            out[i] = 0x7f;
            continue;
        }
        uint8_t sign = (v < 0 || (v == 0 && signbit(v))) ? 0x80 : 0;
        double a = fabs(v);
        uint8_t best = 0;
        double bd = INFINITY;
        for (int c = 0; c <= 0x7e; ++c) {
            double cv = e4m3_value((uint8_t)c);
            double dd = fabs(cv - a);
            if (dd < bd || (dd == bd && (c & 1) == 0 && (best & 1) == 1)) {
                bd = dd;
                best = (uint8_t)c;
            }
        }
        if (a >= 448.0) best = 0x7e;
        out[i] = (uint8_t)(sign | best);
    }
}

/* ------------------------------------------------------------------ */
/* approximate distance of the reduced-precision scan                   */
/* ------------------------------------------------------------------ */
/*
 * The paper scans FP32 payloads only (Algorithm 3).  The precision path of
 * this build scans a rounded copy of every list, keeps each query's best 4k
 * members by an approximate distance and re-ranks those exactly in FP32.
 * This is the FP64 value of that approximate distance for one query q and
 * rows x (the reading of the precision pattern this build takes; the
 * paper has no passage for it):
 *
 *   mode 0 (BF16): ||q||^2 + ||x||^2 - 2 sum_j bf(q_j) bf(x_j), the norms
 *     of the unrounded FP32 vectors and bf() the bfloat16 rounding above;
 *   mode 1 (FP8 E4M3 residual codes): with the row's list centroid c
 *     (cent, one row of d per x row), r = fl32(q - c), y = fl32(x - c),
 *     the list's inverse scale t_l (inv_l, one per row) and the query's
 *     own t_q = fl32(448 / fl32(2 max_j |r_j|)) (1 when r = 0):
 *     ||r||^2 + ||y||^2 - 2 s sum_j e(r_j, t_q) e(y_j, t_l), where
 *     e(v, t) is the value of the E4M3 code of fl32(v t) (encoder above)
 *     and s = 1 / (t_l t_q) undoes both scales.
 *
 * mag[i] (optional) = the two norms + 2 s sum_j |code products|: the size
 * against which an FP32 accumulation of the same terms is judged.
 */
static float bf16_round(float v)
{
    uint16_t b;
    float r;
    oivf_to_bf16(&v, &b, 1);
    oivf_from_bf16(&b, &r, 1);
    return r;
}

static double e4m3_round(float v, float inv_scale)
{
    uint8_t c;
    double r;
    oivf_to_e4m3(&v, inv_scale, &c, 1);
    oivf_from_e4m3(&c, &r, 1);
    return r;
}

void oivf_approx_dists(const float *q, const float *x, int64_t n, int d, int mode,
                       const float *cent, const float *inv_l, double *out, double *mag)
{
    for (int64_t i = 0; i < n; ++i) {
        const float *xi = x + (size_t)i * d;
        double qn = 0.0, xn = 0.0, dot = 0.0, ab = 0.0, s = 1.0;
        if (mode == 0) {
            for (int j = 0; j < d; ++j) {
                qn += (double)q[j] * (double)q[j];
                xn += (double)xi[j] * (double)xi[j];
                const double p = (double)bf16_round(q[j]) * (double)bf16_round(xi[j]);
                dot += p;
                ab += fabs(p);
            }
        } else {
            const float *c = cent + (size_t)i * d;
            float mx = 0.0f;
            for (int j = 0; j < d; ++j) {
                const float r = q[j] - c[j];
                if (fabsf(r) > mx) mx = fabsf(r);
            }
            const float tq = mx > 0.0f ? 448.0f / (2.0f * mx) : 1.0f;
            for (int j = 0; j < d; ++j) {
                const float r = q[j] - c[j];
                const float y = xi[j] - c[j];
                qn += (double)r * (double)r;
                xn += (double)y * (double)y;
                const double p = e4m3_round(r, tq) * e4m3_round(y, inv_l[i]);
                dot += p;
                ab += fabs(p);
            }
            s = 1.0 / ((double)inv_l[i] * (double)tq);
        }
        out[i] = qn + xn - 2.0 * s * dot;
        if (mag) mag[i] = qn + xn + 2.0 * s * ab;
    }
}

/* ------------------------------------------------------------------ */
/* coarse quantizer training                                            */
/* ------------------------------------------------------------------ */
/*
 * The paper takes its coarse quantizer from Faiss and does not describe
 * training (Sec. 4.1).  The reading used here is Lloyd's k-means:
 *   - initial centroids: nlist distinct training rows.  Row r_t is the t-th
 *     output of SplitMix64 (Steele, Lea and Flood, "Fast splittable
 *     pseudorandom number generators", OOPSLA 2014) from the state `seed`,
 *     reduced mod n; a row already taken is skipped;
 *   - one iteration: every row goes to its nearest centroid (the FP64
 *     definition of the coarse quantizer above, ties to the lowest index);
 *     every centroid with at least one row becomes the FP32 rounding of the
 *     FP64 mean of its rows, summed in row order; a centroid with no rows
 *     keeps its value.
 */

/* SplitMix64: the state advances by the golden-ratio increment; the output
 * is the state passed through two xor-shift-multiply rounds and a final
 * xor-shift. */
static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void oivf_splitmix64(uint64_t seed, int64_t n, uint64_t *out)
{
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) out[i] = splitmix64_next(&s);
}

/* nearest of `nlist` centroids `c` to x; ties to the lowest index */
static int32_t nearest_of(const float *c, int nlist, int d, const float *x)
{
    int32_t best = 0;
    double bd = sqdist(x, c, d);
    for (int k = 1; k < nlist; ++k) {
        double dk = sqdist(x, c + (size_t)k * d, d);
        if (dk < bd) {
            bd = dk;
            best = k;
        }
    }
    return best;
}

/* the initial rows; returns -1 when fewer than nlist distinct rows exist */
int oivf_kmeans_init_rows(int64_t n, int nlist, uint64_t seed, int64_t *rows)
{
    if (n < nlist) return -1;
    unsigned char *taken = calloc((size_t)n, 1);
    if (!taken) return -1;
    uint64_t s = seed;
    int k = 0;
    while (k < nlist) {
        int64_t r = (int64_t)(splitmix64_next(&s) % (uint64_t)n);
        if (taken[r]) continue;
        taken[r] = 1;
        rows[k++] = r;
    }
    free(taken);
    return 0;
}

/* Lloyd's k-means as above; cent (nlist x d) receives the result; lab (n)
 * the assignment to the final centroids (may be NULL).  Returns O_OK or
 * O_E_ARG. */
int oivf_kmeans(const float *x, int64_t n, int d, int nlist, int iters, uint64_t seed,
                float *cent, int32_t *lab_out)
{
    if (n < nlist || nlist < 1 || d < 1 || iters < 0) return O_E_ARG;
    int64_t *rows = malloc(sizeof(int64_t) * (size_t)nlist);
    int32_t *lab = malloc(sizeof(int32_t) * (size_t)n);
    double *sum = malloc(sizeof(double) * (size_t)nlist * d);
    int64_t *cnt = malloc(sizeof(int64_t) * (size_t)nlist);
    if (!rows || !lab || !sum || !cnt || oivf_kmeans_init_rows(n, nlist, seed, rows)) {
        free(rows);
        free(lab);
        free(sum);
        free(cnt);
        return O_E_ARG;
    }
    for (int k = 0; k < nlist; ++k)
        memcpy(cent + (size_t)k * d, x + (size_t)rows[k] * d, sizeof(float) * (size_t)d);
    for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) lab[i] = nearest_of(cent, nlist, d, x + (size_t)i * d);
        memset(sum, 0, sizeof(double) * (size_t)nlist * d);
        memset(cnt, 0, sizeof(int64_t) * (size_t)nlist);
        for (int64_t i = 0; i < n; ++i) {
            const int32_t k = lab[i];
            ++cnt[k];
            for (int j = 0; j < d; ++j) sum[(size_t)k * d + j] += (double)x[(size_t)i * d + j];
        }
        for (int k = 0; k < nlist; ++k)
            if (cnt[k] > 0)
                for (int j = 0; j < d; ++j)
                    cent[(size_t)k * d + j] = (float)(sum[(size_t)k * d + j] / (double)cnt[k]);
    }
    if (lab_out) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) lab_out[i] = nearest_of(cent, nlist, d, x + (size_t)i * d);
    }
    free(rows);
    free(lab);
    free(sum);
    free(cnt);
    return O_OK;
}

/*
 * FP8 residual codes (precision path; no passage, a reading): list l keeps
 * E4M3(fl32(fl32(x_j - c_lj) * s_l)) with s_l = fl32(448 / R_l), R_l the
 * distance from c_l to its nearest other centroid (FP64, squared distance
 * summed in index order); with a single list or R_l = 0 the raw-magnitude
 * rule fl32(448 / (2 max_j |c_lj|)) (1 for a zero centroid).
 */
void oivf_fp8_list_scales(const float *cent, int nlist, int d, float *out)
{
    for (int l = 0; l < nlist; ++l) {
        const float *cl = cent + (size_t)l * d;
        double best = INFINITY;
        for (int o = 0; o < nlist; ++o) {
            if (o == l) continue;
            const double s = sqdist(cl, cent + (size_t)o * d, d);
            if (s < best) best = s;
        }
        if (best > 0.0 && best < INFINITY) {
            out[l] = (float)(448.0 / sqrt(best));
        } else {
            double mx = 0.0;
            for (int j = 0; j < d; ++j) mx = fmax(mx, fabs((double)cl[j]));
            out[l] = mx > 0.0 ? (float)(448.0 / (2.0 * mx)) : 1.0f;
        }
    }
}
