// Checkpoint of the whole device state of an index (no counterpart in the
// paper, whose index lives only as long as its process): sivf_save writes
// the create configuration and every array that carries state to a file;
// sivf_load creates an index with that configuration and restores the
// arrays, so the loaded index equals the saved one bit for bit and resumes
// with the same results.  Derived arrays (centroid norms and bounds, the
// BF16 copies of the centroids, the TMA descriptors) are recomputed; the
// per-call bookkeeping arrays are at their between-call values in both.
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "kernels.cuh"

namespace {

constexpr char kMagic[8] = {'S', 'I', 'V', 'F', 'C', 'K', 'P', '1'};
constexpr uint32_t kVersion = 1;
constexpr size_t kStage = (size_t)64 << 20;  // pinned staging buffer

struct Header {
    char magic[8];
    uint32_t version;
    int32_t d, nlist, C;
    int64_t n_max, n_slabs, dir_cap;
    uint32_t dtypes, have_centroids;
};

struct Array {
    void *dev;
    size_t bytes;
};

// every array that carries state, in file order (null ones are absent from
// the index and from the file)
std::vector<Array> state_arrays(sivf_index *ix)
{
    const size_t S = (size_t)ix->n_slabs, rows = S * ix->C, L = ix->nlist, d = ix->d;
    return {
        {ix->cent, L * d * 4},
        {ix->inv_scale8, L * 4},
        {ix->x32, rows * d * 4},
        {ix->xb16, ix->xb16 ? rows * d * 2 : 0},
        {ix->x8, ix->x8 ? rows * d : 0},
        {ix->xnorm, rows * 4},
        {ix->rnorm, ix->rnorm ? rows * 4 : 0},
        {ix->ids, rows * 8},
        {ix->bits, S * ix->W * 4},
        {ix->meta, S * sizeof(sivf::SlabMeta)},
        {ix->free_list, S * 4},
        {ix->free_top, 4},
        {ix->head, L * 4},
        {ix->nslabs, L * 4},
        {ix->list_live, L * 4},
        {ix->dir, L * (size_t)ix->dir_cap * 4},
        {ix->att, (size_t)ix->n_max * 8},
        {ix->stat, 4 * 8},
    };
}

struct File {
    FILE *f = nullptr;
    ~File()
    {
        if (f) fclose(f);
    }
};

struct Pinned {
    void *p = nullptr;
    ~Pinned()
    {
        if (p) cudaFreeHost(p);
    }
};

}  // namespace

extern "C" {

sivf_status sivf_save(sivf_index *ix, const char *path, void *stream)
{
    if (!ix || !path) return SIVF_E_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return sivf::set_error(ix, SIVF_E_CUDA, "stream synchronize failed");
    uint32_t err = 0;
    if (cudaMemcpy(&err, ix->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return sivf::set_error(ix, SIVF_E_CUDA, "reading the error word failed");
    if (err) return sivf::set_error(ix, SIVF_E_CORRUPT, "the index has a device error; not saved");
    File out;
    out.f = fopen(path, "wb");
    if (!out.f) return sivf::set_error(ix, SIVF_E_ARG, "cannot open the checkpoint file for writing");
    Header h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.d = ix->d;
    h.nlist = ix->nlist;
    h.C = ix->C;
    h.n_max = ix->n_max;
    h.n_slabs = ix->n_slabs;
    h.dir_cap = ix->dir_cap;
    h.dtypes = ix->dtypes;
    h.have_centroids = ix->have_centroids ? 1u : 0u;
    if (fwrite(&h, sizeof(h), 1, out.f) != 1)
        return sivf::set_error(ix, SIVF_E_ARG, "checkpoint write failed");
    Pinned buf;
    if (cudaMallocHost(&buf.p, kStage) != cudaSuccess)
        return sivf::set_error(ix, SIVF_E_NOMEM, "pinned staging buffer");
    for (const Array &a : state_arrays(ix)) {
        const uint64_t n = a.dev ? a.bytes : 0;
        if (fwrite(&n, 8, 1, out.f) != 1)
            return sivf::set_error(ix, SIVF_E_ARG, "checkpoint write failed");
        for (size_t off = 0; off < n; off += kStage) {
            const size_t len = std::min(kStage, (size_t)n - off);
            if (cudaMemcpy(buf.p, (const char *)a.dev + off, len, cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return sivf::set_error(ix, SIVF_E_CUDA, "device read failed");
            if (fwrite(buf.p, 1, len, out.f) != len)
                return sivf::set_error(ix, SIVF_E_ARG, "checkpoint write failed");
        }
    }
    if (fflush(out.f) != 0) return sivf::set_error(ix, SIVF_E_ARG, "checkpoint write failed");
    return SIVF_OK;
}

sivf_status sivf_load(const char *path, sivf_index **out)
{
    if (!path || !out) return SIVF_E_ARG;
    *out = nullptr;
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return SIVF_E_ARG;
    Header h;
    if (fread(&h, sizeof(h), 1, in.f) != 1 || memcmp(h.magic, kMagic, 8) != 0 ||
        h.version != kVersion)
        return SIVF_E_ARG;
    sivf_config cfg;
    cfg.d = h.d;
    cfg.nlist = h.nlist;
    cfg.slab_size = h.C;
    cfg.n_max = h.n_max;
    cfg.n_slabs = h.n_slabs;
    cfg.dir_cap = h.dir_cap;
    cfg.scan_dtypes = h.dtypes;
    sivf_index *ix = nullptr;
    sivf_status st = sivf_create(&cfg, &ix);
    if (st) return st;
    auto bad = [&](sivf_status s, const char *what) {
        sivf::set_error(ix, s, what);
        sivf_destroy(ix);
        return s;
    };
    if (ix->dir_cap != h.dir_cap) return bad(SIVF_E_ARG, "checkpoint configuration mismatch");
    Pinned buf;
    if (cudaMallocHost(&buf.p, kStage) != cudaSuccess) return bad(SIVF_E_NOMEM, "pinned staging buffer");
    std::vector<float> scales((size_t)h.nlist);
    int idx = 0;
    for (const Array &a : state_arrays(ix)) {
        uint64_t n = 0;
        if (fread(&n, 8, 1, in.f) != 1 || n != (a.dev ? a.bytes : 0))
            return bad(SIVF_E_ARG, "checkpoint array size mismatch or truncated file");
        for (size_t off = 0; off < n; off += kStage) {
            const size_t len = std::min(kStage, (size_t)n - off);
            if (fread(buf.p, 1, len, in.f) != len) return bad(SIVF_E_ARG, "truncated checkpoint");
            if (idx == 1) {  // FP8 scales: restored after the centroid preparation
                memcpy((char *)scales.data() + off, buf.p, len);
                continue;
            }
            if (cudaMemcpy((char *)a.dev + off, buf.p, len, cudaMemcpyHostToDevice) != cudaSuccess)
                return bad(SIVF_E_CUDA, "device write failed");
        }
        ++idx;
    }
    if (h.have_centroids) {
        sivf::centroid_prep(ix, 0);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            sivf::assign_stage_choose(ix, 0) != cudaSuccess)
            return bad(SIVF_E_CUDA, "centroid preparation failed");
        ix->have_centroids = true;
    }
    if (cudaMemcpy(ix->inv_scale8, scales.data(), scales.size() * 4, cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return bad(SIVF_E_CUDA, "device write failed");
    int64_t live = 0;
    if (cudaMemcpy(&live, ix->stat, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return bad(SIVF_E_CUDA, "device read failed");
    ix->ntotal_hint = live;
    *out = ix;
    return SIVF_OK;
}

}  // extern "C"
