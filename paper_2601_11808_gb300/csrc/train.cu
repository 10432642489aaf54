// Training of the coarse quantizer (the paper takes a trained Faiss
// quantizer, Sec. 4.1, and does not describe training): Lloyd's k-means.
// The assignment step is the exact coarse assignment of coarse.cu; this
// file holds the other steps: the initial centroids (given training rows),
// the per-centroid FP64 sums and counts of the assigned rows, and the new
// centroids as the FP32 rounding of the FP64 means (a centroid with no rows
// keeps its value).
#include "device_utils.cuh"
#include "kernels.cuh"

namespace sivf {

__global__ void k_train_gather(const float *__restrict__ x, int d, const int64_t *__restrict__ rows,
                               int L, float *__restrict__ cent)
{
    pdl_begin();
    const int64_t n = (int64_t)L * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        cent[e] = x[(size_t)rows[e / d] * d + e % d];
}

// one warp per row: the row's label, then every coordinate added in FP64
__global__ void k_train_accum(const float *__restrict__ x, int64_t n, int d,
                              const int32_t *__restrict__ lab, double *__restrict__ sum,
                              int32_t *__restrict__ cnt)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const int32_t c = lab[i];
        if (lane == 0) atomicAdd(&cnt[c], 1);
        const float *xr = x + (size_t)i * d;
        double *sr = sum + (size_t)c * d;
        for (int j = lane; j < d; j += 32) atomicAdd(&sr[j], (double)xr[j]);
    }
}

__global__ void k_train_update(const double *__restrict__ sum, const int32_t *__restrict__ cnt,
                               int L, int d, float *__restrict__ cent)
{
    pdl_begin();
    const int64_t n = (int64_t)L * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[e / d];
        if (c > 0) cent[e] = __double2float_rn(__ddiv_rn(sum[e], (double)c));
    }
}

void train_gather(sivf_index *ix, const float *x, const int64_t *rows, cudaStream_t st)
{
    ix->launches += 1;
    const int64_t n = (int64_t)ix->nlist * ix->d;
    launch_pdl(k_train_gather, (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st, x,
               ix->d, rows, ix->nlist, ix->cent);
}

void train_step(sivf_index *ix, const float *x, int64_t n, const int32_t *lab, double *sum,
                int32_t *cnt, cudaStream_t st)
{
    const int L = ix->nlist, d = ix->d;
    cudaMemsetAsync(sum, 0, sizeof(double) * (size_t)L * d, st);
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)L, st);
    ix->launches += 2;
    launch_pdl(k_train_accum, (unsigned)std::min<int64_t>((n * 32 + 255) / 256, 152 * 16), 256, 0,
               st, x, n, d, lab, sum, cnt);
    const int64_t e = (int64_t)L * d;
    launch_pdl(k_train_update, (unsigned)std::min<int64_t>((e + 255) / 256, 152 * 8), 256, 0, st,
               sum, cnt, L, d, ix->cent);
}

}  // namespace sivf
