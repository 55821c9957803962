// K5: near-zone product with the stored blocks plus the self term (eq. 2):
//   y_a = alpha_a c_a + sum over stored pairs (a, b) of N_ab c_b   (alpha of a's scatterer),
// N_ab = P_a G_{a-b} P_b^T for boxes within Chebyshev distance 1 (the self block
// without coincident dipoles).  Blocks are nb_a x nb_b column-major, so the threads
// of a CTA (one per test row i) read a column contiguously.  HBM-bound on the blocks.
#include "ie_internal.h"

namespace ie {
namespace {

__global__ void near_kernel(const int32_t *__restrict__ nb, const int64_t *__restrict__ off, int64_t n,
                            const int32_t *__restrict__ start, const int32_t *__restrict__ src,
                            const int64_t *__restrict__ boff, const float2 *__restrict__ Nblk,
                            const double *__restrict__ alpha_box,
                            const float2 *__restrict__ c, float2 *__restrict__ y, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ float2 cs[kNU];
    int a = blockIdx.x, r = blockIdx.y;
    int na = nb[a];
    const double alpha = alpha_box[a];
    const float2 *cr = c + (int64_t)r * n;
    // threads own rows i = threadIdx.x + k*blockDim.x (at most 2 per thread for 192 rows)
    double accr[2] = {0, 0}, acci[2] = {0, 0};
    for (int t = start[a]; t < start[a + 1]; ++t) {
        int b = src[t];
        int nbb = nb[b];
        __syncthreads();
        for (int j = threadIdx.x; j < nbb; j += blockDim.x) cs[j] = cr[off[b] + j];
        __syncthreads();
        const float2 *N = Nblk + boff[t];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            int i = threadIdx.x + k * blockDim.x;
            if (i >= na) continue;
            float pr = 0.f, pi = 0.f;
            for (int j = 0; j < nbb; ++j) {
                float2 v = N[(int64_t)j * na + i];
                float2 x = cs[j];
                pr = fmaf(v.x, x.x, fmaf(-v.y, x.y, pr));
                pi = fmaf(v.x, x.y, fmaf(v.y, x.x, pi));
            }
            accr[k] += pr;
            acci[k] += pi;
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        int i = threadIdx.x + k * blockDim.x;
        if (i >= na) continue;
        float2 x = cr[off[a] + i];
        y[(int64_t)r * n + off[a] + i] =
            make_float2((float)(accr[k] + alpha * x.x), (float)(acci[k] + alpha * x.y));
    }
}

}  // namespace

ie_status launch_near(const ie_plan p, const float2 *c, float2 *y, int nrhs, cudaStream_t st, const int *gate) {
    int maxnb = 0;
    for (int v : p->nb) maxnb = v > maxnb ? v : maxnb;
    int threads = maxnb <= 32 ? 32 : (maxnb <= 64 ? 64 : (maxnb <= 128 ? 128 : 96));
    if (maxnb > 128) threads = 96;   // 2 rows per thread up to 192
    near_kernel<<<dim3(p->nbox, nrhs), threads, 0, st>>>(p->d_nb, p->d_off, p->n, p->d_near_start, p->d_near_src,
                                                         p->d_near_boff, p->d_Nblk, p->d_alpha_box, c, y, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie
