// K5: near-zone product with the stored blocks plus the self term (eq. 2):
//   y_a = alpha_a c_a + sum over stored pairs (a, b) of N_ab c_b   (alpha of a's scatterer),
// N_ab = P_a G_{a-b} P_b^T for boxes within Chebyshev distance 1 (the self block
// without coincident dipoles).  Blocks are nb_a x nb_b column-major, so a warp's lanes
// (one per test row) read a column contiguously.  HBM-bound on the blocks.
#include "ie_internal.h"

namespace ie {
namespace {

constexpr int kNearWarps = 8;

// One CTA per (test box a, rhs); its 8 warps split the stored blocks of row a.  A warp
// takes whole blocks: lane l owns rows l, l + 32, ... (ROWS of them, na <= 32 ROWS); the
// block's source coefficients sit in the lanes' registers and are broadcast by
// shuffles.  Columns go in groups of G whose loads are all issued before the group's
// arithmetic, so each lane keeps G x ROWS independent reads in flight.  Per block the
// sums run in FP32 and are added into FP64 per-warp totals, combined in shared memory.
template <int ROWS>
__global__ void __launch_bounds__(kNearWarps * 32, 2)
near_kernel(const int32_t *__restrict__ nb, const int64_t *__restrict__ off, int64_t n,
            const int32_t *__restrict__ start, const int32_t *__restrict__ src,
            const int64_t *__restrict__ boff, const float2 *__restrict__ Nblk,
            const double *__restrict__ alpha_box,
            const float2 *__restrict__ c, float2 *__restrict__ y, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    constexpr int G = ROWS == 1 ? 16 : (ROWS == 2 ? 8 : 4);     // columns per load group
    constexpr int XR = ROWS;                                     // source values per lane (every nb <= 32 ROWS)
    __shared__ double2 part[kNearWarps][32 * ROWS];
    const int a = blockIdx.x, r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int na = nb[a];
    const float2 *cr = c + (int64_t)r * n;
    double2 acc[ROWS];
#pragma unroll
    for (int k = 0; k < ROWS; ++k) acc[k] = make_double2(0, 0);
    for (int t = start[a] + warp; t < start[a + 1]; t += kNearWarps) {
        const int b = src[t];
        const int nbb = nb[b];
        const float2 *cb = cr + off[b];
        float2 xs[XR];                           // c_b[lane + 32 m]
#pragma unroll
        for (int m = 0; m < XR; ++m) {
            const int j = lane + 32 * m;
            xs[m] = j < nbb ? cb[j] : make_float2(0.f, 0.f);
        }
        const float2 *N = Nblk + boff[t];
        float2 p[ROWS];
#pragma unroll
        for (int k = 0; k < ROWS; ++k) p[k] = make_float2(0.f, 0.f);
        for (int j0 = 0; j0 < nbb; j0 += G) {
            float2 v[G][ROWS];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    const int i = lane + 32 * k, j = j0 + g;
                    v[g][k] = (i < na && j < nbb) ? N[(int64_t)j * na + i] : make_float2(0.f, 0.f);
                }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 + g;            // warp-uniform; lanes past nbb hold zeros
                const int m = j >> 5, src_lane = j & 31;
                float2 x = make_float2(0.f, 0.f);
#pragma unroll
                for (int mm = 0; mm < XR; ++mm)
                    if (mm == m) x = xs[mm];
                const float xr = __shfl_sync(0xffffffffu, x.x, src_lane);
                const float xi = __shfl_sync(0xffffffffu, x.y, src_lane);
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    p[k].x = fmaf(v[g][k].x, xr, fmaf(-v[g][k].y, xi, p[k].x));
                    p[k].y = fmaf(v[g][k].x, xi, fmaf(v[g][k].y, xr, p[k].y));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < ROWS; ++k) {
            acc[k].x += p[k].x;
            acc[k].y += p[k].y;
        }
    }
#pragma unroll
    for (int k = 0; k < ROWS; ++k) part[warp][lane + 32 * k] = acc[k];
    __syncthreads();
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        double sr = 0, si = 0;
#pragma unroll
        for (int w = 0; w < kNearWarps; ++w) {
            sr += part[w][i].x;
            si += part[w][i].y;
        }
        const float2 x = cr[off[a] + i];
        const double alpha = alpha_box[a];
        y[(int64_t)r * n + off[a] + i] = make_float2((float)(sr + alpha * x.x), (float)(si + alpha * x.y));
    }
}

}  // namespace

ie_status launch_near(const ie_plan p, const float2 *c, float2 *y, int nrhs, cudaStream_t st, const int *gate) {
    int maxnb = 0;
    for (int v : p->nb) maxnb = v > maxnb ? v : maxnb;
    const dim3 grid(p->nbox, nrhs);
    if (maxnb <= 32)
        near_kernel<1><<<grid, kNearWarps * 32, 0, st>>>(p->d_nb, p->d_off, p->n, p->d_near_start, p->d_near_src,
                                                         p->d_near_boff, p->d_Nblk, p->d_alpha_box, c, y, gate);
    else if (maxnb <= 64)
        near_kernel<2><<<grid, kNearWarps * 32, 0, st>>>(p->d_nb, p->d_off, p->n, p->d_near_start, p->d_near_src,
                                                         p->d_near_boff, p->d_Nblk, p->d_alpha_box, c, y, gate);
    else
        near_kernel<6><<<grid, kNearWarps * 32, 0, st>>>(p->d_nb, p->d_off, p->n, p->d_near_start, p->d_near_src,
                                                         p->d_near_boff, p->d_Nblk, p->d_alpha_box, c, y, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie
