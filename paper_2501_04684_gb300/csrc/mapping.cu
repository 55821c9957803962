// K2 / K4: mapping to uniform basis functions (Alg. 1, x_b = P_b^T c_b) and inverse
// mapping (Alg. 3, r_b = P_b y_b); the 16-bit hi/lo split of the mapped vectors for
// the tensor-core translation; the plane-wave excitation (§5) tested with P.
//
// Layouts: c, r: [rhs][n] complex64 (box b's coefficients at off[b] .. off[b+1]);
// P: [n][192] complex64 (row off[b]+i is basis function i of box b);
// X, Y: [rhs][nbox][192] complex64.  All HBM-bound: one CTA per (box, rhs).
#include "ie_internal.h"

namespace ie {
namespace {

// x[u] = sum_i P[i][u] c[i]: 192 threads, one per dipole unknown u.  FP32 products
// in runs of 16, runs summed in FP64.
__global__ void aggregate_kernel(const float2 *__restrict__ P, const int32_t *__restrict__ nb,
                                 const int64_t *__restrict__ off, int64_t n, int nbox,
                                 const float2 *__restrict__ c, float2 *__restrict__ X, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ float2 cs[kNU];
    int b = blockIdx.x, r = blockIdx.y, u = threadIdx.x;
    int nbb = nb[b];
    const float2 *cb = c + (int64_t)r * n + off[b];
    for (int i = u; i < nbb; i += blockDim.x) cs[i] = cb[i];
    __syncthreads();
    const float2 *Pb = P + off[b] * kNU;
    double ar = 0, ai = 0;
    for (int i0 = 0; i0 < nbb; i0 += 16) {
        float pr = 0.f, pi = 0.f;
        int i1 = min(nbb, i0 + 16);
        for (int i = i0; i < i1; ++i) {
            float2 p = Pb[(int64_t)i * kNU + u];
            float2 cv = cs[i];
            pr = fmaf(p.x, cv.x, fmaf(-p.y, cv.y, pr));
            pi = fmaf(p.x, cv.y, fmaf(p.y, cv.x, pi));
        }
        ar += pr;
        ai += pi;
    }
    X[((int64_t)r * nbox + b) * kNU + u] = make_float2((float)ar, (float)ai);
}

__global__ void copy_kernel(const float4 *__restrict__ a, float4 *__restrict__ b, int64_t n4,
                            const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n4) b[i] = a[i];
}

// 16-bit hi/lo split of X for the tensor-core path.  Layout [hl][rhs][nbox][chunk][reim][32]:
// per column 384 values, K-chunk major (chunk = u / 32), re and im rows of a chunk adjacent.
// FP16: the column is scaled by 2^-e so that max |x| < 2^14; e is stored.
// With a symmetry map, block z writes copy z of the signed-permuted input
// x^Q[u] = +-x[U_Q(u)] at Xtc + z * (2 planes); the scale is the same for every copy.
template <bool FP16>
__global__ void split_kernel(const float2 *__restrict__ X, int nbox, int nrhs, uint16_t *__restrict__ Xtc,
                             int32_t *__restrict__ Xexp, float *__restrict__ Xinf, const uint16_t *__restrict__ symmap,
                             const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    int b = blockIdx.x, r = blockIdx.y, u = threadIdx.x;
    const int sg = blockIdx.z;
    int64_t col = (int64_t)r * nbox + b;
    float2 x;
    if (symmap) {
        const uint16_t e = symmap[sg * kNU + u];
        x = X[col * kNU + (e & 0xFF)];
        if (e & 0x100) x = make_float2(-x.x, -x.y);
    } else {
        x = X[col * kNU + u];
    }
    const bool write_exp = sg == 0;
    float scale = 1.f;
    if (FP16) {
        __shared__ float red[8], red2[8];
        __shared__ float s_scale;
        float m = fmaxf(fabsf(x.x), fabsf(x.y));
        float m2 = x.x * x.x + x.y * x.y;     // for max_u |x_u| (the networks' input norm)
        for (int o = 16; o; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if ((u & 31) == 0) red[u >> 5] = m, red2[u >> 5] = m2;
        __syncthreads();
        if (u == 0) {
            float mm = 0.f, mm2 = 0.f;
            for (int w = 0; w < kNU / 32; ++w) mm = fmaxf(mm, red[w]), mm2 = fmaxf(mm2, red2[w]);
            if (write_exp && Xinf) Xinf[col] = sqrtf(mm2);
            int e = 0;
            if (mm > 0.f) {
                frexpf(mm, &e);
                e -= 14;
            }
            if (write_exp) Xexp[col] = e;
            s_scale = ldexpf(1.f, -e);
        }
        __syncthreads();
        scale = s_scale;
    } else if (u == 0 && write_exp) {
        Xexp[col] = 0;
    }
    int64_t plane = (int64_t)nrhs * nbox * 2 * kNU;
    // K-chunk-major within the column: [chunk of 32][re 32, im 32], so one K-chunk of a
    // column (both rows) is 128 contiguous bytes for the tensor-core gathers
    uint16_t *cre = Xtc + 2 * plane * sg + (col * 2) * kNU + (u >> 5) * 64 + (u & 31);
    float v[2] = {x.x * scale, x.y * scale};
    uint16_t hi[2], lo[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (FP16) {
            __half h = __float2half_rn(v[t]);
            hi[t] = __half_as_ushort(h);
            lo[t] = __half_as_ushort(__float2half_rn(v[t] - __half2float(h)));
        } else {
            __nv_bfloat16 h = __float2bfloat16_rn(v[t]);
            hi[t] = __bfloat16_as_ushort(h);
            lo[t] = __bfloat16_as_ushort(__float2bfloat16_rn(v[t] - __bfloat162float(h)));
        }
    }
    cre[0] = hi[0];
    cre[32] = hi[1];
    cre[plane] = lo[0];
    cre[plane + 32] = lo[1];
}

// r[i] (+)= sum_u P[i][u] y[u], y = sum over slabs (FP64).  One warp per basis row,
// lanes over u; FP32 products and tree reduction.
__global__ void disaggregate_kernel(const float2 *__restrict__ P, const int32_t *__restrict__ nb,
                                    const int64_t *__restrict__ off, int64_t n, int nbox,
                                    const float2 *__restrict__ Yslab, int nslab, size_t slab_stride,
                                    float2 *__restrict__ out, int accumulate, int identity,
                                    const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ float2 ys[kNU];
    int b = blockIdx.x, r = blockIdx.y;
    int64_t col = (int64_t)r * nbox + b;
    for (int u = threadIdx.x; u < kNU; u += blockDim.x) {
        double sr = 0, si = 0;
        for (int s = 0; s < nslab; ++s) {
            float2 v = Yslab[s * slab_stride + col * kNU + u];
            sr += v.x;
            si += v.y;
        }
        ys[u] = make_float2((float)sr, (float)si);
    }
    __syncthreads();
    float2 *ob = out + (int64_t)r * n + off[b];
    int nbb = nb[b];
    if (identity) {
        for (int u = threadIdx.x; u < kNU; u += blockDim.x) {
            float2 v = ys[u];
            if (accumulate) {
                float2 o = ob[u];
                v.x += o.x;
                v.y += o.y;
            }
            ob[u] = v;
        }
        return;
    }
    const float2 *Pb = P + off[b] * kNU;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nbb; i += nw) {
        float pr = 0.f, pi = 0.f;
        const float2 *row = Pb + (int64_t)i * kNU;
#pragma unroll
        for (int t = 0; t < kNU / 32; ++t) {
            float2 p = row[lane + 32 * t];
            float2 y = ys[lane + 32 * t];
            pr = fmaf(p.x, y.x, fmaf(-p.y, y.y, pr));
            pi = fmaf(p.x, y.y, fmaf(p.y, y.x, pi));
        }
        for (int o = 16; o; o >>= 1) {
            pr += __shfl_xor_sync(0xffffffffu, pr, o);
            pi += __shfl_xor_sync(0xffffffffu, pi, o);
        }
        if (lane == 0) {
            if (accumulate) {
                float2 o = ob[i];
                pr += o.x;
                pi += o.y;
            }
            ob[i] = make_float2(pr, pi);
        }
    }
}

__global__ void zero_kernel(float4 *__restrict__ p, int64_t n4, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n4; i += stride) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// nslab regions of n4 float4 each, stride4 float4 apart (blockIdx.y = region).
__global__ void zero_slabs_kernel(float4 *__restrict__ p, int64_t n4, int64_t stride4, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    float4 *q = p + (int64_t)blockIdx.y * stride4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void sum_slabs_kernel(const float2 *__restrict__ Yslab, int nslab, size_t slab_stride, int64_t count,
                                 float2 *__restrict__ Y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double sr = 0, si = 0;
    for (int s = 0; s < nslab; ++s) {
        float2 v = Yslab[s * slab_stride + i];
        sr += v.x;
        si += v.y;
    }
    Y[i] = make_float2((float)sr, (float)si);
}

// Plane wave at the dipole sites, e[3s+a] = pol[a] exp(-j k khat . r_s) (FP64 phase),
// then v_b = P_b e_b as in disaggregate_kernel.
__global__ void plane_wave_kernel(double k, double a, int G, const int32_t *__restrict__ ijk,
                                  const float2 *__restrict__ P, const int32_t *__restrict__ nb,
                                  const int64_t *__restrict__ off, int64_t n,
                                  const double *__restrict__ khat, const double *__restrict__ pol,
                                  const int32_t *__restrict__ box_group, int nrhs,
                                  float2 *__restrict__ v, int identity) {
    __shared__ float2 es[kNU];
    int b = blockIdx.x, r = blockIdx.y;
    const int w = box_group[b] * nrhs + r;        // incidence of this scatterer's column r
    double h = a / kLattice;
    for (int s = threadIdx.x; s < kSites; s += blockDim.x) {
        int ii[3] = {s & 3, (s >> 2) & 3, s >> 4};
        double ph = 0;
        for (int c = 0; c < 3; ++c) {
            double pos = a * ((double)ijk[3 * b + c] + 0.5 - 0.5 * G) + h * (ii[c] + 0.5) - 0.5 * a;
            ph += khat[3 * w + c] * pos;
        }
        double sn, cs;
        sincos(-k * ph, &sn, &cs);
        for (int c = 0; c < 3; ++c) es[3 * s + c] = make_float2((float)(pol[3 * w + c] * cs), (float)(pol[3 * w + c] * sn));
    }
    __syncthreads();
    float2 *vb = v + (int64_t)r * n + off[b];
    if (identity) {
        for (int u = threadIdx.x; u < kNU; u += blockDim.x) vb[u] = es[u];
        return;
    }
    const float2 *Pb = P + off[b] * kNU;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < nb[b]; i += nw) {
        double pr = 0, pi = 0;
        const float2 *row = Pb + (int64_t)i * kNU;
        for (int t = 0; t < kNU / 32; ++t) {
            float2 p = row[lane + 32 * t];
            float2 e = es[lane + 32 * t];
            pr += (double)p.x * e.x - (double)p.y * e.y;
            pi += (double)p.x * e.y + (double)p.y * e.x;
        }
        for (int o = 16; o; o >>= 1) {
            pr += __shfl_xor_sync(0xffffffffu, pr, o);
            pi += __shfl_xor_sync(0xffffffffu, pi, o);
        }
        if (lane == 0) vb[i] = make_float2((float)pr, (float)pi);
    }
}

}  // namespace

ie_status launch_aggregate(const ie_plan p, const float2 *c, float2 *X, int nrhs, cudaStream_t st, const int *gate) {
    if (p->identity) {
        // n == nbox * 192 and [rhs][n] == [rhs][nbox][192]
        int64_t n4 = (int64_t)nrhs * p->n / 2;
        copy_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4 *>(c),
                                                                  reinterpret_cast<float4 *>(X), n4, gate);
    } else {
        aggregate_kernel<<<dim3(p->nbox, nrhs), kNU, 0, st>>>(p->d_P, p->d_nb, p->d_off, p->n, p->nbox, c, X, gate);
    }
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_split_tc(const ie_plan p, const float2 *X, int nrhs, bool fp16, cudaStream_t st, const int *gate) {
    const dim3 grid(p->nbox, nrhs, p->sym ? kSym : 1);
    const uint16_t *map = p->sym ? p->d_symmap : nullptr;
    if (fp16)
        split_kernel<true><<<grid, kNU, 0, st>>>(X, p->nbox, nrhs, p->d_Xtc, p->d_Xexp, p->d_Xinf, map, gate);
    else
        split_kernel<false><<<grid, kNU, 0, st>>>(X, p->nbox, nrhs, p->d_Xtc, p->d_Xexp, nullptr, map, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

// The 48 signed-permuted copies x^Q[u] = +-x[U_Q(u)] of the FP32 translation input,
// layout [Q][rhs][nbox][192].
__global__ void permute_sym_kernel(const float2 *__restrict__ X, int nbox, int nrhs, const uint16_t *__restrict__ symmap,
                                   float2 *__restrict__ Xsym, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int b = blockIdx.x, r = blockIdx.y, sg = blockIdx.z, u = threadIdx.x;
    const int64_t col = (int64_t)r * nbox + b;
    const uint16_t e = symmap[sg * kNU + u];
    float2 x = X[col * kNU + (e & 0xFF)];
    if (e & 0x100) x = make_float2(-x.x, -x.y);
    Xsym[((int64_t)sg * nrhs * nbox + col) * kNU + u] = x;
}

ie_status launch_permute_sym(const ie_plan p, const float2 *X, int nrhs, cudaStream_t st, const int *gate) {
    permute_sym_kernel<<<dim3(p->nbox, nrhs, kSym), kNU, 0, st>>>(X, p->nbox, nrhs, p->d_symmap, p->d_Xsym, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_disaggregate(const ie_plan p, const float2 *Yslab, int nslab, size_t stride, float2 *r, int nrhs,
                              bool accumulate, cudaStream_t st, const int *gate) {
    disaggregate_kernel<<<dim3(p->nbox, nrhs), 256, 0, st>>>(p->d_P, p->d_nb, p->d_off, p->n, p->nbox, Yslab, nslab,
                                                             stride, r, accumulate ? 1 : 0, p->identity ? 1 : 0, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_zero(void *ptr, size_t bytes, cudaStream_t st, const int *gate) {
    if (bytes == 0) return IE_OK;
    if (bytes % 16) {
        set_error("launch_zero: size %zu not a multiple of 16", bytes);
        return IE_ERR_INVALID;
    }
    int64_t n4 = (int64_t)(bytes / 16);
    int64_t grid = (n4 + 255) / 256;
    if (grid > 4096) grid = 4096;
    zero_kernel<<<(unsigned)grid, 256, 0, st>>>(reinterpret_cast<float4 *>(ptr), n4, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_zero_slabs(float2 *base, int nslab, size_t stride, size_t count, cudaStream_t st, const int *gate) {
    if (count == 0 || nslab == 0) return IE_OK;
    if ((count * sizeof(float2)) % 16 || (stride * sizeof(float2)) % 16) {
        set_error("launch_zero_slabs: sizes not multiples of 16 bytes");
        return IE_ERR_INVALID;
    }
    const int64_t n4 = (int64_t)(count * sizeof(float2) / 16);
    int64_t gx = (n4 + 255) / 256;
    if (gx > 1024) gx = 1024;
    zero_slabs_kernel<<<dim3((unsigned)gx, (unsigned)nslab), 256, 0, st>>>(reinterpret_cast<float4 *>(base), n4,
                                                                          (int64_t)(stride * sizeof(float2) / 16),
                                                                          gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_sum_slabs(const ie_plan p, const float2 *Yslab, int nslab, size_t stride, float2 *Y, int nrhs,
                           cudaStream_t st) {
    int64_t count = (int64_t)nrhs * p->nbox * kNU;
    sum_slabs_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(Yslab, nslab, stride, count, Y);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_plane_wave(const ie_plan p, const double *d_khat, const double *d_pol, int nrhs, float2 *v,
                            cudaStream_t st) {
    plane_wave_kernel<<<dim3(p->nbox, nrhs), 256, 0, st>>>(p->k, p->a, p->G, p->d_ijk, p->d_P, p->d_nb, p->d_off,
                                                           p->n, d_khat, d_pol, p->d_box_group, nrhs, v,
                                                           p->identity ? 1 : 0);
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie
