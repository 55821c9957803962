// K1: coupling blocks G_d (eq. 13) from the free-space dyadic Green's function
// (eq. 5, eq. 6), evaluated in FP64 on the device and stored for the translation
// kernels; and the stored near-zone blocks P_a G_{a-b} P_b^T (eq. 2).
//
// Geometry: dipole site s = ix + 4 iy + 16 iz of a box sits at the cell-centred
// offset h*((ix,iy,iz) + 1/2) - a/2 with h = a/4.  For test box = basis box + d the
// separation of test site l and basis site q is R = h (4 d + l - q), a multiple of
// the lattice spacing, so G_d depends only on d.
#include "ie_internal.h"

namespace ie {
namespace {

// One thread per (displacement, test site l, basis site q): the 3x3 block of G_d.
// row_major = false: layout [d][k][m] (k = basis unknown, m = test unknown), the
// FP32 translation kernel's A^T operand; true: [d][m][k].
__global__ void coupling_fp32_kernel(double k, double eta, double h, const int32_t *__restrict__ disp, int64_t nd,
                                     float2 *__restrict__ out, int row_major) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * kSites * kSites) return;
    int64_t di = t / (kSites * kSites);
    int rem = (int)(t % (kSites * kSites));
    int q = rem / kSites;          // basis site (slower)
    int l = rem % kSites;          // test site (faster: coalesced m)
    int dx = disp[3 * di], dy = disp[3 * di + 1], dz = disp[3 * di + 2];
    int mx = 4 * dx + (l & 3) - (q & 3);
    int my = 4 * dy + ((l >> 2) & 3) - ((q >> 2) & 3);
    int mz = 4 * dz + (l >> 4) - (q >> 4);
    double2 D[9];
    bool coincident = (mx == 0 && my == 0 && mz == 0);
    if (!coincident) dyad_fp64(k, eta, h * mx, h * my, h * mz, D);
    float2 *blk = out + di * (int64_t)kNU * kNU;
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            float2 v = coincident ? make_float2(0.f, 0.f)
                                  : make_float2((float)D[3 * al + be].x, (float)D[3 * al + be].y);
            int m = 3 * l + al, kk = 3 * q + be;
            if (row_major)
                blk[(int64_t)m * kNU + kk] = v;
            else
                blk[(int64_t)kk * kNU + m] = v;
        }
}

// Tensor-core images of every far coupling block, from the FP32 store.
// Real embedding of y = G x with G = Gr + j Gi, split operands x = [xr; xi]:
// real row 2m holds Gr[m][:], row 2m+1 holds Gi[m][:]; the GEMM against the
// columns xr and xi gives Gr xr, Gr xi, Gi xr, Gi xi, combined in the epilogue.
// Image (mb, kc, hl): rows 128 mb .. +127, source unknowns 32 kc .. +31, hi or lo
// 16-bit part, in the 64-byte-swizzled K-major layout of tcgen05.mma: row r is 64 B,
// its 16-byte chunk c lands at chunk c ^ ((r / 2) mod 4).  One CTA per displacement.
// fp16: scaled by 2^-e (e stored) so that |entries| <= 2^14.
template <bool FP16>
__global__ void coupling_tc_kernel(const float2 *__restrict__ Cs, int64_t nd, uint16_t *__restrict__ out,
                                   int32_t *__restrict__ exps) {
    int64_t di = blockIdx.x;
    if (di >= nd) return;
    const float2 *blk = Cs + di * (int64_t)kNU * kNU;   // [k][m]
    __shared__ float red[32];
    __shared__ float s_scale;
    float scale = 1.f;
    if (FP16) {
        float mx = 0.f;
        for (int i = threadIdx.x; i < kNU * kNU; i += blockDim.x) {
            float2 v = blk[i];
            mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
            int e = 0;
            if (m > 0.f) {
                frexpf(m, &e);     // m = f 2^e, f in [0.5, 1)
                e -= 14;           // m 2^-e < 2^14
            }
            exps[di] = e;
            s_scale = ldexpf(1.f, -e);
        }
        __syncthreads();
        scale = s_scale;
    }
    uint16_t *img0 = out + di * (int64_t)kTcDispElems;
    // 36 images x 128 rows x 4 chunks of 16 bytes
    for (int w = threadIdx.x; w < kTcImagesPerDisp * 128 * 4; w += blockDim.x) {
        int c = w & 3;
        int r = (w >> 2) & 127;
        int img = w >> 9;               // (mb * 6 + kc) * 2 + hl
        int hl = img & 1;
        int kc = (img >> 1) % kTcKChunks;
        int mb = (img >> 1) / kTcKChunks;
        int R = 128 * mb + r;
        int m = R >> 1, part = R & 1;
        uint16_t vals[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            int kk = kTcK * kc + 8 * c + e;
            float2 g = blk[(int64_t)kk * kNU + m];
            float x = (part ? g.y : g.x) * scale;
            if (FP16) {
                __half hi = __float2half_rn(x);
                __half lo = __float2half_rn(x - __half2float(hi));
                vals[e] = __half_as_ushort(hl ? lo : hi);
            } else {
                __nv_bfloat16 hi = __float2bfloat16_rn(x);
                __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                vals[e] = __bfloat16_as_ushort(hl ? lo : hi);
            }
        }
        uint4 pk;
        pk.x = vals[0] | ((uint32_t)vals[1] << 16);
        pk.y = vals[2] | ((uint32_t)vals[3] << 16);
        pk.z = vals[4] | ((uint32_t)vals[5] << 16);
        pk.w = vals[6] | ((uint32_t)vals[7] << 16);
        uint4 *dst = reinterpret_cast<uint4 *>(img0 + (int64_t)img * kTcImageElems + r * kTcK +
                                               8 * (c ^ ((r >> 1) & 3)));
        *dst = pk;
    }
}

// Near blocks: N_ab = P_a G_{a-b} P_b^T (test box a, basis box b), nb_a x nb_b,
// column-major.  One CTA per stored pair; basis columns in chunks of 32.
// Partial sums over 32 terms in FP32, chunk sums in FP64.
constexpr int kNearJ = 32;

__global__ void near_blocks_kernel(const float2 *__restrict__ Cnear,     // [27][k][m], index by e
                                   const int32_t *__restrict__ ijk, const int32_t *__restrict__ nb,
                                   const int64_t *__restrict__ off, const float2 *__restrict__ P,
                                   const int32_t *__restrict__ pair_a, const int32_t *__restrict__ pair_b,
                                   const int64_t *__restrict__ boff, int64_t npairs, float2 *__restrict__ Nblk) {
    extern __shared__ float2 sm[];
    float2 *Pb = sm;                    // [kNearJ][192]
    float2 *W = sm + kNearJ * kNU;      // [192][kNearJ]
    int64_t pi = blockIdx.x;
    if (pi >= npairs) return;
    int a = pair_a[pi], b = pair_b[pi];
    int ex = ijk[3 * a] - ijk[3 * b], ey = ijk[3 * a + 1] - ijk[3 * b + 1], ez = ijk[3 * a + 2] - ijk[3 * b + 2];
    int e = (ex + 1) * 9 + (ey + 1) * 3 + (ez + 1);
    const float2 *C = Cnear + (int64_t)e * kNU * kNU;   // [k][m]
    int na = nb[a], nbb = nb[b];
    const float2 *Pa = P + off[a] * kNU;
    const float2 *Pbg = P + off[b] * kNU;
    float2 *N = Nblk + boff[pi];
    for (int j0 = 0; j0 < nbb; j0 += kNearJ) {
        int nj = min(kNearJ, nbb - j0);
        __syncthreads();
        for (int i = threadIdx.x; i < nj * kNU; i += blockDim.x) Pb[i] = Pbg[(int64_t)j0 * kNU + i];
        __syncthreads();
        // W[m][jj] = sum_k C[m][k] Pb[jj][k]
        for (int o = threadIdx.x; o < kNU * nj; o += blockDim.x) {
            int m = o % kNU, jj = o / kNU;
            double wr = 0, wi = 0;
            for (int k0 = 0; k0 < kNU; k0 += 32) {
                float pr = 0.f, pim = 0.f;
                for (int kk = k0; kk < k0 + 32; ++kk) {
                    float2 g = C[(int64_t)kk * kNU + m];
                    float2 pv = Pb[jj * kNU + kk];
                    pr = fmaf(g.x, pv.x, fmaf(-g.y, pv.y, pr));
                    pim = fmaf(g.x, pv.y, fmaf(g.y, pv.x, pim));
                }
                wr += pr;
                wi += pim;
            }
            W[m * kNearJ + jj] = make_float2((float)wr, (float)wi);
        }
        __syncthreads();
        // N[i][j0+jj] = sum_m Pa[i][m] W[m][jj]
        for (int o = threadIdx.x; o < na * nj; o += blockDim.x) {
            int i = o % na, jj = o / na;
            double nr = 0, ni = 0;
            for (int m0 = 0; m0 < kNU; m0 += 32) {
                float pr = 0.f, pim = 0.f;
                for (int m = m0; m < m0 + 32; ++m) {
                    float2 pa = Pa[(int64_t)i * kNU + m];
                    float2 w = W[m * kNearJ + jj];
                    pr = fmaf(pa.x, w.x, fmaf(-pa.y, w.y, pr));
                    pim = fmaf(pa.x, w.y, fmaf(pa.y, w.x, pim));
                }
                nr += pr;
                ni += pim;
            }
            N[(int64_t)(j0 + jj) * na + i] = make_float2((float)nr, (float)ni);
        }
    }
}

// Identity mapping: the near block is G_e itself (192 x 192, column-major = [k][m]).
__global__ void near_blocks_identity_kernel(const float2 *__restrict__ Cnear, const int32_t *__restrict__ ijk,
                                            const int32_t *__restrict__ pair_a, const int32_t *__restrict__ pair_b,
                                            const int64_t *__restrict__ boff, int64_t npairs,
                                            float2 *__restrict__ Nblk) {
    int64_t pi = blockIdx.x;
    if (pi >= npairs) return;
    int a = pair_a[pi], b = pair_b[pi];
    int e = (ijk[3 * a] - ijk[3 * b] + 1) * 9 + (ijk[3 * a + 1] - ijk[3 * b + 1] + 1) * 3 +
            (ijk[3 * a + 2] - ijk[3 * b + 2] + 1);
    const float4 *src = reinterpret_cast<const float4 *>(Cnear + (int64_t)e * kNU * kNU);
    float4 *dst = reinterpret_cast<float4 *>(Nblk + boff[pi]);
    for (int i = threadIdx.x; i < kNU * kNU / 2; i += blockDim.x) dst[i] = src[i];
}

}  // namespace

ie_status launch_coupling_fp32(double k, double eta, double a, const int32_t *d_disp, int64_t nd, float2 *out,
                               bool row_major, cudaStream_t st) {
    if (nd <= 0) return IE_OK;
    int64_t threads = nd * kSites * kSites;
    int bs = 256;
    int64_t grid = (threads + bs - 1) / bs;
    coupling_fp32_kernel<<<(unsigned)grid, bs, 0, st>>>(k, eta, a / kLattice, d_disp, nd, out, row_major ? 1 : 0);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_coupling_simt(const ie_plan p, const int32_t *d_disp, int64_t nd, float2 *out, bool row_major,
                               cudaStream_t st) {
    return launch_coupling_fp32(p->k, p->eta, p->a, d_disp, nd, out, row_major, st);
}

ie_status launch_coupling_tc(const float2 *Cs, int64_t nd, uint16_t *out, int32_t *exps, bool fp16, cudaStream_t st) {
    if (nd <= 0) return IE_OK;
    if (fp16)
        coupling_tc_kernel<true><<<(unsigned)nd, 256, 0, st>>>(Cs, nd, out, exps);
    else
        coupling_tc_kernel<false><<<(unsigned)nd, 256, 0, st>>>(Cs, nd, out, exps);
    IE_CK_LAUNCH();
    return IE_OK;
}

ie_status launch_near_blocks(ie_plan p, cudaStream_t st) {
    if (p->n_near_pairs == 0) return IE_OK;
    // the 27 near displacements, e = (ex+1)*9 + (ey+1)*3 + (ez+1)
    std::vector<int32_t> ds(27 * 3);
    for (int e = 0; e < 27; ++e) {
        ds[3 * e] = e / 9 - 1;
        ds[3 * e + 1] = (e / 3) % 3 - 1;
        ds[3 * e + 2] = e % 3 - 1;
    }
    int32_t *d_ds = nullptr;
    float2 *d_C = nullptr;
    int32_t *d_pa = nullptr;
    IE_CK(cudaMallocAsync(&d_ds, ds.size() * sizeof(int32_t), st));
    IE_CK(cudaMallocAsync(&d_C, (size_t)27 * kNU * kNU * sizeof(float2), st));
    IE_CK(cudaMallocAsync(&d_pa, (size_t)p->n_near_pairs * sizeof(int32_t), st));
    IE_CK(cudaMemcpyAsync(d_ds, ds.data(), ds.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    IE_TRY(launch_coupling_simt(p, d_ds, 27, d_C, false, st));
    // target box of every stored pair
    std::vector<int32_t> start(p->nbox + 1);
    IE_CK(cudaMemcpyAsync(start.data(), p->d_near_start, start.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    IE_CK(cudaStreamSynchronize(st));
    std::vector<int32_t> pa(p->n_near_pairs);
    for (int a = 0; a < p->nbox; ++a)
        for (int i = start[a]; i < start[a + 1]; ++i) pa[i] = a;
    IE_CK(cudaMemcpyAsync(d_pa, pa.data(), pa.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (p->identity) {
        near_blocks_identity_kernel<<<(unsigned)p->n_near_pairs, 256, 0, st>>>(d_C, p->d_ijk, d_pa, p->d_near_src,
                                                                               p->d_near_boff, p->n_near_pairs,
                                                                               p->d_Nblk);
    } else {
        size_t smem = (size_t)2 * kNearJ * kNU * sizeof(float2);
        IE_CK(cudaFuncSetAttribute(near_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        near_blocks_kernel<<<(unsigned)p->n_near_pairs, 256, smem, st>>>(d_C, p->d_ijk, p->d_nb, p->d_off, p->d_P,
                                                                         d_pa, p->d_near_src, p->d_near_boff,
                                                                         p->n_near_pairs, p->d_Nblk);
    }
    IE_CK_LAUNCH();
    IE_CK(cudaFreeAsync(d_ds, st));
    IE_CK(cudaFreeAsync(d_C, st));
    IE_CK(cudaFreeAsync(d_pa, st));
    return IE_OK;
}

}  // namespace ie
