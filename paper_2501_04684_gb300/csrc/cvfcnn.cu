// CVFCNN translation surrogate of §3 (IE_PREC_CVFCNN).
//
// Each stored block G_c gets a complex network 192 -> H -> 192: the input x is scaled
// by s = ||x||_inf, the hidden layer is z = W1 x / s + b1 with the Cartesian ReLU
// max(Re z, 0) + j max(Im z, 0), the output s (W2 h + b2) replaces G_c x in Alg. 2.
//
// Weights (plan creation), once per canonical displacement c = sorted |d|: the block is
// regenerated in FP64, its SVD G = U S V^H is computed by one-sided Jacobi (one CTA per
// block, Hestenes rotations on the columns, round-robin pairing), and the network is set
// to its linear regime on the unit
// l-inf ball: W1 = V_H^H, W2 = U_H S_H, b1_h = beta_h (1 + j) with beta_h the l1 norm
// of row h of W1 (so Re and Im of W1 x/s + b1 stay >= 0), b2 = -W2 b1.  The output is
// then U_H S_H V_H^H x: the best rank-H approximation of G_c (Eckart-Young), whose
// relative error on inputs with independent entries is the SVD's Frobenius tail.  With
// the symmetric store the canonical networks are the stored ones; with the full store
// each displacement d = Q c gets the canonical network turned into its frame.
//
// Inference: one CTA per work item of the FP32 path (a displacement group's run of at
// most 64 columns): the column scales, GEMM 1 (64 x 64 x 192, 4 x 4 complex register
// tile of two row pairs and two column pairs, 16-byte shared loads) with the bias and the
// ReLU in its epilogue into shared memory, GEMM 2 (192 x 64 x 64), the bias, the
// rescale and the scatter-add into the far-field slabs (with the symmetry maps when
// the store is symmetry-compressed).  1.92x fewer multiply-adds than G_c x at H = 50.
#include "ie_internal.h"

#include <algorithm>
#include <vector>

namespace ie {
namespace {

constexpr int kJacobiThreads = 1024;
constexpr int kMaxSweeps = 16;             // the rank-50 tails are then within 1e-6 of the SVD's
constexpr double kJacobiTol = 1e-13;       // relative orthogonality of a column pair
constexpr double kJacobiAbs = 1e-14;       // noise floor, in units of ||G||_F (|p| + |q|)
constexpr int kTileN = 64;
constexpr int kKC = 16;
constexpr int kThreads = 256;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---------------------------------------------------------------- weights
// G_d in FP64, column-major: A[blk][k][m] = G_d[m][k] (k basis unknown, m test unknown).
// One thread per (block, test site l, basis site q).
__global__ void blocks_fp64_kernel(double k, double eta, double h, const int32_t *__restrict__ disp, int64_t nd,
                                   double2 *__restrict__ A) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * kSites * kSites) return;
    int64_t di = t / (kSites * kSites);
    int rem = (int)(t % (kSites * kSites));
    int q = rem / kSites;
    int l = rem % kSites;
    int dx = disp[3 * di], dy = disp[3 * di + 1], dz = disp[3 * di + 2];
    int mx = 4 * dx + (l & 3) - (q & 3);
    int my = 4 * dy + ((l >> 2) & 3) - ((q >> 2) & 3);
    int mz = 4 * dz + (l >> 4) - (q >> 4);
    double2 D[9];
    bool coincident = (mx == 0 && my == 0 && mz == 0);
    if (!coincident) dyad_fp64(k, eta, h * mx, h * my, h * mz, D);
    double2 *blk = A + di * (int64_t)kNU * kNU;
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be)
            blk[(int64_t)(3 * q + be) * kNU + 3 * l + al] = coincident ? make_double2(0.0, 0.0) : D[3 * al + be];
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One-sided Jacobi SVD of one block per CTA: rotate column pairs of A (and V, from I)
// until every pair is orthogonal, |p^H q| <= max(kJacobiTol |p| |q|,
// kJacobiAbs ||G||_F (|p| + |q|)), or kMaxSweeps sweeps have run; then A = U S and
// G V = U S.  The second bound is the rounding noise that rotations leave in p^H q
// (entries carry errors of about eps sqrt(192) ||G||_F): pairs of columns far below the
// largest could never meet the relative test.  Columns whose singular values cluster
// near the noise converge slowly and may use up the sweeps; truncating A V keeps an exact
// record of the error whether or not they did: G - B_H V_H^H = B_drop V_drop^H.
// FP64 is the cost here (GB300 runs it at a small fraction of its FP32 rate): one
// sweep is ~25 MFLOP per block, so blocks are fitted once per canonical displacement.  For the
// pair (p, q): g = p^H q = |g| e^{i phi}; with q~ = q e^{-i phi} the Gram matrix is real,
// zeta = (|q|^2 - |p|^2) / (2 |g|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t, and p <- c p - s q~, q <- s p + c q~.  Rounds pair
// the 192 columns by the circle method (191 rounds of 96 disjoint pairs per sweep).
__global__ void __launch_bounds__(kJacobiThreads) jacobi_svd_kernel(double2 *__restrict__ A, double2 *__restrict__ V,
                                                                   int *__restrict__ sweeps_out) {
    double2 *a = A + (size_t)blockIdx.x * kNU * kNU;
    double2 *v = V + (size_t)blockIdx.x * kNU * kNU;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    __shared__ int s_rot;
    __shared__ double s_red[32];
    double fro = 0.0;
    for (int i = tid; i < kNU * kNU; i += blockDim.x) {
        v[i] = make_double2((i / kNU) == (i % kNU) ? 1.0 : 0.0, 0.0);
        fro += a[i].x * a[i].x + a[i].y * a[i].y;
    }
    fro = warp_sum(fro);
    if (lane == 0) s_red[warp] = fro;
    __syncthreads();
    fro = 0.0;
    for (int w = 0; w < nwarp; ++w) fro += s_red[w];
    const double noise = kJacobiAbs * sqrt(fro);
    int sweeps = 0;
    for (int sw = 0; sw < kMaxSweeps; ++sw) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < kNU - 1; ++r) {
            for (int kk = warp; kk < kNU / 2; kk += nwarp) {
                int p, q;
                if (kk == 0) {
                    p = r;
                    q = kNU - 1;
                } else {
                    p = (r + kk) % (kNU - 1);
                    q = (r - kk + (kNU - 1)) % (kNU - 1);
                }
                double2 *cp = a + (size_t)p * kNU, *cq = a + (size_t)q * kNU;
                double app = 0.0, aqq = 0.0, gr = 0.0, gi = 0.0;
                for (int i = lane; i < kNU; i += 32) {
                    const double2 x = cp[i], y = cq[i];
                    app += x.x * x.x + x.y * x.y;
                    aqq += y.x * y.x + y.y * y.y;
                    gr += x.x * y.x + x.y * y.y;
                    gi += x.x * y.y - x.y * y.x;
                }
                app = warp_sum(app);
                aqq = warp_sum(aqq);
                gr = warp_sum(gr);
                gi = warp_sum(gi);
                const double g = hypot(gr, gi);
                if (g > noise * (sqrt(app) + sqrt(aqq)) && g > kJacobiTol * sqrt(app * aqq)) {   // same in every lane
                    const double zeta = (aqq - app) / (2.0 * g);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    const double er = gr / g, ei = -gi / g;          // e^{-i phi}
                    double2 *vp = v + (size_t)p * kNU, *vq = v + (size_t)q * kNU;
                    for (int i = lane; i < kNU; i += 32) {
                        double2 x = cp[i], y = cq[i];
                        double yr = y.x * er - y.y * ei, yi = y.x * ei + y.y * er;
                        cp[i] = make_double2(c * x.x - s * yr, c * x.y - s * yi);
                        cq[i] = make_double2(s * x.x + c * yr, s * x.y + c * yi);
                        x = vp[i];
                        y = vq[i];
                        yr = y.x * er - y.y * ei;
                        yi = y.x * ei + y.y * er;
                        vp[i] = make_double2(c * x.x - s * yr, c * x.y - s * yi);
                        vq[i] = make_double2(s * x.x + c * yr, s * x.y + c * yi);
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            __syncthreads();
        }
        sweeps = sw + 1;
        const bool done = (s_rot == 0);
        __syncthreads();
        if (done) break;
    }
    if (tid == 0) sweeps_out[blockIdx.x] = sweeps;
}

// Weights of one block from its converged Jacobi state (see the file comment), in the
// inference layout; tail[blk] = sqrt(sum of the dropped S^2 / sum of all S^2).
__global__ void cvfcnn_weights_kernel(const double2 *__restrict__ A, const double2 *__restrict__ V, int H,
                                      float2 *__restrict__ W, double *__restrict__ tail) {
    const double2 *a = A + (size_t)blockIdx.x * kNU * kNU;
    const double2 *v = V + (size_t)blockIdx.x * kNU * kNU;
    float2 *w = W + (size_t)blockIdx.x * kCvBlockElems;
    __shared__ double s2[kNU];
    __shared__ int sel[kCvHp];
    __shared__ double beta[kCvHp];
    __shared__ double dropped[kNU];
    const int tid = threadIdx.x;
    for (int j = tid; j < kNU; j += blockDim.x) {
        double t = 0.0;
        for (int i = 0; i < kNU; ++i) {
            const double2 x = a[(size_t)j * kNU + i];
            t += x.x * x.x + x.y * x.y;
        }
        s2[j] = t;
    }
    __syncthreads();
    for (int j = tid; j < kNU; j += blockDim.x) {
        int rank = 0;
        for (int i = 0; i < kNU; ++i) rank += (s2[i] > s2[j]) || (s2[i] == s2[j] && i < j);
        if (rank < H) sel[rank] = j;
        dropped[j] = rank < H ? 0.0 : s2[j];
    }
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0, drop = 0.0;
        for (int j = 0; j < kNU; ++j) {
            tot += s2[j];
            drop += dropped[j];
        }
        tail[blockIdx.x] = tot > 0.0 ? sqrt(drop / tot) : 0.0;
    }
    // W1^T [u][h] = conj(V[u][j_h])
    for (int idx = tid; idx < kNU * kCvHp; idx += blockDim.x) {
        const int u = idx / kCvHp, h = idx % kCvHp;
        float2 val = make_float2(0.f, 0.f);
        if (h < H) {
            const double2 x = v[(size_t)sel[h] * kNU + u];
            val = make_float2((float)x.x, (float)-x.y);
        }
        w[kCvW1 + idx] = val;
    }
    // beta_h = sum_u |W1[h][u]| of the stored (rounded) weights, so that the bound holds
    // for what the inference kernel multiplies; a relative margin covers its FP32 sums
    for (int h = tid; h < kCvHp; h += blockDim.x) {
        double b = 0.0;
        if (h < H)
            for (int u = 0; u < kNU; ++u) {
                const double2 x = v[(size_t)sel[h] * kNU + u];
                b += hypot((double)(float)x.x, (double)(float)x.y);
            }
        beta[h] = h < H ? b * (1.0 + 1e-5) : 0.0;
        w[kCvB1 + h] = make_float2((float)beta[h], (float)beta[h]);
    }
    // W2^T [h][u] = (U S)[u][j_h] = column j_h of the rotated A
    for (int idx = tid; idx < kCvHp * kNU; idx += blockDim.x) {
        const int h = idx / kNU, u = idx % kNU;
        float2 val = make_float2(0.f, 0.f);
        if (h < H) {
            const double2 x = a[(size_t)sel[h] * kNU + u];
            val = make_float2((float)x.x, (float)x.y);
        }
        w[kCvW2 + idx] = val;
    }
    __syncthreads();
    // b2 = -W2 b1 from the stored values: the bias terms cancel as closely as FP32 allows
    for (int u = tid; u < kNU; u += blockDim.x) {
        double br = 0.0, bi = 0.0;
        for (int h = 0; h < H; ++h) {
            const float2 x = w[kCvW2 + (size_t)h * kNU + u];
            const double bh = (double)(float)beta[h];
            br += bh * ((double)x.x - (double)x.y);     // (x.x + j x.y)(1 + j) beta
            bi += bh * ((double)x.x + (double)x.y);
        }
        w[kCvB2 + u] = make_float2((float)-br, (float)-bi);
    }
}

// Weights of displacement d = Q c from those of its canonical c: net_d(x) = S net_c(S^T x)
// with S[U(u)][u] = +-1 (the symmetry map), i.e. W1_d[h][U(u)] = +-W1_c[h][u], b1_d = b1_c,
// W2_d[U(u)][h] = +-W2_c[u][h], b2_d[U(u)] = +-b2_c[u].  One CTA per displacement.
__global__ void cvfcnn_expand_kernel(const float2 *__restrict__ Wc, const int32_t *__restrict__ gcanon,
                                     const int32_t *__restrict__ gsigma, const uint16_t *__restrict__ map,
                                     float2 *__restrict__ Wd) {
    const float2 *src = Wc + (size_t)gcanon[blockIdx.x] * kCvBlockElems;
    float2 *out = Wd + (size_t)blockIdx.x * kCvBlockElems;
    const uint16_t *m = map + (size_t)gsigma[blockIdx.x] * kNU;
    for (int idx = threadIdx.x; idx < kNU * kCvHp; idx += blockDim.x) {
        const int u = idx / kCvHp, h = idx % kCvHp;
        const uint16_t e = m[u];
        const float sg = (e & 0x100) ? -1.f : 1.f;
        const float2 w1 = src[kCvW1 + idx];                          // W1^T[u][h]
        out[kCvW1 + (size_t)(e & 0xFF) * kCvHp + h] = make_float2(sg * w1.x, sg * w1.y);
        const float2 w2 = src[kCvW2 + (size_t)h * kNU + u];           // W2^T[h][u]
        out[kCvW2 + (size_t)h * kNU + (e & 0xFF)] = make_float2(sg * w2.x, sg * w2.y);
    }
    for (int h = threadIdx.x; h < kCvHp; h += blockDim.x) out[kCvB1 + h] = src[kCvB1 + h];
    for (int u = threadIdx.x; u < kNU; u += blockDim.x) {
        const uint16_t e = m[u];
        const float sg = (e & 0x100) ? -1.f : 1.f;
        const float2 b = src[kCvB2 + u];
        out[kCvB2 + (e & 0xFF)] = make_float2(sg * b.x, sg * b.y);
    }
}

// ---------------------------------------------------------------- inference
struct SmemCv {
    union {
        struct {
            float2 W[2][kKC][kCvHp];     // W1^T chunk [k][h]
            float2 X[2][kKC][kTileN];    // input chunk [k][col]
        } s1;
        float2 W2[2][kKC][kNU];          // W2^T chunk [h][u]
    } u;
    float2 Hd[kCvHp][kTileN];            // hidden activations [h][col]
    float2 b2[kNU];                      // output bias
    float scale[kTileN];                 // s = ||x||_inf per column
    float inv[kTileN];
};

// Symmetry-compressed store: the network of displacement d is the stored block's
// network in the frame of d, so a column reads the signed-permuted input copy Q of its
// group and adds output row u at U_Q(u).  Items are packed: an item's columns may come
// from every group of one stored block (pgroup: the group of each pair), each with its
// own copy, slab and output map.
struct SymArgs {
    const int32_t *gcanon = nullptr;     // [disp] stored block (null: no symmetry)
    const int32_t *gsigma = nullptr;     // [disp] copy Q of the input
    const int32_t *pgroup = nullptr;     // [pair] group of the pair (packed items)
    const uint16_t *map = nullptr;       // [48][192]
    size_t stride = 0;                   // complex elements between input copies
};

__global__ void __launch_bounds__(kThreads, 2)
cvfcnn_translate_kernel(const WorkItem *__restrict__ items, const float2 *__restrict__ Wall,
                        const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                        const float2 *__restrict__ X, float2 *__restrict__ Yslab, size_t slab_stride, int nbox,
                        const SymArgs sy, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemCv &S = *reinterpret_cast<SmemCv *>(smem_raw);
    const WorkItem it = items[blockIdx.x];
    const int tid = threadIdx.x;
    const int ncols = it.npairs * it.nr;
    const float2 *Wb = Wall + (size_t)(sy.gcanon ? sy.gcanon[it.disp] : it.disp) * kCvBlockElems;
    auto group_of = [&](int pair) { return sy.pgroup ? __ldg(sy.pgroup + pair) : it.disp; };
    // input of column col (its pair's source box, right-hand side and input copy)
    auto column_input = [&](int col) {
        const int pair = it.pair0 + col / it.nr;
        const float2 *x = X + ((int64_t)(col % it.nr) * nbox + src[pair]) * kNU;
        return sy.gcanon ? x + (size_t)__ldg(sy.gsigma + group_of(pair)) * sy.stride : x;
    };

    // column scales: 4 threads per column, 48 entries each
    {
        const int c = tid >> 2, qq = tid & 3;
        const int cc = c < ncols ? c : 0;
        const float2 *xc = column_input(cc);
        float m = 0.f;
        for (int u = qq; u < kNU; u += 4) {
            const float2 x = xc[u];
            m = fmaxf(m, x.x * x.x + x.y * x.y);
        }
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        if (qq == 0) {
            const float s = c < ncols ? sqrtf(m) : 0.f;
            S.scale[c] = s;
            S.inv[c] = s > 0.f ? 1.f / s : 0.f;
        }
    }

    // GEMM 1: z[h][col] = sum_u W1[h][u] x[u][col]
    const int lcol = tid & (kTileN - 1);
    const int lkq = tid >> 6;
    const int lc = lcol < ncols ? lcol : 0;
    const float2 *xcol = column_input(lc);
    auto load1 = [&](int kc, int buf) {
        const float4 *gw = reinterpret_cast<const float4 *>(Wb + kCvW1 + (size_t)kc * kKC * kCvHp);
        float4 *sw = reinterpret_cast<float4 *>(&S.u.s1.W[buf][0][0]);
#pragma unroll
        for (int t = 0; t < 2; ++t) cp_async16(sw + tid + t * kThreads, gw + tid + t * kThreads);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int kk = lkq * 4 + t;
            cp_async8(&S.u.s1.X[buf][kk][lcol], xcol + kc * kKC + kk);
        }
        cp_commit();
    };
    const int hm = tid >> 4;      // hidden rows {2hm, 2hm+1} + 32 i
    const int hn = tid & 15;      // columns {2hn, 2hn+1} + 32 j
    float2 z[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) z[i][j] = make_float2(0.f, 0.f);
    constexpr int nK1 = kNU / kKC;   // 12
    load1(0, 0);
    for (int kc = 0; kc < nK1; ++kc) {
        const int buf = kc & 1;
        if (kc + 1 < nK1) {
            load1(kc + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float4 v = *reinterpret_cast<const float4 *>(&S.u.s1.W[buf][kk][2 * hm + 32 * i]);
                a[2 * i] = make_float2(v.x, v.y);
                a[2 * i + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float4 v = *reinterpret_cast<const float4 *>(&S.u.s1.X[buf][kk][2 * hn + 32 * j]);
                b[2 * j] = make_float2(v.x, v.y);
                b[2 * j + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    z[i][j].x = fmaf(a[i].x, b[j].x, z[i][j].x);
                    z[i][j].x = fmaf(-a[i].y, b[j].y, z[i][j].x);
                    z[i][j].y = fmaf(a[i].x, b[j].y, z[i][j].y);
                    z[i][j].y = fmaf(a[i].y, b[j].x, z[i][j].y);
                }
        }
        __syncthreads();
    }
    // bias and Cartesian ReLU: h = relu(z / s + b1)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = 2 * hm + 32 * (i >> 1) + (i & 1);
        const float2 b1 = Wb[kCvB1 + row];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = 2 * hn + 32 * (j >> 1) + (j & 1);
            const float iv = S.inv[col];
            float2 h = make_float2(fmaxf(fmaf(z[i][j].x, iv, b1.x), 0.f), fmaxf(fmaf(z[i][j].y, iv, b1.y), 0.f));
            if (col >= ncols) h = make_float2(0.f, 0.f);
            S.Hd[row][col] = h;
        }
    }
    for (int u = tid; u < kNU; u += kThreads) S.b2[u] = Wb[kCvB2 + u];
    __syncthreads();   // Hd complete; the GEMM-1 buffers are free for GEMM 2

    // GEMM 2: o[u][col] = sum_h W2[u][h] h[h][col]
    auto load2 = [&](int kc, int buf) {
        const float4 *gw = reinterpret_cast<const float4 *>(Wb + kCvW2 + (size_t)kc * kKC * kNU);
        float4 *sw = reinterpret_cast<float4 *>(&S.u.W2[buf][0][0]);
#pragma unroll
        for (int t = 0; t < 6; ++t) cp_async16(sw + tid + t * kThreads, gw + tid + t * kThreads);
        cp_commit();
    };
    const int tm = tid >> 3;     // rows {2tm, 2tm+1} + 64 i
    const int tn = tid & 7;      // cols {2tn, 2tn+1} + 16 j
    float2 acc[6][8];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
    constexpr int nK2 = kCvHp / kKC;   // 4
    load2(0, 0);
    for (int kc = 0; kc < nK2; ++kc) {
        const int buf = kc & 1;
        if (kc + 1 < nK2) {
            load2(kc + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
            float2 a[6], b[8];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float4 v = *reinterpret_cast<const float4 *>(&S.u.W2[buf][kk][2 * tm + 64 * j]);
                a[2 * j] = make_float2(v.x, v.y);
                a[2 * j + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 v = *reinterpret_cast<const float4 *>(&S.Hd[kc * kKC + kk][2 * tn + 16 * j]);
                b[2 * j] = make_float2(v.x, v.y);
                b[2 * j + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
                    acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
                    acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
                    acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
                }
        }
        __syncthreads();
    }

    // output bias, rescale, scatter-add into the slab of the column's group (group mod kSlabs)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int col = 2 * tn + 16 * (j >> 1) + (j & 1);
        if (col >= ncols) continue;
        const float s = S.scale[col];
        float2 o[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 b = S.b2[2 * tm + 64 * (i >> 1) + (i & 1)];
            o[i] = make_float2(s * (acc[i][j].x + b.x), s * (acc[i][j].y + b.y));
        }
        const int pair = it.pair0 + col / it.nr;
        const int r = col % it.nr;
        const int grp = group_of(pair);
        float2 *ycol = Yslab + (size_t)(grp % kSlabs) * slab_stride + ((int64_t)r * nbox + dst[pair]) * kNU;
        if (sy.gcanon) {
            const uint16_t *map = sy.map + __ldg(sy.gsigma + grp) * kNU;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const uint16_t e = __ldg(map + 2 * tm + 64 * (i >> 1) + (i & 1));
                const float sg = (e & 0x100) ? -1.f : 1.f;
                atomicAdd(ycol + (e & 0xFF), make_float2(sg * o[i].x, sg * o[i].y));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float4 v = make_float4(o[2 * i].x, o[2 * i].y, o[2 * i + 1].x, o[2 * i + 1].y);
                atomicAdd(reinterpret_cast<float4 *>(ycol + 2 * tm + 64 * i), v);
            }
        }
    }
}

}  // namespace

ie_status launch_cvfcnn_fit(ie_plan p, const int32_t *canon_disp, int64_t ncanon, const int32_t *gcanon,
                            const int32_t *gsigma, const uint16_t *map, cudaStream_t st) {
    const int64_t nblk = p->n_blocks;
    if (nblk == 0 || ncanon == 0) return IE_OK;
    IE_TRY(dalloc_t(p, &p->d_cvW, (size_t)nblk * kCvBlockElems));
    const bool expand = gcanon != nullptr;
    const int64_t chunk = std::min(ncanon, kCvFitChunk);
    double2 *A = nullptr, *V = nullptr;
    double *tail = nullptr;
    int *sweeps = nullptr;
    float2 *Wc = nullptr;
    cudaError_t ae = cudaMallocAsync(&A, (size_t)chunk * kNU * kNU * sizeof(double2), st);
    if (ae == cudaSuccess) ae = cudaMallocAsync(&V, (size_t)chunk * kNU * kNU * sizeof(double2), st);
    if (ae == cudaSuccess) ae = cudaMallocAsync(&tail, (size_t)chunk * sizeof(double), st);
    if (ae == cudaSuccess) ae = cudaMallocAsync(&sweeps, (size_t)chunk * sizeof(int), st);
    if (ae == cudaSuccess && expand) ae = cudaMallocAsync(&Wc, (size_t)ncanon * kCvBlockElems * sizeof(float2), st);
    float2 *Wfit = expand ? Wc : p->d_cvW;
    std::vector<double> h_tail(chunk);
    std::vector<int> h_sweeps(chunk);
    ie_status s = IE_OK;
    if (ae != cudaSuccess) {
        cudaGetLastError();
        set_error("CVFCNN fit scratch: %s", cudaGetErrorString(ae));
        s = ae == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    }
    p->cv_sweeps = 0;
    p->cv_tail = 0.0;
    for (int64_t b0 = 0; b0 < ncanon && s == IE_OK; b0 += chunk) {
        const int64_t m = std::min(chunk, ncanon - b0);
        const int64_t threads = m * kSites * kSites;
        blocks_fp64_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(p->k, p->eta, p->a / kLattice,
                                                                          canon_disp + 3 * b0, m, A);
        count_launches(1);
        jacobi_svd_kernel<<<(unsigned)m, kJacobiThreads, 0, st>>>(A, V, sweeps);
        count_launches(1);
        cvfcnn_weights_kernel<<<(unsigned)m, 256, 0, st>>>(A, V, p->cv_hidden, Wfit + b0 * kCvBlockElems, tail);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_tail.data(), tail, m * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_sweeps.data(), sweeps, m * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("CVFCNN fit: %s", cudaGetErrorString(e));
            s = IE_ERR_CUDA;
            break;
        }
        for (int64_t i = 0; i < m; ++i) {
            p->cv_sweeps = std::max(p->cv_sweeps, h_sweeps[i]);
            p->cv_tail = std::max(p->cv_tail, h_tail[i]);
        }
    }
    if (s == IE_OK && expand) {
        cvfcnn_expand_kernel<<<(unsigned)nblk, 256, 0, st>>>(Wc, gcanon, gsigma, map, p->d_cvW);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("CVFCNN expansion: %s", cudaGetErrorString(e));
            s = IE_ERR_CUDA;
        }
    }
    for (void *ptr : {(void *)A, (void *)V, (void *)tail, (void *)sweeps, (void *)Wc})
        if (ptr) cudaFreeAsync(ptr, st);
    return s;
}

void launch_cvfcnn_expand(const float2 *Wc, const int32_t *gcanon, const int32_t *gsigma, const uint16_t *map,
                          int64_t nblk, float2 *Wd, cudaStream_t st) {
    if (nblk <= 0) return;
    cvfcnn_expand_kernel<<<(unsigned)nblk, 256, 0, st>>>(Wc, gcanon, gsigma, map, Wd);
    count_launches(1);
}

ie_status prepare_translate_cvfcnn() {
    IE_CK(cudaFuncSetAttribute(cvfcnn_translate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(SmemCv)));
    return IE_OK;
}

ie_status launch_translate_cvfcnn(ie_plan p, const float2 *X, float2 *Yslab, int nrhs, cudaStream_t st,
                                  const int *gate) {
    if (!(p->prec_mask & IE_PRECMASK(IE_PREC_CVFCNN_FP32)))
        return set_error("the plan holds no FP32 CVFCNN surrogates"), IE_ERR_UNSUPPORTED;
    WorkList *wl = nullptr;
    IE_TRY(work_list_for(p, IE_PREC_CVFCNN_FP32, nrhs, &wl));
    if (wl->n == 0) return IE_OK;
    SymArgs sy;
    if (p->sym) {
        IE_TRY(launch_permute_sym(p, X, nrhs, st, gate));
        X = p->d_Xsym;
        sy.gcanon = p->d_gcanon;
        sy.gsigma = p->d_gsigma;
        sy.pgroup = p->d_pgroup;
        sy.map = p->d_symmap;
        sy.stride = (size_t)nrhs * p->nbox * kNU;
    }
    cvfcnn_translate_kernel<<<(unsigned)wl->n, kThreads, sizeof(SmemCv), st>>>(
        wl->d_items, p->d_cvW, p->d_src, p->d_dst, X, Yslab, slab_stride(p), p->nbox, sy, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie

using namespace ie;

extern "C" ie_status ie_cvfcnn_set_weights(ie_plan p, const float *W1, const float *b1, const float *W2,
                                           const float *b2, void *stream) {
    if (!p || !W1 || !b1 || !W2 || !b2) return set_error("null argument"), IE_ERR_INVALID;
    if (!p->d_cvW) return set_error("the plan holds no CVFCNN surrogates"), IE_ERR_UNSUPPORTED;
    const int H = p->cv_hidden;
    const int64_t nblk = p->n_blocks;
    std::vector<float2> w((size_t)nblk * kCvBlockElems, make_float2(0.f, 0.f));
    auto cx = [](const float *a, size_t i) { return make_float2(a[2 * i], a[2 * i + 1]); };
    for (int64_t c = 0; c < nblk; ++c) {
        float2 *o = w.data() + (size_t)c * kCvBlockElems;
        for (int h = 0; h < H; ++h) {
            for (int u = 0; u < kNU; ++u) {
                o[kCvW1 + (size_t)u * kCvHp + h] = cx(W1, ((size_t)c * H + h) * kNU + u);
                o[kCvW2 + (size_t)h * kNU + u] = cx(W2, ((size_t)c * kNU + u) * H + h);
            }
            o[kCvB1 + h] = cx(b1, (size_t)c * H + h);
        }
        for (int u = 0; u < kNU; ++u) o[kCvB2 + u] = cx(b2, (size_t)c * kNU + u);
    }
    cudaStream_t st = (cudaStream_t)stream;
    IE_CK(cudaMemcpyAsync(p->d_cvW, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    IE_TRY(build_cvfcnn_images(p, st));
    IE_CK(cudaStreamSynchronize(st));
    return IE_OK;
}

extern "C" ie_status ie_cvfcnn_get_weights(ie_plan p, float *W1, float *b1, float *W2, float *b2, void *stream) {
    if (!p || !W1 || !b1 || !W2 || !b2) return set_error("null argument"), IE_ERR_INVALID;
    if (!p->d_cvW) return set_error("the plan holds no CVFCNN surrogates"), IE_ERR_UNSUPPORTED;
    const int H = p->cv_hidden;
    const int64_t nblk = p->n_blocks;
    std::vector<float2> w((size_t)nblk * kCvBlockElems);
    cudaStream_t st = (cudaStream_t)stream;
    IE_CK(cudaMemcpyAsync(w.data(), p->d_cvW, w.size() * sizeof(float2), cudaMemcpyDeviceToHost, st));
    IE_CK(cudaStreamSynchronize(st));
    auto put = [](float *a, size_t i, float2 v) { a[2 * i] = v.x, a[2 * i + 1] = v.y; };
    for (int64_t c = 0; c < nblk; ++c) {
        const float2 *o = w.data() + (size_t)c * kCvBlockElems;
        for (int h = 0; h < H; ++h) {
            for (int u = 0; u < kNU; ++u) {
                put(W1, ((size_t)c * H + h) * kNU + u, o[kCvW1 + (size_t)u * kCvHp + h]);
                put(W2, ((size_t)c * kNU + u) * H + h, o[kCvW2 + (size_t)h * kNU + u]);
            }
            put(b1, (size_t)c * H + h, o[kCvB1 + h]);
        }
        for (int u = 0; u < kNU; ++u) put(b2, (size_t)c * kNU + u, o[kCvB2 + u]);
    }
    return IE_OK;
}
