// Mapping construction of §2.1 (eq. 9-11): the rows of P_b for subdomain basis
// functions made of point dipoles.  The 192 uniform dipoles of a box radiate A
// (3 N_s x 192) at N_s Fibonacci samples on a sphere S about the box centre; a
// function radiates B_f there (eq. 4); eq. 11 takes C_f = A^+ B_f, row f of P_b.
//
// A is the same for every box, so A^+ is formed once: a Householder QR of A in one
// CTA, then one warp per unit vector e_i applies Q^H and back-substitutes with R,
// which gives column i of A^+ = R^-1 Q_1^H.  With a Tikhonov weight the factorised
// matrix is [A; lambda I] (lambda = t ||A||_F) and the first 3 N_s columns of its
// pseudo-inverse are (A^H A + lambda^2 I)^-1 A^H.  The per-function work (fields on S,
// the product with A^+, the residual on S) is one CTA per 8 functions.  All FP64:
// A's condition number is about 1e7, so FP32 would lose the fit.
#include "ie_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ie {
namespace {

constexpr int kMinSamples = 64;                   // 3 N_s >= 192: full column rank possible
constexpr int kMaxSamples = 256;
constexpr int kFunPerCta = 8;
constexpr int kMapThreads = 256;
constexpr int kPinvWarps = 8;
constexpr int64_t kMapChunk = int64_t(1) << 16;   // functions per device pass

struct Sphere {
    double k, eta, a, radius;   // radius of S (absolute)
    int ns;                     // samples on S
};

__device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline double2 cmul_conj(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ inline double2 warp_sum2(double2 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Sample l of the spherical Fibonacci lattice on S: polar angle arccos(1 - (2l+1)/N_s),
// azimuth 2 pi l / golden ratio.
__device__ inline void sample_point(const Sphere &s, int l, double r[3]) {
    constexpr double kPi = 3.14159265358979323846;
    const double golden = 0.5 + 0.5 * sqrt(5.0);
    double z = 1.0 - (2.0 * l + 1.0) / s.ns;
    double st = sqrt((1.0 - z) * (1.0 + z));
    double sa, ca;
    sincos(2.0 * kPi * l / golden, &sa, &ca);
    r[0] = s.radius * st * ca;
    r[1] = s.radius * st * sa;
    r[2] = s.radius * z;
}

// A (column-major, 3 N_s rows): entry (3l + alpha, 3j + beta) = D_{alpha beta}(r_l - s_j),
// s_j the cell-centred lattice site j of a box centred at the origin.  One thread per
// (sample, site).  Written into the factorised matrix (leading dimension lda >= 3 N_s)
// and into A0 (leading dimension 3 N_s), kept for the residuals.
__global__ void sample_matrix_kernel(Sphere s, double2 *__restrict__ A, int lda, double2 *__restrict__ A0) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s.ns * kSites) return;
    int l = t % s.ns, j = t / s.ns;
    double r[3];
    sample_point(s, l, r);
    const double h = s.a / kLattice;
    double q[3] = {h * ((j & 3) + 0.5) - 0.5 * s.a, h * (((j >> 2) & 3) + 0.5) - 0.5 * s.a,
                   h * ((j >> 4) + 0.5) - 0.5 * s.a};
    double2 D[9];
    dyad_fp64(s.k, s.eta, r[0] - q[0], r[1] - q[1], r[2] - q[2], D);
    const size_t m = 3 * (size_t)s.ns;
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const size_t row = 3 * (size_t)l + al, col = 3 * (size_t)j + be;
            A[row + (size_t)lda * col] = D[3 * al + be];
            A0[row + m * col] = D[3 * al + be];
        }
}

// Householder QR of A (m x 192, column-major) in one CTA.  Step j maps column j below
// the diagonal onto alpha e_j with H_j = I - tau_j v_j v_j^H, alpha = -e^{i arg x0} ||x||,
// v_j = x - alpha e_j (stored in V, rows j..m-1), tau_j = 2 / ||v_j||^2; R stays in the
// upper triangle of A.  *status = 1 if a column is zero (rank deficient).
// tikhonov > 0: rows m_data .. m_data+191 (zero on entry) first receive lambda I,
// lambda = tikhonov * ||A[0 .. m_data)||_F.
__global__ void __launch_bounds__(1024) householder_qr_kernel(double2 *__restrict__ A, int m, int m_data,
                                                              double tikhonov, double2 *__restrict__ V,
                                                              double *__restrict__ tau, int *__restrict__ status) {
    __shared__ double red[32];
    __shared__ double2 s_v0;
    __shared__ double s_tau;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    if (tikhonov > 0.0) {
        double ss = 0.0;
        for (int c = 0; c < kNU; ++c)
            for (int i = tid; i < m_data; i += blockDim.x) {
                const double2 x = A[i + (size_t)m * c];
                ss += x.x * x.x + x.y * x.y;
            }
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) red[warp] = ss;
        __syncthreads();
        if (tid < kNU) {
            double tot = 0.0;
            for (int w = 0; w < nwarp; ++w) tot += red[w];
            A[(m_data + tid) + (size_t)m * tid] = make_double2(tikhonov * sqrt(tot), 0.0);
        }
        __syncthreads();
    }
    for (int j = 0; j < kNU; ++j) {
        double2 *a = A + (size_t)m * j;
        double ss = 0.0;
        for (int i = j + tid; i < m; i += blockDim.x) ss += a[i].x * a[i].x + a[i].y * a[i].y;
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) red[warp] = ss;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < nwarp; ++w) tot += red[w];
            double xn = sqrt(tot);
            double2 x0 = a[j];
            double ax0 = hypot(x0.x, x0.y);
            double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
            if (xn == 0.0) {
                *status = 1;
                s_tau = 0.0;
                s_v0 = make_double2(0.0, 0.0);
            } else {
                s_v0 = make_double2(ph.x * (ax0 + xn), ph.y * (ax0 + xn));
                s_tau = 1.0 / (xn * (xn + ax0));            // ||v||^2 = 2 xn (xn + |x0|)
                a[j] = make_double2(-ph.x * xn, -ph.y * xn);  // R_jj = alpha
            }
            tau[j] = s_tau;
        }
        __syncthreads();
        double2 *v = V + (size_t)m * j;
        for (int i = j + tid; i < m; i += blockDim.x) v[i] = (i == j) ? s_v0 : a[i];
        __syncthreads();
        for (int c = j + 1 + warp; c < kNU; c += nwarp) {
            double2 *ac = A + (size_t)m * c;
            double2 d = make_double2(0.0, 0.0);
            for (int i = j + lane; i < m; i += 32) {
                double2 t = cmul_conj(v[i], ac[i]);
                d.x += t.x;
                d.y += t.y;
            }
            d = warp_sum2(d);
            double2 f = make_double2(s_tau * d.x, s_tau * d.y);
            for (int i = j + lane; i < m; i += 32) {
                double2 t = cmul(f, v[i]);
                ac[i].x -= t.x;
                ac[i].y -= t.y;
            }
        }
        __syncthreads();
    }
}

// Column i < m_out of the pseudo-inverse of the factorised m-row matrix (stored as row i
// of Apinv, [m_out][192]): y = Q^H e_i = H_191 ... H_0 e_i, then R x = y[0..192) by back
// substitution.  One warp per i, y in shared memory.
__global__ void pinv_kernel(const double2 *__restrict__ R, const double2 *__restrict__ V,
                            const double *__restrict__ tau, int m, int m_out, double2 *__restrict__ Apinv) {
    extern __shared__ double2 ys[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kPinvWarps + warp;
    if (i >= m_out) return;   // the whole warp leaves; nothing below synchronises the block
    double2 *y = ys + (size_t)warp * m;
    for (int r = lane; r < m; r += 32) y[r] = make_double2(r == i ? 1.0 : 0.0, 0.0);
    __syncwarp();
    for (int j = 0; j < kNU; ++j) {
        const double2 *v = V + (size_t)m * j;
        double2 d = make_double2(0.0, 0.0);
        for (int r = j + lane; r < m; r += 32) {
            double2 t = cmul_conj(v[r], y[r]);
            d.x += t.x;
            d.y += t.y;
        }
        d = warp_sum2(d);
        const double tj = tau[j];
        double2 f = make_double2(tj * d.x, tj * d.y);
        for (int r = j + lane; r < m; r += 32) {
            double2 t = cmul(f, v[r]);
            y[r].x -= t.x;
            y[r].y -= t.y;
        }
        __syncwarp();
    }
    for (int r = kNU - 1; r >= 0; --r) {
        double2 rr = R[r + (size_t)m * r];
        double2 yr = y[r];
        double den = rr.x * rr.x + rr.y * rr.y;
        double2 xr = make_double2((yr.x * rr.x + yr.y * rr.y) / den, (yr.y * rr.x - yr.x * rr.y) / den);
        __syncwarp();
        if (lane == 0) y[r] = xr;
        for (int q = lane; q < r; q += 32) {
            double2 t = cmul(R[q + (size_t)m * r], xr);
            y[q].x -= t.x;
            y[q].y -= t.y;
        }
        __syncwarp();
    }
    for (int u = lane; u < kNU; u += 32) Apinv[(size_t)i * kNU + u] = y[u];
}

struct MapArgs {
    Sphere s;
    int64_t n_fun;
    const int64_t *off;       // n_fun + 1, rebased to this chunk's dipoles
    const double *pos;        // [dipole][3]
    const double2 *mom;       // [dipole][3]
    const double2 *Apinv;     // [m][192]
    const double2 *A0;        // [192][m] (column-major A)
    double2 *P;               // [n_fun][192]
    double *res;              // [n_fun] or null
};

// Eight functions per CTA: their fields on S (eq. 4 summed over the point dipoles),
// C_f = A^+ B_f (eq. 11), and ||A C_f - B_f|| / ||B_f||.
__global__ void __launch_bounds__(kMapThreads) map_kernel(MapArgs g) {
    extern __shared__ double2 sm[];
    __shared__ double red[2][kFunPerCta][kMapThreads / 32];
    const int m = 3 * g.s.ns;
    double2 *B = sm;                        // [kFunPerCta][m]
    double2 *C = sm + kFunPerCta * m;       // [kFunPerCta][192]
    const int64_t f0 = (int64_t)blockIdx.x * kFunPerCta;
    for (int idx = threadIdx.x; idx < kFunPerCta * g.s.ns; idx += blockDim.x) {
        const int t = idx / g.s.ns, l = idx % g.s.ns;
        const int64_t f = f0 + t;
        double2 e[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
        if (f < g.n_fun) {
            double r[3];
            sample_point(g.s, l, r);
            for (int64_t d = g.off[f]; d < g.off[f + 1]; ++d) {
                double2 D[9];
                dyad_fp64(g.s.k, g.s.eta, r[0] - g.pos[3 * d], r[1] - g.pos[3 * d + 1], r[2] - g.pos[3 * d + 2], D);
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) {
                        double2 p = cmul(D[3 * al + be], g.mom[3 * d + be]);
                        e[al].x += p.x;
                        e[al].y += p.y;
                    }
            }
        }
#pragma unroll
        for (int al = 0; al < 3; ++al) B[t * m + 3 * l + al] = e[al];
    }
    __syncthreads();
    if (threadIdx.x < kNU) {
        const int u = threadIdx.x;
        double2 acc[kFunPerCta];
#pragma unroll
        for (int t = 0; t < kFunPerCta; ++t) acc[t] = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) {
            const double2 w = g.Apinv[(size_t)i * kNU + u];
#pragma unroll
            for (int t = 0; t < kFunPerCta; ++t) {
                double2 p = cmul(w, B[t * m + i]);
                acc[t].x += p.x;
                acc[t].y += p.y;
            }
        }
#pragma unroll
        for (int t = 0; t < kFunPerCta; ++t) {
            C[t * kNU + u] = acc[t];
            if (f0 + t < g.n_fun) g.P[(f0 + t) * kNU + u] = acc[t];
        }
    }
    if (!g.res) return;
    __syncthreads();
    double rr[kFunPerCta], bb[kFunPerCta];
#pragma unroll
    for (int t = 0; t < kFunPerCta; ++t) rr[t] = bb[t] = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 s[kFunPerCta];
#pragma unroll
        for (int t = 0; t < kFunPerCta; ++t) s[t] = make_double2(0.0, 0.0);
        for (int u = 0; u < kNU; ++u) {
            const double2 a = g.A0[i + (size_t)m * u];
#pragma unroll
            for (int t = 0; t < kFunPerCta; ++t) {
                double2 p = cmul(a, C[t * kNU + u]);
                s[t].x += p.x;
                s[t].y += p.y;
            }
        }
#pragma unroll
        for (int t = 0; t < kFunPerCta; ++t) {
            const double2 b = B[t * m + i];
            const double dx = s[t].x - b.x, dy = s[t].y - b.y;
            rr[t] += dx * dx + dy * dy;
            bb[t] += b.x * b.x + b.y * b.y;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < kFunPerCta; ++t) {
        for (int o = 16; o; o >>= 1) {
            rr[t] += __shfl_xor_sync(0xffffffffu, rr[t], o);
            bb[t] += __shfl_xor_sync(0xffffffffu, bb[t], o);
        }
        if (lane == 0) {
            red[0][t][warp] = rr[t];
            red[1][t][warp] = bb[t];
        }
    }
    __syncthreads();
    if (threadIdx.x < kFunPerCta) {
        const int t = threadIdx.x;
        double r2 = 0.0, b2 = 0.0;
        for (int w = 0; w < kMapThreads / 32; ++w) {
            r2 += red[0][t][w];
            b2 += red[1][t][w];
        }
        if (f0 + t < g.n_fun) g.res[f0 + t] = b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
    }
}

// Device buffers of one ie_map_basis call, freed on every return path.
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    ie_status get(T **out, size_t count) {
        *out = nullptr;
        if (count == 0) return IE_OK;
        cudaError_t e = cudaMalloc((void **)out, count * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
        }
        ptrs.push_back(*out);
        return IE_OK;
    }
};

bool finite_positive(double x) { return std::isfinite(x) && x > 0.0; }

ie_status validate(const ie_mapping_spec *spec, int64_t n_fun, const int64_t *fun_off, const double *pos,
                   const double *mom, const double *P) {
    if (!spec) return set_error("null spec"), IE_ERR_INVALID;
    if (!finite_positive(spec->k) || !finite_positive(spec->eta) || !finite_positive(spec->box_edge))
        return set_error("k, eta and box_edge must be positive and finite"), IE_ERR_INVALID;
    if (spec->lattice != kLattice) return set_error("lattice %d: only 4 is supported", spec->lattice), IE_ERR_INVALID;
    if (spec->n_samples < kMinSamples || spec->n_samples > kMaxSamples)
        return set_error("n_samples %d outside [%d, %d]", spec->n_samples, kMinSamples, kMaxSamples), IE_ERR_INVALID;
    if (!std::isfinite(spec->sample_radius) || !(spec->sample_radius > 0.5 * std::sqrt(3.0)))
        return set_error("sample_radius %g must exceed sqrt(3)/2 (S must enclose the box)", spec->sample_radius),
               IE_ERR_INVALID;
    if (!std::isfinite(spec->tikhonov) || spec->tikhonov < 0.0)
        return set_error("tikhonov %g must be finite and >= 0", spec->tikhonov), IE_ERR_INVALID;
    if (n_fun < 0) return set_error("n_fun %lld < 0", (long long)n_fun), IE_ERR_INVALID;
    if (n_fun == 0) return IE_OK;
    if (!fun_off || !P) return set_error("null fun_off or P"), IE_ERR_INVALID;
    if (fun_off[0] != 0) return set_error("fun_off[0] = %lld, must be 0", (long long)fun_off[0]), IE_ERR_INVALID;
    for (int64_t f = 0; f < n_fun; ++f)
        if (fun_off[f + 1] < fun_off[f])
            return set_error("fun_off decreases at function %lld", (long long)f), IE_ERR_INVALID;
    const int64_t nd = fun_off[n_fun];
    if (nd > 0 && (!pos || !mom)) return set_error("null pos or mom"), IE_ERR_INVALID;
    const double rs = spec->sample_radius * spec->box_edge;
    for (int64_t d = 0; d < nd; ++d) {
        const double *x = pos + 3 * d;
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(x[c])) return set_error("non-finite position of dipole %lld", (long long)d), IE_ERR_INVALID;
        for (int c = 0; c < 6; ++c)
            if (!std::isfinite(mom[6 * d + c]))
                return set_error("non-finite moment of dipole %lld", (long long)d), IE_ERR_INVALID;
        if (!(std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) < rs))
            return set_error("dipole %lld lies outside the sampling sphere (radius %g)", (long long)d, rs),
                   IE_ERR_INVALID;
    }
    return IE_OK;
}

}  // namespace
}  // namespace ie

using namespace ie;

extern "C" ie_status ie_map_basis(const ie_mapping_spec *spec, int64_t n_fun, const int64_t *fun_off,
                                  const double *pos, const double *mom, double *P, double *residual,
                                  void *stream) {
    IE_TRY(validate(spec, n_fun, fun_off, pos, mom, P));
    if (n_fun == 0) return IE_OK;
    NvtxRange nv("ie_map_basis");
    cudaStream_t st = (cudaStream_t)stream;
    const Sphere s{spec->k, spec->eta, spec->box_edge, spec->sample_radius * spec->box_edge, spec->n_samples};
    const int m = 3 * s.ns;                                      // rows of A
    const int mf = spec->tikhonov > 0.0 ? m + kNU : m;           // rows of the factorised matrix
    Scratch sc;
    double2 *A, *A0, *V, *Apinv;
    double *tau;
    int *status;
    IE_TRY(sc.get(&A, (size_t)mf * kNU));
    IE_TRY(sc.get(&A0, (size_t)m * kNU));
    IE_TRY(sc.get(&V, (size_t)mf * kNU));
    IE_TRY(sc.get(&Apinv, (size_t)m * kNU));
    IE_TRY(sc.get(&tau, kNU));
    IE_TRY(sc.get(&status, 1));
    IE_CK(cudaMemsetAsync(status, 0, sizeof(int), st));
    IE_CK(cudaMemsetAsync(A, 0, (size_t)mf * kNU * sizeof(double2), st));
    IE_CK(cudaMemsetAsync(V, 0, (size_t)mf * kNU * sizeof(double2), st));

    sample_matrix_kernel<<<(s.ns * kSites + 255) / 256, 256, 0, st>>>(s, A, mf, A0);
    IE_CK_LAUNCH();
    householder_qr_kernel<<<1, 1024, 0, st>>>(A, mf, m, spec->tikhonov, V, tau, status);
    IE_CK_LAUNCH();
    int h_status = 0;
    IE_CK(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    IE_CK(cudaStreamSynchronize(st));
    if (h_status) return set_error("the uniform-dipole field matrix A is rank deficient"), IE_ERR_INVALID;
    const size_t pinv_smem = (size_t)kPinvWarps * mf * sizeof(double2);
    IE_CK(cudaFuncSetAttribute(pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pinv_smem));
    pinv_kernel<<<(m + kPinvWarps - 1) / kPinvWarps, 32 * kPinvWarps, pinv_smem, st>>>(A, V, tau, mf, m, Apinv);
    IE_CK_LAUNCH();

    const size_t map_smem = (size_t)kFunPerCta * (m + kNU) * sizeof(double2);
    IE_CK(cudaFuncSetAttribute(map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)map_smem));
    const int64_t chunk = n_fun < kMapChunk ? n_fun : kMapChunk;
    int64_t max_dip = 0;
    for (int64_t f0 = 0; f0 < n_fun; f0 += chunk) {
        int64_t f1 = f0 + chunk < n_fun ? f0 + chunk : n_fun;
        max_dip = std::max(max_dip, fun_off[f1] - fun_off[f0]);
    }
    int64_t *d_off;
    double *d_pos, *d_res = nullptr;
    double2 *d_mom, *d_P;
    IE_TRY(sc.get(&d_off, (size_t)chunk + 1));
    IE_TRY(sc.get(&d_pos, 3 * (size_t)max_dip));
    IE_TRY(sc.get(&d_mom, 3 * (size_t)max_dip));
    IE_TRY(sc.get(&d_P, (size_t)chunk * kNU));
    if (residual) IE_TRY(sc.get(&d_res, (size_t)chunk));
    std::vector<int64_t> off(chunk + 1);
    for (int64_t f0 = 0; f0 < n_fun; f0 += chunk) {
        const int64_t nf = std::min(chunk, n_fun - f0);
        const int64_t d0 = fun_off[f0], nd = fun_off[f0 + nf] - d0;
        for (int64_t f = 0; f <= nf; ++f) off[f] = fun_off[f0 + f] - d0;
        IE_CK(cudaMemcpyAsync(d_off, off.data(), (nf + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        if (nd > 0) {
            IE_CK(cudaMemcpyAsync(d_pos, pos + 3 * d0, 3 * nd * sizeof(double), cudaMemcpyHostToDevice, st));
            IE_CK(cudaMemcpyAsync(d_mom, mom + 6 * d0, 3 * nd * sizeof(double2), cudaMemcpyHostToDevice, st));
        }
        MapArgs g{s, nf, d_off, d_pos, d_mom, Apinv, A0, d_P, d_res};
        map_kernel<<<(unsigned)((nf + kFunPerCta - 1) / kFunPerCta), kMapThreads, map_smem, st>>>(g);
        IE_CK_LAUNCH();
        IE_CK(cudaMemcpyAsync(P + 2 * (size_t)f0 * kNU, d_P, (size_t)nf * kNU * sizeof(double2),
                              cudaMemcpyDeviceToHost, st));
        if (residual)
            IE_CK(cudaMemcpyAsync(residual + f0, d_res, nf * sizeof(double), cudaMemcpyDeviceToHost, st));
        // the staging buffers are reused by the next chunk
        IE_CK(cudaStreamSynchronize(st));
    }
    return IE_OK;
}
