// K6 / K8: restarted GMRES without preconditioning (§5, the paper's iterative
// solver) with device-resident state, and outer iterative refinement.
//
// Each right-hand side is an independent GMRES(m) (x0 = 0).  Arnoldi uses classical
// Gram-Schmidt applied twice (dot products accumulated in FP64), Givens rotations
// and the small least-squares solve run in FP64; Krylov vectors are FP32.  One
// restart cycle (m iterations, the solution update and the restart residual) is
// captured once as a CUDA graph and replayed; every kernel reads per-RHS flags in
// device memory, so iterations after convergence cost nothing but the launch and
// the host synchronises once per cycle.
#include <chrono>
#include <cmath>
#include <cstdio>

#include "ie_internal.h"

struct ie_solver_s {
    ie_plan plan = nullptr;
    int R = 1, m = 50, max_iters = 1000, prec = IE_PREC_FP32;
    double tol = 1e-6;
    int64_t n = 0;
    int nblk = 1;
    float2 *V = nullptr;         // [(m+1)][R][n]
    float2 *W = nullptr;         // [R][n]
    double2 *H = nullptr;        // [R][m][m+1]
    double *cs = nullptr;        // [R][m]
    double2 *sn = nullptr;       // [R][m]
    double2 *g = nullptr;        // [R][m+1]
    double2 *hbuf = nullptr;     // [R][m+1]
    double2 *partial = nullptr;  // [R][m+1][nblk]
    double *bnorm = nullptr;     // [R]
    double *relres = nullptr;    // [R]
    int *st = nullptr;           // [4 + 4R]: any_active, any_not_done, done[R], active[R], jend[R], iters[R], j, body runs
    float2 *Vcur = nullptr;      // [R][n] current Krylov vector (input of the product)
    cudaGraphConditionalHandle hcond = 0;
    bool use_while = false;
    int64_t body_kernels = 0, end_kernels = 0, body_runs_seen = 0;
    const float2 *v = nullptr;
    float2 *x = nullptr;
    const float2 *cap_v = nullptr;   // pointers baked into the captured cycle
    float2 *cap_x = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev = nullptr;
    int matvecs_per_cycle = 0;
    int cycles_run = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;
};

namespace ie {
namespace {

constexpr int kDotThreads = 256;
constexpr int kEPT = 4;                        // elements per thread in the dot kernels
constexpr int kChunk = kDotThreads * kEPT;

__device__ inline int *st_done(int *st, int R) { return st + 2; }
__device__ inline int *st_active(int *st, int R) { return st + 2 + R; }
__device__ inline int *st_jend(int *st, int R) { return st + 2 + 2 * R; }
__device__ inline int *st_iters(int *st, int R) { return st + 2 + 3 * R; }
__device__ inline int *st_jdev(int *st, int R) { return st + 2 + 4 * R; }     // Arnoldi index of the cycle
__device__ inline int *st_body(int *st, int R) { return st + 3 + 4 * R; }     // iterations run by the graph

// j >= 0: index given by the launch; kDevJ: read the cycle's index from device memory
// (the WHILE-node graph runs one body for every iteration).
constexpr int kDevJ = -2;
__device__ inline int resolve_j(int j, int *st, int R) { return j >= 0 ? j : *st_jdev(st, R); }

__device__ inline double2 block_sum2(double2 v) {
    __shared__ double2 red[kDotThreads / 32];
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double2 s = make_double2(0, 0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s.x += red[i].x, s.y += red[i].y;
    return s;   // valid in thread 0
}

// partial[r][i][blk] = sum over the block's slice of conj(V_i[r]) . W[r], i <= j.
// j < 0: partial[r][0][blk] = sum |W[r]|^2 (norm pass).  Only rows with active[r]
// (or not done[r] when use_done) take part.
__global__ void dots_kernel(const float2 *__restrict__ V, const float2 *__restrict__ Wv, int64_t n, int R, int jarg,
                            double2 *__restrict__ partial, int nblk, int m, int *st, int use_done, int norm) {
    int r = blockIdx.y, blk = blockIdx.x;
    const int j = norm ? -1 : resolve_j(jarg, st, R);
    bool on = use_done ? !st_done(st, R)[r] : st_active(st, R)[r];
    if (!on) return;
    int64_t base = (int64_t)blk * kChunk;
    float2 w[kEPT];
    const float2 *wr = Wv + (int64_t)r * n;
#pragma unroll
    for (int t = 0; t < kEPT; ++t) {
        int64_t e = base + threadIdx.x + t * kDotThreads;
        w[t] = e < n ? wr[e] : make_float2(0.f, 0.f);
    }
    double2 *pr = partial + ((int64_t)r * (m + 1)) * nblk;
    if (j < 0) {
        double s = 0;
#pragma unroll
        for (int t = 0; t < kEPT; ++t) s += (double)w[t].x * w[t].x + (double)w[t].y * w[t].y;
        double2 tot = block_sum2(make_double2(s, 0));
        if (threadIdx.x == 0) pr[blk] = tot;
        return;
    }
    for (int i = 0; i <= j; ++i) {
        const float2 *vi = V + ((int64_t)i * R + r) * n;
        double sr = 0, si = 0;
#pragma unroll
        for (int t = 0; t < kEPT; ++t) {
            int64_t e = base + threadIdx.x + t * kDotThreads;
            float2 a = e < n ? vi[e] : make_float2(0.f, 0.f);
            // conj(a) * w
            sr += (double)a.x * w[t].x + (double)a.y * w[t].y;
            si += (double)a.x * w[t].y - (double)a.y * w[t].x;
        }
        double2 tot = block_sum2(make_double2(sr, si));
        if (threadIdx.x == 0) pr[(int64_t)i * nblk + blk] = tot;
    }
}

// hbuf[r][i] = sum_blk partial; H[r][j][i] += hbuf (Arnoldi coefficient of pass).
__global__ void reduce_dots_kernel(const double2 *__restrict__ partial, int nblk, int m, int R, int jarg,
                                   double2 *__restrict__ hbuf, double2 *__restrict__ H, int *st) {
    int r = blockIdx.x;
    if (!st_active(st, R)[r]) return;
    const int j = resolve_j(jarg, st, R);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 *p = partial + ((int64_t)r * (m + 1) + i) * nblk;
        double sx = 0, sy = 0;
        for (int b = 0; b < nblk; ++b) sx += p[b].x, sy += p[b].y;
        hbuf[(int64_t)r * (m + 1) + i] = make_double2(sx, sy);
        double2 &h = H[((int64_t)r * m + j) * (m + 1) + i];
        h.x += sx;
        h.y += sy;
    }
}

// W[r] -= sum_{i<=j} V_i[r] hbuf[r][i]
__global__ void update_kernel(const float2 *__restrict__ V, float2 *__restrict__ Wv, int64_t n, int R, int jarg,
                              int m, const double2 *__restrict__ hbuf, int *st) {
    int r = blockIdx.y;
    if (!st_active(st, R)[r]) return;
    const int j = resolve_j(jarg, st, R);
    __shared__ float2 h[65];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        double2 v = hbuf[(int64_t)r * (m + 1) + i];
        h[i] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    float2 *wr = Wv + (int64_t)r * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float2 w = wr[e];
        for (int i = 0; i <= j; ++i) {
            float2 a = V[((int64_t)i * R + r) * n + e];
            w.x -= a.x * h[i].x - a.y * h[i].y;
            w.y -= a.x * h[i].y + a.y * h[i].x;
        }
        wr[e] = w;
    }
}

// ||W[r]|| -> H[r][j][j+1] (and hbuf[r][0] = norm for the scaling kernel).
__global__ void norm_finish_kernel(const double2 *__restrict__ partial, int nblk, int m, int R, int jarg,
                                   double2 *__restrict__ hbuf, double2 *__restrict__ H, int *st) {
    int r = blockIdx.x;
    if (!st_active(st, R)[r]) return;
    const int j = resolve_j(jarg, st, R);
    if (threadIdx.x != 0) return;
    const double2 *p = partial + ((int64_t)r * (m + 1)) * nblk;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += p[b].x;
    double hn = sqrt(s);
    H[((int64_t)r * m + j) * (m + 1) + j + 1] = make_double2(hn, 0);
    hbuf[(int64_t)r * (m + 1)] = make_double2(hn, 0);
}

// V_{j+1}[r] = W[r] / hn, also written to Vcur (the next product's input)
__global__ void scale_kernel(const float2 *__restrict__ Wv, float2 *__restrict__ V, float2 *__restrict__ Vcur,
                             int64_t n, int R, int m, const double2 *__restrict__ hbuf, int *st, int jarg) {
    int r = blockIdx.y;
    if (!st_active(st, R)[r]) return;
    const int j = resolve_j(jarg, st, R);
    double hn = hbuf[(int64_t)r * (m + 1)].x;
    float s = hn > 0 ? (float)(1.0 / hn) : 0.f;
    const float2 *wr = Wv + (int64_t)r * n;
    float2 *vr = V + ((int64_t)(j + 1) * R + r) * n;
    float2 *cr = Vcur + (int64_t)r * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float2 w = wr[e];
        float2 o = make_float2(w.x * s, w.y * s);
        vr[e] = o;
        cr[e] = o;
    }
}

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double cabs2(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }

// Givens update of column j, residual estimate, per-RHS termination; one thread per RHS.
__global__ void givens_kernel(double2 *__restrict__ H, double *__restrict__ cs, double2 *__restrict__ sn,
                              double2 *__restrict__ g, const double *__restrict__ bnorm, double *__restrict__ relres,
                              int m, int R, int jarg, double tol, int max_iters, int *st,
                              cudaGraphConditionalHandle cond) {
    int r = threadIdx.x;
    const int j = resolve_j(jarg, st, R);
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    if (r < R && st_active(st, R)[r]) {
        double2 *h = H + ((int64_t)r * m + j) * (m + 1);
        double *c = cs + (int64_t)r * m;
        double2 *s = sn + (int64_t)r * m;
        double2 *gr = g + (int64_t)r * (m + 1);
        for (int i = 0; i < j; ++i) {
            double2 a = h[i], b = h[i + 1];
            double2 t = make_double2(c[i] * a.x + cmul(s[i], b).x, c[i] * a.y + cmul(s[i], b).y);
            double2 u = cmul(conj2(s[i]), a);
            h[i + 1] = make_double2(-u.x + c[i] * b.x, -u.y + c[i] * b.y);
            h[i] = t;
        }
        double2 a = h[j], b = h[j + 1];
        double na = cabs2(a), nb = cabs2(b);
        double den = sqrt(na * na + nb * nb);
        double cj;
        double2 sj;
        if (den == 0) {
            cj = 1, sj = make_double2(0, 0);
        } else if (na == 0) {
            cj = 0, sj = make_double2(b.x / nb, -b.y / nb);
        } else {
            cj = na / den;
            double2 ph = make_double2(a.x / na, a.y / na);
            sj = cmul(ph, make_double2(b.x / den, -b.y / den));
        }
        c[j] = cj;
        s[j] = sj;
        double2 hj = make_double2(cj * a.x + cmul(sj, b).x, cj * a.y + cmul(sj, b).y);
        h[j] = hj;
        h[j + 1] = make_double2(0, 0);
        double2 gj = gr[j];
        double2 gn = cmul(conj2(sj), gj);
        gr[j + 1] = make_double2(-gn.x, -gn.y);
        gr[j] = make_double2(cj * gj.x, cj * gj.y);
        int it = ++st_iters(st, R)[r];
        st_jend(st, R)[r] = j + 1;
        double res = cabs2(gr[j + 1]) / bnorm[r];
        relres[r] = res;
        bool breakdown = nb == 0;
        if (res <= tol || it >= max_iters || breakdown || j + 1 == m) st_active(st, R)[r] = 0;
        if (st_active(st, R)[r]) any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st[0] = any;
        if (jarg == kDevJ) {
            *st_jdev(st, R) = j + 1;
            *st_body(st, R) += 1;
            cudaGraphSetConditional(cond, any ? 1u : 0u);   // WHILE node: run the next iteration?
        }
    }
}

// Back substitution H[0:jend,0:jend] y = g[0:jend]; y stored in hbuf[r].
__global__ void lsq_kernel(const double2 *__restrict__ H, const double2 *__restrict__ g, double2 *__restrict__ y,
                           int m, int R, int *st) {
    int r = threadIdx.x;
    if (r >= R) return;
    int je = st_jend(st, R)[r];
    double2 *yr = y + (int64_t)r * (m + 1);
    for (int i = je - 1; i >= 0; --i) {
        double2 s = g[(int64_t)r * (m + 1) + i];
        for (int k = i + 1; k < je; ++k) {
            double2 t = cmul(H[((int64_t)r * m + k) * (m + 1) + i], yr[k]);
            s.x -= t.x, s.y -= t.y;
        }
        double2 d = H[((int64_t)r * m + i) * (m + 1) + i];
        double dd = d.x * d.x + d.y * d.y;
        yr[i] = dd > 0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd) : make_double2(0, 0);
    }
}

// x[r] += sum_{i<jend} V_i[r] y[r][i]
__global__ void xupdate_kernel(const float2 *__restrict__ V, float2 *__restrict__ x, int64_t n, int R, int m,
                               const double2 *__restrict__ y, int *st) {
    int r = blockIdx.y;
    int je = st_jend(st, R)[r];
    if (je == 0) return;
    __shared__ float2 ys[65];
    for (int i = threadIdx.x; i < je; i += blockDim.x) {
        double2 v = y[(int64_t)r * (m + 1) + i];
        ys[i] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    float2 *xr = x + (int64_t)r * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float2 acc = xr[e];
        for (int i = 0; i < je; ++i) {
            float2 a = V[((int64_t)i * R + r) * n + e];
            acc.x += a.x * ys[i].x - a.y * ys[i].y;
            acc.y += a.x * ys[i].y + a.y * ys[i].x;
        }
        xr[e] = acc;
    }
}

// V_0[r] = v[r] - W[r] for rows not done (W = Z x); `copy` = 1: V_0 = v (start).
__global__ void residual_kernel(const float2 *__restrict__ v, const float2 *__restrict__ Wv, float2 *__restrict__ V0,
                                int64_t n, int R, int copy, int *st) {
    int r = blockIdx.y;
    if (st_done(st, R)[r]) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = (int64_t)r * n + e;
        float2 a = v[i];
        if (!copy) {
            float2 b = Wv[i];
            a.x -= b.x;
            a.y -= b.y;
        }
        V0[i] = a;
    }
}

// Begin a cycle from V_0 = residual: beta = ||V_0||; termination tests; g, H reset.
// start = 1: also sets bnorm = beta (x0 = 0) and clears the counters.
__global__ void begin_cycle_kernel(const double2 *__restrict__ partial, int nblk, int m, int R, double tol,
                                   int max_iters, double *__restrict__ bnorm, double *__restrict__ relres,
                                   double2 *__restrict__ g, double2 *__restrict__ H, double2 *__restrict__ hbuf,
                                   int start, int *st) {
    __shared__ int any_active, any_open;
    if (threadIdx.x == 0) any_active = 0, any_open = 0;
    __syncthreads();
    for (int r = 0; r < R; ++r) {
        // zero this RHS's H (all threads), then thread 0 decides
        bool skip = !start && st_done(st, R)[r];
        if (!skip)
            for (int i = threadIdx.x; i < m * (m + 1); i += blockDim.x) H[(int64_t)r * m * (m + 1) + i] = make_double2(0, 0);
        if (threadIdx.x == 0) {
            if (start) {
                st_done(st, R)[r] = 0;
                st_iters(st, R)[r] = 0;
            }
            st_jend(st, R)[r] = 0;
            st_active(st, R)[r] = 0;
            if (!st_done(st, R)[r]) {
                const double2 *p = partial + ((int64_t)r * (m + 1)) * nblk;
                double s = 0;
                for (int b = 0; b < nblk; ++b) s += p[b].x;
                double beta = sqrt(s);
                if (start) bnorm[r] = beta;
                double rel = bnorm[r] > 0 ? beta / bnorm[r] : 0.0;
                relres[r] = rel;
                if (bnorm[r] == 0 || rel <= tol || st_iters(st, R)[r] >= max_iters) {
                    st_done(st, R)[r] = 1;
                } else {
                    st_active(st, R)[r] = 1;
                    double2 *gr = g + (int64_t)r * (m + 1);
                    gr[0] = make_double2(beta, 0);
                    for (int i = 1; i <= m; ++i) gr[i] = make_double2(0, 0);
                    hbuf[(int64_t)r * (m + 1)] = make_double2(beta, 0);
                    any_active = 1;
                }
                if (!st_done(st, R)[r]) any_open = 1;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st[0] = any_active;
        st[1] = any_open;
        *st_jdev(st, R) = 0;
    }
}

// V_0[r] /= beta (hbuf[r][0]) for active rows.
__global__ void scale_v0_kernel(float2 *__restrict__ V0, float2 *__restrict__ Vcur, int64_t n, int R, int m,
                                const double2 *__restrict__ hbuf, int *st) {
    int r = blockIdx.y;
    if (!st_active(st, R)[r]) return;
    double b = hbuf[(int64_t)r * (m + 1)].x;
    float s = (float)(1.0 / b);
    float2 *vr = V0 + (int64_t)r * n;
    float2 *cr = Vcur + (int64_t)r * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float2 a = vr[e];
        float2 o = make_float2(a.x * s, a.y * s);
        vr[e] = o;
        cr[e] = o;
    }
}

// ---- refinement helpers (FP64 outer loop) ----
__global__ void ref_residual_kernel(const float2 *__restrict__ v, const float2 *__restrict__ Wv,
                                    float2 *__restrict__ rout, int64_t n, double2 *__restrict__ partial, int nblk) {
    // r = v - W in FP64; partial[r][blk] = (||r||^2, ||v||^2)
    int r = blockIdx.y, blk = blockIdx.x;
    double s = 0, sv = 0;
    for (int t = 0; t < kEPT; ++t) {
        int64_t e = (int64_t)blk * kChunk + threadIdx.x + t * kDotThreads;
        if (e >= n) continue;
        int64_t i = (int64_t)r * n + e;
        float2 a = v[i], b = Wv[i];
        double rx = (double)a.x - (double)b.x, ry = (double)a.y - (double)b.y;
        rout[i] = make_float2((float)rx, (float)ry);
        s += rx * rx + ry * ry;
        sv += (double)a.x * a.x + (double)a.y * a.y;
    }
    double2 tot = block_sum2(make_double2(s, sv));
    if (threadIdx.x == 0) partial[(int64_t)r * nblk + blk] = tot;
}

__global__ void ref_accumulate_kernel(double2 *__restrict__ x64, const float2 *__restrict__ d, float2 *__restrict__ x32,
                                      int64_t total, int zero) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        double2 a = zero ? make_double2(0, 0) : x64[i];
        if (!zero) {
            a.x += d[i].x;
            a.y += d[i].y;
        }
        x64[i] = a;
        x32[i] = make_float2((float)a.x, (float)a.y);
    }
}

int vec_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)std::min<int64_t>(g, 1024);
}

}  // namespace
}  // namespace ie

using namespace ie;

namespace ie {
void destroy_cached_solvers(ie_plan p) {
    for (auto &kv : p->solvers) ie_solver_destroy(kv.second);
    p->solvers.clear();
}
}  // namespace ie

namespace {

// A solver of `plan` for these options, created on first use and kept in the plan.
ie_status cached_solver(ie_plan p, int nrhs, const ie_solve_opts &o, ie_solver *out) {
    char key[160];
    snprintf(key, sizeof(key), "%d/%d/%d/%.17g/%d", nrhs, o.restart, o.max_iters, o.tol, o.prec);
    for (auto &kv : p->solvers)
        if (kv.first == key) {
            *out = kv.second;
            return IE_OK;
        }
    ie_solver s = nullptr;
    IE_TRY(ie_solver_create(p, nrhs, &o, &s));
    p->solvers.emplace_back(key, s);
    *out = s;
    return IE_OK;
}

ie_status salloc(ie_solver s, void **p, size_t bytes) {
    *p = nullptr;
    if (!bytes) return IE_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("solver cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    }
    s->allocs.push_back(*p);
    s->bytes += bytes;
    return IE_OK;
}
template <class T>
ie_status salloc_t(ie_solver s, T **p, size_t count) {
    return salloc(s, reinterpret_cast<void **>(p), count * sizeof(T));
}

size_t solver_bytes(int64_t n, int R, int m) {
    int nblk = (int)((n + kChunk - 1) / kChunk);
    size_t b = 0;
    b += (size_t)(m + 1) * R * n * sizeof(float2);
    b += (size_t)R * n * sizeof(float2);
    b += (size_t)R * m * (m + 1) * sizeof(double2);
    b += (size_t)R * m * (sizeof(double) + sizeof(double2));
    b += (size_t)R * (m + 1) * sizeof(double2) * 2;
    b += (size_t)R * (m + 1) * nblk * sizeof(double2);
    b += (size_t)R * 2 * sizeof(double) + (4 + 4 * R) * sizeof(int);
    b += (size_t)R * n * sizeof(float2);
    return b;
}

void fill_defaults(ie_solve_opts *o) {
    o->restart = 50;
    o->max_iters = 1000;
    o->tol = 1e-6;
    o->prec = IE_PREC_FP32;
    o->refine = 0;
    o->refine_prec = IE_PREC_FP32;
    o->inner_tol = 1e-3;
    o->max_refine = 20;
}

// One Arnoldi iteration (product, CGS2, norm, scaling, Givens).  jarg = kDevJ takes
// the index from device memory (body of the WHILE node).
ie_status enqueue_iteration(ie_solver s, cudaStream_t st, int jarg) {
    ie_plan p = s->plan;
    int R = s->R, m = s->m;
    int64_t n = s->n;
    dim3 vg(vec_grid(n), R), dg(s->nblk, R);
    IE_TRY(apply(p, IE_FULL, s->prec, s->Vcur, s->W, R, st, s->st));
    for (int pass = 0; pass < 2; ++pass) {
        dots_kernel<<<dg, kDotThreads, 0, st>>>(s->V, s->W, n, R, jarg, s->partial, s->nblk, m, s->st, 0, 0);
        reduce_dots_kernel<<<R, 64, 0, st>>>(s->partial, s->nblk, m, R, jarg, s->hbuf, s->H, s->st);
        update_kernel<<<vg, 256, 0, st>>>(s->V, s->W, n, R, jarg, m, s->hbuf, s->st);
    }
    dots_kernel<<<dg, kDotThreads, 0, st>>>(s->V, s->W, n, R, jarg, s->partial, s->nblk, m, s->st, 0, 1);
    norm_finish_kernel<<<R, 32, 0, st>>>(s->partial, s->nblk, m, R, jarg, s->hbuf, s->H, s->st);
    scale_kernel<<<vg, 256, 0, st>>>(s->W, s->V, s->Vcur, n, R, m, s->hbuf, s->st, jarg);
    givens_kernel<<<1, 64, 0, st>>>(s->H, s->cs, s->sn, s->g, s->bnorm, s->relres, m, R, jarg, s->tol, s->max_iters,
                                    s->st, s->hcond);
    count_launches(9);   // the ten kernels above (IE_CK_LAUNCH adds the last)
    IE_CK_LAUNCH();
    return IE_OK;
}

// Solution update x += V y and the restart: true residual, its norm, next cycle.
ie_status enqueue_end(ie_solver s, cudaStream_t st) {
    ie_plan p = s->plan;
    int R = s->R, m = s->m;
    int64_t n = s->n;
    dim3 vg(vec_grid(n), R), dg(s->nblk, R);
    lsq_kernel<<<1, 64, 0, st>>>(s->H, s->g, s->hbuf, m, R, s->st);
    xupdate_kernel<<<vg, 256, 0, st>>>(s->V, s->x, n, R, m, s->hbuf, s->st);
    count_launches(2);
    IE_TRY(apply(p, IE_FULL, s->prec, s->x, s->W, R, st, s->st + 1));
    residual_kernel<<<vg, 256, 0, st>>>(s->v, s->W, s->V, n, R, 0, s->st);
    dots_kernel<<<dg, kDotThreads, 0, st>>>(s->V, s->V, n, R, 0, s->partial, s->nblk, m, s->st, 1, 1);
    begin_cycle_kernel<<<1, 256, 0, st>>>(s->partial, s->nblk, m, R, s->tol, s->max_iters, s->bnorm, s->relres, s->g,
                                          s->H, s->hbuf, 0, s->st);
    scale_v0_kernel<<<vg, 256, 0, st>>>(s->V, s->Vcur, n, R, m, s->hbuf, s->st);
    count_launches(3);   // residual, dots, begin_cycle (+ scale below)
    IE_CK_LAUNCH();
    return IE_OK;
}

int64_t count_kernel_nodes(cudaGraph_t graph) {
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) != cudaSuccess) return 0;
    int64_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}

// One restart cycle as a graph: a WHILE node whose body is one Arnoldi iteration
// (the Givens kernel sets the condition from the per-RHS flags), then the end of
// the cycle.  Skipped iterations cost nothing and the cycle needs no host sync.
ie_status build_while_graph(ie_solver s, cudaGraph_t *out) {
    cudaGraph_t g = nullptr;
    IE_CK(cudaGraphCreate(&g, 0));
    auto fail = [&](cudaError_t e, const char *what) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        set_error("%s: %s", what, cudaGetErrorString(e));
        return IE_ERR_CUDA;
    };
    cudaError_t e = cudaGraphConditionalHandleCreate(&s->hcond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = s->hcond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) return fail(e, "cudaGraphAddNode(while)");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(e, "capture body");
    capture_begin();
    ie_status st1 = enqueue_iteration(s, s->cap, kDevJ);
    capture_end();
    cudaGraph_t tmp = nullptr;
    e = cudaStreamEndCapture(s->cap, &tmp);
    if (st1 != IE_OK) {
        cudaGraphDestroy(g);
        return st1;
    }
    if (e != cudaSuccess) return fail(e, "end capture body");
    s->body_kernels = count_kernel_nodes(body);
    e = cudaStreamBeginCaptureToGraph(s->cap, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(e, "capture end");
    capture_begin();
    ie_status st2 = enqueue_end(s, s->cap);
    capture_end();
    e = cudaStreamEndCapture(s->cap, &tmp);
    if (st2 != IE_OK) {
        cudaGraphDestroy(g);
        return st2;
    }
    if (e != cudaSuccess) return fail(e, "end capture end");
    s->end_kernels = count_kernel_nodes(g);
    *out = g;
    return IE_OK;
}

// Fallback: the m iterations unrolled with explicit indices (every kernel gated).
ie_status build_unrolled_graph(ie_solver s, cudaGraph_t *out) {
    s->hcond = 0;
    IE_CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    capture_begin();
    ie_status e = IE_OK;
    for (int j = 0; j < s->m && e == IE_OK; ++j) e = enqueue_iteration(s, s->cap, j);
    if (e == IE_OK) e = enqueue_end(s, s->cap);
    capture_end();
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s->cap, &graph);
    if (e != IE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return e;
    }
    IE_CK(ce);
    s->body_kernels = 0;
    s->end_kernels = count_kernel_nodes(graph);
    *out = graph;
    return IE_OK;
}

ie_status read_info(ie_solver s, ie_solve_info *info, int *done) {
    int R = s->R;
    std::vector<int> st(4 + 4 * R);
    std::vector<double> rel(R);
    IE_CK(cudaMemcpy(st.data(), s->st, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
    IE_CK(cudaMemcpy(rel.data(), s->relres, R * sizeof(double), cudaMemcpyDeviceToHost));
    if (done) *done = st[1] == 0;
    if (info) {
        int it = 0;
        double rr = 0;
        bool conv = true;
        for (int r = 0; r < R; ++r) {
            it = std::max(it, st[2 + 3 * R + r]);
            rr = std::max(rr, rel[r]);
            if (rel[r] > s->tol) conv = false;
        }
        info->iterations = it;
        info->relres = rr;
        info->converged = conv ? 1 : 0;
        // products: one per WHILE-body run (or m per unrolled cycle) plus one restart per cycle
        int64_t body = st[3 + 4 * R];
        info->matvecs = (int)(s->use_while ? body + s->cycles_run : (int64_t)s->cycles_run * s->matvecs_per_cycle);
        if (s->use_while && body > s->body_runs_seen) {
            count_launches((body - s->body_runs_seen) * s->body_kernels);
            s->body_runs_seen = body;
        }
    }
    return IE_OK;
}

}  // namespace

extern "C" {

void ie_solve_opts_default(ie_solve_opts *o) {
    if (o) fill_defaults(o);
}

ie_status ie_solver_footprint(ie_plan p, int nrhs, const ie_solve_opts *opts, size_t *bytes) {
    if (!p || !bytes) return set_error("null argument"), IE_ERR_INVALID;
    ie_solve_opts o;
    fill_defaults(&o);
    if (opts) o = *opts;
    *bytes = solver_bytes(p->n, nrhs, o.restart);
    return IE_OK;
}

ie_status ie_solver_create(ie_plan p, int nrhs, const ie_solve_opts *opts, ie_solver *out) {
    if (!p || !out) return set_error("null argument"), IE_ERR_INVALID;
    *out = nullptr;
    ie_solve_opts o;
    fill_defaults(&o);
    if (opts) o = *opts;
    if (nrhs < 1 || nrhs > p->max_rhs || nrhs > 64) return set_error("bad nrhs %d", nrhs), IE_ERR_INVALID;
    if (o.restart < 1 || o.restart > 64) return set_error("restart must be in [1, 64]"), IE_ERR_INVALID;
    if (o.refine) return set_error("solver objects do not refine; use ie_solve"), IE_ERR_INVALID;
    if (!(p->prec_mask & IE_PRECMASK(o.prec))) return set_error("precision not in plan"), IE_ERR_UNSUPPORTED;
    ie_solver s = new ie_solver_s();
    auto fail = [&](ie_status st) {
        ie_solver_destroy(s);
        return st;
    };
    s->plan = p;
    s->R = nrhs;
    s->m = o.restart;
    s->max_iters = o.max_iters;
    s->tol = o.tol;
    s->prec = o.prec;
    s->n = p->n;
    s->nblk = (int)((p->n + kChunk - 1) / kChunk);
    int R = nrhs, m = o.restart;
    ie_status e;
#define SA(ptr, cnt)                                   \
    do {                                               \
        e = salloc_t(s, &(ptr), (size_t)(cnt));        \
        if (e != IE_OK) return fail(e);                \
    } while (0)
    SA(s->V, (size_t)(m + 1) * R * s->n);
    SA(s->W, (size_t)R * s->n);
    SA(s->H, (size_t)R * m * (m + 1));
    SA(s->cs, (size_t)R * m);
    SA(s->sn, (size_t)R * m);
    SA(s->g, (size_t)R * (m + 1));
    SA(s->hbuf, (size_t)R * (m + 1));
    SA(s->partial, (size_t)R * (m + 1) * s->nblk);
    SA(s->bnorm, R);
    SA(s->relres, R);
    SA(s->st, 4 + 4 * R);
    SA(s->Vcur, (size_t)R * s->n);
#undef SA
    if (cudaMemset(s->st, 0, (4 + 4 * R) * sizeof(int)) != cudaSuccess) return fail(IE_ERR_CUDA);
    // work lists must exist before graph capture (they allocate)
    WorkList *wl = nullptr;
    e = work_list(p, o.prec != IE_PREC_FP32, R, &wl);
    if (e != IE_OK) return fail(e);
    if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
        set_error("stream/event creation failed");
        return fail(IE_ERR_CUDA);
    }
    s->matvecs_per_cycle = m + 1;
    *out = s;
    return IE_OK;
}

ie_status ie_solver_destroy(ie_solver s) {
    if (!s) return IE_OK;
    cudaDeviceSynchronize();
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->ev) cudaEventDestroy(s->ev);
    for (void *q : s->allocs) cudaFree(q);
    delete s;
    return IE_OK;
}

ie_status ie_solver_start(ie_solver s, const void *v, void *c, void *stream) {
    if (!s || !v || !c) return set_error("null argument"), IE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    s->v = (const float2 *)v;
    s->x = (float2 *)c;
    s->cycles_run = 0;
    int R = s->R, m = s->m;
    int64_t n = s->n;
    IE_CK(cudaMemsetAsync(s->st, 0, (4 + 4 * R) * sizeof(int), st));
    s->body_runs_seen = 0;
    IE_CK(cudaMemsetAsync(s->x, 0, (size_t)R * n * sizeof(float2), st));
    dim3 vg(vec_grid(n), R), dg(s->nblk, R);
    residual_kernel<<<vg, 256, 0, st>>>(s->v, nullptr, s->V, n, R, 1, s->st);
    dots_kernel<<<dg, kDotThreads, 0, st>>>(s->V, s->V, n, R, 0, s->partial, s->nblk, m, s->st, 1, 1);
    begin_cycle_kernel<<<1, 256, 0, st>>>(s->partial, s->nblk, m, R, s->tol, s->max_iters, s->bnorm, s->relres, s->g,
                                          s->H, s->hbuf, 1, s->st);
    scale_v0_kernel<<<vg, 256, 0, st>>>(s->V, s->Vcur, n, R, m, s->hbuf, s->st);
    count_launches(3);
    IE_CK_LAUNCH();
    // the captured cycle reads v and x through fixed pointers: recapture if they moved
    if (s->exec && (s->cap_v != s->v || s->cap_x != s->x)) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    return IE_OK;
}

ie_status ie_solver_advance(ie_solver s, int cycles, void *stream) {
    if (!s || cycles < 0) return set_error("bad argument"), IE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < cycles; ++c) {
        if (!s->exec) {
            // build the cycle graph on the private stream, ordered after `st`
            IE_CK(cudaEventRecord(s->ev, st));
            IE_CK(cudaStreamWaitEvent(s->cap, s->ev, 0));
            cudaGraph_t graph = nullptr;
            s->use_while = build_while_graph(s, &graph) == IE_OK;
            if (!s->use_while) IE_TRY(build_unrolled_graph(s, &graph));
            cudaError_t ie_ = cudaGraphInstantiate(&s->exec, graph, 0);
            cudaGraphDestroy(graph);
            IE_CK(ie_);
            s->cap_v = s->v;
            s->cap_x = s->x;
        }
        IE_CK(cudaGraphLaunch(s->exec, st));
        count_launches(s->end_kernels);
        s->cycles_run++;
    }
    IE_CK(cudaEventRecord(s->ev, st));
    return IE_OK;
}

ie_status ie_solver_poll(ie_solver s, int *done, ie_solve_info *info) {
    if (!s || !done) return set_error("null argument"), IE_ERR_INVALID;
    cudaError_t q = cudaEventQuery(s->ev);
    if (q == cudaErrorNotReady) {
        *done = 0;
        return IE_OK;
    }
    IE_CK(q);
    return read_info(s, info, done);
}

ie_status ie_solve(ie_plan p, const void *v, void *c, int nrhs, const ie_solve_opts *opts, ie_solve_info *info,
                   void *stream) {
    auto t0 = std::chrono::steady_clock::now();
    if (!p || !v || !c) return set_error("null argument"), IE_ERR_INVALID;
    ie_solve_opts o;
    fill_defaults(&o);
    if (opts) o = *opts;
    cudaStream_t st = (cudaStream_t)stream;
    ie_solve_info inf{};
    ie_status result = IE_OK;
    if (!o.refine) {
        ie_solver s = nullptr;
        IE_TRY(cached_solver(p, nrhs, o, &s));
        ie_status e = ie_solver_start(s, v, c, stream);
        int done = 0;
        int max_cycles = (o.max_iters + o.restart - 1) / o.restart + 2;
        for (int cyc = 0; e == IE_OK && !done && cyc < max_cycles; ++cyc) {
            e = ie_solver_advance(s, 1, stream);
            if (e == IE_OK && cudaStreamSynchronize(st) != cudaSuccess) e = IE_ERR_CUDA;
            if (e == IE_OK) e = read_info(s, &inf, &done);
        }
        if (e == IE_OK) e = read_info(s, &inf, &done);
        if (e != IE_OK) return e;
        result = inf.converged ? IE_OK : IE_ERR_NOT_CONVERGED;
    } else {
        // outer refinement: x64 += GMRES_prec(r), r = v - Z_refine(x) in FP64
        if (!(p->prec_mask & IE_PRECMASK(o.refine_prec)) || !(p->prec_mask & IE_PRECMASK(o.prec)))
            return set_error("refinement precisions not in plan"), IE_ERR_UNSUPPORTED;
        int64_t n = p->n;
        int64_t total = (int64_t)nrhs * n;
        int nblk = (int)((n + kChunk - 1) / kChunk);
        double2 *x64 = nullptr, *part = nullptr;
        float2 *rv = nullptr, *d = nullptr, *Wz = nullptr;
        IE_CK(cudaMallocAsync(&x64, total * sizeof(double2), st));
        IE_CK(cudaMallocAsync(&rv, total * sizeof(float2), st));
        IE_CK(cudaMallocAsync(&d, total * sizeof(float2), st));
        IE_CK(cudaMallocAsync(&Wz, total * sizeof(float2), st));
        IE_CK(cudaMallocAsync(&part, (size_t)nrhs * nblk * sizeof(double2), st));
        ref_accumulate_kernel<<<vec_grid(total), 256, 0, st>>>(x64, nullptr, (float2 *)c, total, 1);
        count_launches(1);
        ie_solve_opts io = o;
        io.refine = 0;
        io.tol = o.inner_tol;
        ie_solver s = nullptr;
        ie_status e = cached_solver(p, nrhs, io, &s);
        std::vector<double2> hp((size_t)nrhs * nblk);
        int outer = 0, inner_iters = 0, mv = 0;
        double worst = 1;
        while (e == IE_OK) {
            // r = v - Z x  (FP64 difference of the FP32 product)
            e = apply(p, IE_FULL, o.refine_prec, (const float2 *)c, Wz, nrhs, st);
            mv++;
            if (e != IE_OK) break;
            ref_residual_kernel<<<dim3(nblk, nrhs), kDotThreads, 0, st>>>((const float2 *)v, Wz, rv, n, part, nblk);
            count_launches(1);
            if (cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                e = IE_ERR_CUDA;
                break;
            }
            worst = 0;
            for (int r = 0; r < nrhs; ++r) {
                double rs = 0, vs = 0;
                for (int b = 0; b < nblk; ++b) rs += hp[(size_t)r * nblk + b].x, vs += hp[(size_t)r * nblk + b].y;
                double rel = vs > 0 ? std::sqrt(rs / vs) : 0;
                worst = std::max(worst, rel);
            }
            if (worst <= o.tol || outer >= o.max_refine || inner_iters >= o.max_iters) break;
            // inner solve Z d = r
            e = ie_solver_start(s, rv, d, stream);
            int done = 0;
            ie_solve_info ii{};
            int max_cycles = (o.max_iters + o.restart - 1) / o.restart + 2;
            for (int cyc = 0; e == IE_OK && !done && cyc < max_cycles; ++cyc) {
                e = ie_solver_advance(s, 1, stream);
                if (e == IE_OK && cudaStreamSynchronize(st) != cudaSuccess) e = IE_ERR_CUDA;
                if (e == IE_OK) e = read_info(s, &ii, &done);
            }
            if (e != IE_OK) break;
            inner_iters += ii.iterations;
            mv += ii.matvecs;
            ref_accumulate_kernel<<<vec_grid(total), 256, 0, st>>>(x64, d, (float2 *)c, total, 0);
            count_launches(1);
            outer++;
        }
        cudaFreeAsync(x64, st);
        cudaFreeAsync(rv, st);
        cudaFreeAsync(d, st);
        cudaFreeAsync(Wz, st);
        cudaFreeAsync(part, st);
        cudaStreamSynchronize(st);
        if (e != IE_OK) return e;
        inf.iterations = inner_iters;
        inf.matvecs = mv;
        inf.refinements = outer;
        inf.relres = worst;
        inf.converged = worst <= o.tol;
        result = inf.converged ? IE_OK : IE_ERR_NOT_CONVERGED;
    }
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return result;
}

}  // extern "C"
