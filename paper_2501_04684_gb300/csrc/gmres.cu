// K6 / K8: restarted GMRES without preconditioning (§5, the paper's iterative
// solver) with device-resident state, and outer iterative refinement.
//
// Systems: every (right-hand side, scatterer) pair is an independent GMRES(m) run
// (x0 = 0) over its scatterer's slice of the packed vector [rhs][n]; a plan without
// scatterer groups has one system per right-hand side.  Arnoldi uses classical
// Gram-Schmidt applied twice (dot products accumulated in FP64), Givens rotations and
// the small least-squares solve run in FP64; Krylov vectors are FP32.  Vector kernels
// walk chunks of 1,024 unknowns that never straddle two scatterers.
//
// One restart cycle is one CUDA graph: a WHILE node runs one Arnoldi iteration per
// body launch (the iteration index lives in device memory and the Givens kernel sets
// the condition from the per-system flags), followed by the solution update and the
// restart residual.  The host synchronises once per cycle.
#include <chrono>
#include <cmath>
#include <cstdio>

#include "ie_internal.h"

struct ie_solver_s {
    ie_plan plan = nullptr;
    int R = 1, G = 1, S = 1, m = 50, max_iters = 1000, prec = IE_PREC_FP32;
    double tol = 1e-6;
    int64_t n = 0;
    int C = 1, nblk = 1;                 // chunks per column, max chunks of one scatterer
    int32_t *chunk_group = nullptr;      // [C]
    int64_t *chunk_start = nullptr;      // [C] first unknown of the chunk
    int32_t *chunk_local = nullptr;      // [C] chunk index inside its scatterer
    int64_t *goff = nullptr;             // [G + 1] unknown offsets of the scatterers
    int32_t *nchunk = nullptr;           // [G]
    float2 *V = nullptr;                 // [(m+1)][R][n]
    float2 *W = nullptr;                 // [R][n]
    float2 *Vcur = nullptr;              // [R][n] current Krylov vector (input of the product)
    double2 *H = nullptr;                // [S][m][m+1]
    double *cs = nullptr;                // [S][m]
    double2 *sn = nullptr;               // [S][m]
    double2 *g = nullptr;                // [S][m+1]
    double2 *hbuf = nullptr;             // [S][m+1]
    double2 *partial = nullptr;          // [S][m+1][nblk]
    double *bnorm = nullptr;             // [S]
    double *relres = nullptr;            // [S]
    int *st = nullptr;                   // [4 + 4S], layout below
    cudaGraphConditionalHandle hcond = 0;
    bool use_while = false;
    int64_t body_kernels = 0, end_kernels = 0, body_runs_seen = 0;
    const float2 *v = nullptr;
    float2 *x = nullptr;
    const float2 *cap_v = nullptr;       // pointers baked into the captured cycle
    float2 *cap_x = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev = nullptr;
    int matvecs_per_cycle = 0;
    int cycles_run = 0;
    int *h_st = nullptr;                 // pinned host mirror of st and relres, copied at the end of
    double *h_rel = nullptr;             // every start and advance (read by ie_solver_poll / _state)
    std::vector<void *> allocs;
    size_t bytes = 0;
};

namespace ie {
namespace {

constexpr int kDotThreads = 256;
constexpr int kEPT = 4;                        // unknowns per thread in the vector kernels
constexpr int kChunk = kDotThreads * kEPT;     // unknowns per chunk (one block)
constexpr int kMaxSystems = 1024;
constexpr int kSysThreads = 256;               // threads of the single-block per-system kernels

// st layout: [0] any system active in this cycle, [1] any system not finished, then
// done[S], active[S], jend[S], iters[S], the cycle's Arnoldi index, WHILE-body runs.
__device__ inline int *st_done(int *st, int S) { return st + 2; }
__device__ inline int *st_active(int *st, int S) { return st + 2 + S; }
__device__ inline int *st_jend(int *st, int S) { return st + 2 + 2 * S; }
__device__ inline int *st_iters(int *st, int S) { return st + 2 + 3 * S; }
__device__ inline int *st_jdev(int *st, int S) { return st + 2 + 4 * S; }
__device__ inline int *st_body(int *st, int S) { return st + 3 + 4 * S; }

// j >= 0: index given by the launch; kDevJ: read the cycle's index from device memory.
constexpr int kDevJ = -2;
__device__ inline int resolve_j(int j, int *st, int S) { return j >= 0 ? j : *st_jdev(st, S); }

// Segmented layout of the packed vector.
struct Seg {
    const int32_t *chunk_group;
    const int64_t *chunk_start;
    const int32_t *chunk_local;
    const int64_t *goff;
    const int32_t *nchunk;
    int G;
    int64_t n;
};

// The system of chunk c in column r, the chunk's unknown range [e0, e1) and its
// index inside the scatterer.
__device__ inline int chunk_system(const Seg &sg, int c, int r, int64_t &e0, int64_t &e1, int &local) {
    const int g = sg.chunk_group[c];
    e0 = sg.chunk_start[c];
    e1 = min(e0 + (int64_t)kChunk, sg.goff[g + 1]);
    local = sg.chunk_local[c];
    return r * sg.G + g;
}

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

// partial[s][i][local] = the chunk's sum of conj(V_i) . W, i <= j; norm = 1:
// partial[s][0][local] = the chunk's sum of |W|^2.  Only systems with active[s] (or
// not done[s] when use_done) take part.
__global__ void dots_kernel(const float2 *__restrict__ V, const float2 *__restrict__ Wv, Seg sg, int R, int S,
                            int jarg, double2 *__restrict__ partial, int nblk, int m, int *st, int use_done,
                            int norm) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    const bool on = use_done ? !st_done(st, S)[s] : st_active(st, S)[s];
    if (!on) return;
    const int64_t n = sg.n;
    float2 w[kEPT];
    const float2 *wr = Wv + (int64_t)r * n;
#pragma unroll
    for (int t = 0; t < kEPT; ++t) {
        int64_t e = e0 + threadIdx.x + t * kDotThreads;
        w[t] = e < e1 ? wr[e] : make_float2(0.f, 0.f);
    }
    double2 *pr = partial + ((int64_t)s * (m + 1)) * nblk;
    if (norm) {
        double q = 0;
#pragma unroll
        for (int t = 0; t < kEPT; ++t) q += (double)w[t].x * w[t].x + (double)w[t].y * w[t].y;
        double2 tot = block_sum2(make_double2(q, 0));
        if (threadIdx.x == 0) pr[local] = tot;
        return;
    }
    const int j = resolve_j(jarg, st, S);
    for (int i = 0; i <= j; ++i) {
        const float2 *vi = V + ((int64_t)i * R + r) * n;
        double sr = 0, si = 0;
#pragma unroll
        for (int t = 0; t < kEPT; ++t) {
            int64_t e = e0 + threadIdx.x + t * kDotThreads;
            float2 a = e < e1 ? vi[e] : make_float2(0.f, 0.f);
            sr += (double)a.x * w[t].x + (double)a.y * w[t].y;      // conj(a) * w
            si += (double)a.x * w[t].y - (double)a.y * w[t].x;
        }
        double2 tot = block_sum2(make_double2(sr, si));
        if (threadIdx.x == 0) pr[(int64_t)i * nblk + local] = tot;
    }
}

// hbuf[s][i] = sum over the system's chunks; column j of H gets hbuf (first
// Gram-Schmidt pass, add = 0) or hbuf added (second pass).
__global__ void reduce_dots_kernel(const double2 *__restrict__ partial, const int32_t *__restrict__ nchunk, int G,
                                   int nblk, int m, int S, int jarg, int add, double2 *__restrict__ hbuf,
                                   double2 *__restrict__ H, int *st) {
    const int s = blockIdx.x;
    if (!st_active(st, S)[s]) return;
    const int j = resolve_j(jarg, st, S);
    const int nb = nchunk[s % G];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 *p = partial + ((int64_t)s * (m + 1) + i) * nblk;
        double sx = 0, sy = 0;
        for (int b = 0; b < nb; ++b) sx += p[b].x, sy += p[b].y;
        hbuf[(int64_t)s * (m + 1) + i] = make_double2(sx, sy);
        double2 &h = H[((int64_t)s * m + j) * (m + 1) + i];
        if (add) {
            h.x += sx;
            h.y += sy;
        } else {
            h = make_double2(sx, sy);
        }
    }
}

// W -= sum_{i<=j} V_i hbuf[s][i] over the chunk's unknowns
__global__ void update_kernel(const float2 *__restrict__ V, float2 *__restrict__ Wv, Seg sg, int R, int S, int jarg,
                              int m, const double2 *__restrict__ hbuf, int *st) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    if (!st_active(st, S)[s]) return;
    const int j = resolve_j(jarg, st, S);
    __shared__ float2 h[65];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        double2 v = hbuf[(int64_t)s * (m + 1) + i];
        h[i] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    const int64_t n = sg.n;
    float2 *wr = Wv + (int64_t)r * n;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 w = wr[e];
        for (int i = 0; i <= j; ++i) {
            float2 a = V[((int64_t)i * R + r) * n + e];
            w.x -= a.x * h[i].x - a.y * h[i].y;
            w.y -= a.x * h[i].y + a.y * h[i].x;
        }
        wr[e] = w;
    }
}

// ||W_s|| -> H[s][j][j+1] and hbuf[s][0] (read by the scaling kernel).
__global__ void norm_finish_kernel(const double2 *__restrict__ partial, const int32_t *__restrict__ nchunk, int G,
                                   int nblk, int m, int S, int jarg, double2 *__restrict__ hbuf,
                                   double2 *__restrict__ H, int *st) {
    const int s = blockIdx.x;
    if (!st_active(st, S)[s] || threadIdx.x != 0) return;
    const int j = resolve_j(jarg, st, S);
    const double2 *p = partial + ((int64_t)s * (m + 1)) * nblk;
    double q = 0;
    for (int b = 0; b < nchunk[s % G]; ++b) q += p[b].x;
    const double hn = sqrt(q);
    H[((int64_t)s * m + j) * (m + 1) + j + 1] = make_double2(hn, 0);
    hbuf[(int64_t)s * (m + 1)] = make_double2(hn, 0);
}

// V_{j+1} = W / hn over the chunk, also written to Vcur (the next product's input)
__global__ void scale_kernel(const float2 *__restrict__ Wv, float2 *__restrict__ V, float2 *__restrict__ Vcur, Seg sg,
                             int R, int S, int m, const double2 *__restrict__ hbuf, int *st, int jarg) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    if (!st_active(st, S)[s]) return;
    const int j = resolve_j(jarg, st, S);
    const double hn = hbuf[(int64_t)s * (m + 1)].x;
    const float q = hn > 0 ? (float)(1.0 / hn) : 0.f;
    const int64_t n = sg.n;
    const float2 *wr = Wv + (int64_t)r * n;
    float2 *vr = V + ((int64_t)(j + 1) * R + r) * n;
    float2 *cr = Vcur + (int64_t)r * n;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 w = wr[e];
        float2 o = make_float2(w.x * q, w.y * q);
        vr[e] = o;
        cr[e] = o;
    }
}

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double cabs2(double2 a) { return sqrt(a.x * a.x + a.y * a.y); }

// Givens update of column j, residual estimate and termination of every active
// system; one block, threads over systems.  In the WHILE body it also advances the
// iteration index and sets the loop condition.
__global__ void givens_kernel(double2 *__restrict__ H, double *__restrict__ cs, double2 *__restrict__ sn,
                              double2 *__restrict__ g, const double *__restrict__ bnorm, double *__restrict__ relres,
                              int m, int S, int jarg, double tol, int max_iters, int *st,
                              cudaGraphConditionalHandle cond) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const int j = resolve_j(jarg, st, S);
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        if (!st_active(st, S)[s]) continue;
        double2 *h = H + ((int64_t)s * m + j) * (m + 1);
        double *c = cs + (int64_t)s * m;
        double2 *sv = sn + (int64_t)s * m;
        double2 *gr = g + (int64_t)s * (m + 1);
        for (int i = 0; i < j; ++i) {
            double2 a = h[i], b = h[i + 1];
            double2 sb = cmul(sv[i], b);
            double2 u = cmul(conj2(sv[i]), a);
            h[i] = make_double2(c[i] * a.x + sb.x, c[i] * a.y + sb.y);
            h[i + 1] = make_double2(-u.x + c[i] * b.x, -u.y + c[i] * b.y);
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
        sv[j] = sj;
        double2 sb = cmul(sj, b);
        h[j] = make_double2(cj * a.x + sb.x, cj * a.y + sb.y);
        h[j + 1] = make_double2(0, 0);
        double2 gj = gr[j];
        double2 gn = cmul(conj2(sj), gj);
        gr[j + 1] = make_double2(-gn.x, -gn.y);
        gr[j] = make_double2(cj * gj.x, cj * gj.y);
        int it = ++st_iters(st, S)[s];
        st_jend(st, S)[s] = j + 1;
        double res = cabs2(gr[j + 1]) / bnorm[s];
        relres[s] = res;
        bool breakdown = nb == 0;
        if (res <= tol || it >= max_iters || breakdown || j + 1 == m)
            st_active(st, S)[s] = 0;
        else
            atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st[0] = any;
        if (jarg == kDevJ) {
            *st_jdev(st, S) = j + 1;
            *st_body(st, S) += 1;
            cudaGraphSetConditional(cond, any ? 1u : 0u);   // WHILE node: run the next iteration?
        }
    }
}

// Back substitution H[0:jend,0:jend] y = g[0:jend] per system; y stored in hbuf[s].
__global__ void lsq_kernel(const double2 *__restrict__ H, const double2 *__restrict__ g, double2 *__restrict__ y,
                           int m, int S, int *st) {
    for (int s = threadIdx.x + blockIdx.x * blockDim.x; s < S; s += blockDim.x * gridDim.x) {
        const int je = st_jend(st, S)[s];
        double2 *ys = y + (int64_t)s * (m + 1);
        for (int i = je - 1; i >= 0; --i) {
            double2 q = g[(int64_t)s * (m + 1) + i];
            for (int k = i + 1; k < je; ++k) {
                double2 t = cmul(H[((int64_t)s * m + k) * (m + 1) + i], ys[k]);
                q.x -= t.x, q.y -= t.y;
            }
            double2 d = H[((int64_t)s * m + i) * (m + 1) + i];
            double dd = d.x * d.x + d.y * d.y;
            ys[i] = dd > 0 ? make_double2((q.x * d.x + q.y * d.y) / dd, (q.y * d.x - q.x * d.y) / dd)
                           : make_double2(0, 0);
        }
    }
}

// x += sum_{i<jend} V_i y[s][i] over the chunk
__global__ void xupdate_kernel(const float2 *__restrict__ V, float2 *__restrict__ x, Seg sg, int R, int S, int m,
                               const double2 *__restrict__ y, int *st) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    const int je = st_jend(st, S)[s];
    if (je == 0) return;
    __shared__ float2 ys[65];
    for (int i = threadIdx.x; i < je; i += blockDim.x) {
        double2 v = y[(int64_t)s * (m + 1) + i];
        ys[i] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    const int64_t n = sg.n;
    float2 *xr = x + (int64_t)r * n;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 acc = xr[e];
        for (int i = 0; i < je; ++i) {
            float2 a = V[((int64_t)i * R + r) * n + e];
            acc.x += a.x * ys[i].x - a.y * ys[i].y;
            acc.y += a.x * ys[i].y + a.y * ys[i].x;
        }
        xr[e] = acc;
    }
}

// V_0 = v - W over the chunk for systems not done (W = Z x); copy = 1: V_0 = v.
__global__ void residual_kernel(const float2 *__restrict__ v, const float2 *__restrict__ Wv, float2 *__restrict__ V0,
                                Seg sg, int S, int copy, int *st) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    if (st_done(st, S)[s]) return;
    const int64_t n = sg.n;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
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

// Begin a cycle from V_0 = residual: beta = ||V_0||, termination tests, g reset.
// start = 1: also sets bnorm = beta (x0 = 0) and clears the counters.  One block.
__global__ void begin_cycle_kernel(const double2 *__restrict__ partial, const int32_t *__restrict__ nchunk, int G,
                                   int nblk, int m, int S, double tol, int max_iters, double *__restrict__ bnorm,
                                   double *__restrict__ relres, double2 *__restrict__ g, double2 *__restrict__ hbuf,
                                   int start, int *st) {
    __shared__ int any_active;
    if (threadIdx.x == 0) any_active = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        if (start) {
            st_done(st, S)[s] = 0;
            st_iters(st, S)[s] = 0;
        }
        st_jend(st, S)[s] = 0;
        st_active(st, S)[s] = 0;
        if (st_done(st, S)[s]) continue;
        const double2 *p = partial + ((int64_t)s * (m + 1)) * nblk;
        double q = 0;
        for (int b = 0; b < nchunk[s % G]; ++b) q += p[b].x;
        const double beta = sqrt(q);
        if (start) bnorm[s] = beta;
        const double rel = bnorm[s] > 0 ? beta / bnorm[s] : 0.0;
        relres[s] = rel;
        if (bnorm[s] == 0 || rel <= tol || st_iters(st, S)[s] >= max_iters) {
            st_done(st, S)[s] = 1;
            continue;
        }
        st_active(st, S)[s] = 1;
        double2 *gr = g + (int64_t)s * (m + 1);
        gr[0] = make_double2(beta, 0);
        for (int i = 1; i <= m; ++i) gr[i] = make_double2(0, 0);
        hbuf[(int64_t)s * (m + 1)] = make_double2(beta, 0);
        atomicOr(&any_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st[0] = any_active;
        st[1] = any_active;   // a system not done is active at the start of a cycle
        *st_jdev(st, S) = 0;
    }
}

// V_0 /= beta (hbuf[s][0]) over the chunk for active systems, also into Vcur.
__global__ void scale_v0_kernel(float2 *__restrict__ V0, float2 *__restrict__ Vcur, Seg sg, int S, int m,
                                const double2 *__restrict__ hbuf, int *st) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    if (!st_active(st, S)[s]) return;
    const float q = (float)(1.0 / hbuf[(int64_t)s * (m + 1)].x);
    const int64_t n = sg.n;
    float2 *vr = V0 + (int64_t)r * n;
    float2 *cr = Vcur + (int64_t)r * n;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 a = vr[e];
        float2 o = make_float2(a.x * q, a.y * q);
        vr[e] = o;
        cr[e] = o;
    }
}

// ---- refinement helpers (FP64 outer loop) ----
// r = v - W in FP64 over the chunk; partial[s][local] = (||r||^2, ||v||^2).
__global__ void ref_residual_kernel(const float2 *__restrict__ v, const float2 *__restrict__ Wv,
                                    float2 *__restrict__ rout, Seg sg, int nblk, double2 *__restrict__ partial) {
    const int r = blockIdx.y;
    int64_t e0, e1;
    int local;
    const int s = chunk_system(sg, blockIdx.x, r, e0, e1, local);
    double q = 0, qv = 0;
    const int64_t n = sg.n;
#pragma unroll
    for (int t = 0; t < kEPT; ++t) {
        int64_t e = e0 + threadIdx.x + t * kDotThreads;
        if (e >= e1) continue;
        int64_t i = (int64_t)r * n + e;
        float2 a = v[i], b = Wv ? Wv[i] : make_float2(0.f, 0.f);
        double rx = (double)a.x - (double)b.x, ry = (double)a.y - (double)b.y;
        rout[i] = make_float2((float)rx, (float)ry);
        q += rx * rx + ry * ry;
        qv += (double)a.x * a.x + (double)a.y * a.y;
    }
    double2 tot = block_sum2(make_double2(q, qv));
    if (threadIdx.x == 0) partial[(int64_t)s * nblk + local] = tot;
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
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 1024));
}

// The chunks of every scatterer's slice (host side).
struct Chunks {
    std::vector<int32_t> group, local, nchunk;
    std::vector<int64_t> start;
    int nblk = 1;
};

Chunks make_chunks(const ie_plan p) {
    Chunks c;
    c.nchunk.assign(p->ngroups, 0);
    for (int g = 0; g < p->ngroups; ++g) {
        const int64_t a = p->goff[g], b = p->goff[g + 1];
        int k = 0;
        for (int64_t e = a; e < b; e += kChunk, ++k) {
            c.group.push_back(g);
            c.start.push_back(e);
            c.local.push_back(k);
        }
        c.nchunk[g] = k;
        c.nblk = std::max(c.nblk, k);
    }
    if (c.group.empty()) {      // no unknowns at all: one empty chunk keeps the grids non-empty
        c.group.push_back(0);
        c.start.push_back(0);
        c.local.push_back(0);
    }
    return c;
}

Seg seg_of(const ie_solver s) {
    return Seg{s->chunk_group, s->chunk_start, s->chunk_local, s->goff, s->nchunk, s->G, s->n};
}

}  // namespace

void destroy_cached_solvers(ie_plan p) {
    for (auto &kv : p->solvers) ie_solver_destroy(kv.second);
    p->solvers.clear();
}

}  // namespace ie

using namespace ie;

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

size_t solver_bytes(int64_t n, int R, int G, int m, int C, int nblk) {
    const int64_t S = (int64_t)R * G;
    size_t b = 0;
    b += (size_t)(m + 1) * R * n * sizeof(float2);           // V
    b += (size_t)2 * R * n * sizeof(float2);                 // W, Vcur
    b += (size_t)S * m * (m + 1) * sizeof(double2);          // H
    b += (size_t)S * m * (sizeof(double) + sizeof(double2)); // cs, sn
    b += (size_t)S * (m + 1) * sizeof(double2) * 2;          // g, hbuf
    b += (size_t)S * (m + 1) * nblk * sizeof(double2);       // partial
    b += (size_t)S * 2 * sizeof(double) + (4 + 4 * S) * sizeof(int);
    b += (size_t)C * (2 * sizeof(int32_t) + sizeof(int64_t)) + (size_t)(G + 1) * sizeof(int64_t) + G * sizeof(int32_t);
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
    const int R = s->R, S = s->S, m = s->m, G = s->G;
    const Seg sg = seg_of(s);
    const dim3 cg(s->C, R);
    IE_TRY(apply(p, IE_FULL, s->prec, s->Vcur, s->W, R, st, s->st));
    for (int pass = 0; pass < 2; ++pass) {
        dots_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->W, sg, R, S, jarg, s->partial, s->nblk, m, s->st, 0, 0);
        reduce_dots_kernel<<<S, 64, 0, st>>>(s->partial, s->nchunk, G, s->nblk, m, S, jarg, pass, s->hbuf, s->H,
                                             s->st);
        update_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->W, sg, R, S, jarg, m, s->hbuf, s->st);
    }
    dots_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->W, sg, R, S, jarg, s->partial, s->nblk, m, s->st, 0, 1);
    norm_finish_kernel<<<S, 32, 0, st>>>(s->partial, s->nchunk, G, s->nblk, m, S, jarg, s->hbuf, s->H, s->st);
    scale_kernel<<<cg, kDotThreads, 0, st>>>(s->W, s->V, s->Vcur, sg, R, S, m, s->hbuf, s->st, jarg);
    givens_kernel<<<1, kSysThreads, 0, st>>>(s->H, s->cs, s->sn, s->g, s->bnorm, s->relres, m, S, jarg, s->tol,
                                             s->max_iters, s->st, s->hcond);
    count_launches(9);   // the ten kernels above (IE_CK_LAUNCH adds the last)
    IE_CK_LAUNCH();
    return IE_OK;
}

// Solution update x += V y and the restart: true residual, its norm, next cycle.
ie_status enqueue_end(ie_solver s, cudaStream_t st) {
    ie_plan p = s->plan;
    const int R = s->R, S = s->S, m = s->m, G = s->G;
    const Seg sg = seg_of(s);
    const dim3 cg(s->C, R);
    lsq_kernel<<<(S + 127) / 128, 128, 0, st>>>(s->H, s->g, s->hbuf, m, S, s->st);
    xupdate_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->x, sg, R, S, m, s->hbuf, s->st);
    count_launches(2);
    IE_TRY(apply(p, IE_FULL, s->prec, s->x, s->W, R, st, s->st + 1));
    residual_kernel<<<cg, kDotThreads, 0, st>>>(s->v, s->W, s->V, sg, S, 0, s->st);
    dots_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->V, sg, R, S, 0, s->partial, s->nblk, m, s->st, 1, 1);
    begin_cycle_kernel<<<1, kSysThreads, 0, st>>>(s->partial, s->nchunk, G, s->nblk, m, S, s->tol, s->max_iters,
                                                  s->bnorm, s->relres, s->g, s->hbuf, 0, s->st);
    scale_v0_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->Vcur, sg, S, m, s->hbuf, s->st);
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
// (the Givens kernel sets the condition from the per-system flags), then the end of
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
    const int S = s->S;
    std::vector<int> st(4 + 4 * S);
    std::vector<double> rel(S);
    IE_CK(cudaMemcpy(st.data(), s->st, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
    IE_CK(cudaMemcpy(rel.data(), s->relres, S * sizeof(double), cudaMemcpyDeviceToHost));
    if (done) *done = st[1] == 0;
    if (info) {
        int it = 0;
        double rr = 0;
        bool conv = true;
        for (int q = 0; q < S; ++q) {
            it = std::max(it, st[2 + 3 * S + q]);
            rr = std::max(rr, rel[q]);
            if (rel[q] > s->tol) conv = false;
        }
        info->iterations = it;
        info->relres = rr;
        info->converged = conv ? 1 : 0;
        // products: one per WHILE-body run (or m per unrolled cycle) plus one restart per cycle
        int64_t body = st[3 + 4 * S];
        info->matvecs = (int)(s->use_while ? body + s->cycles_run : (int64_t)s->cycles_run * s->matvecs_per_cycle);
        if (s->use_while && body > s->body_runs_seen) {
            count_launches((body - s->body_runs_seen) * s->body_kernels);
            s->body_runs_seen = body;
        }
    }
    return IE_OK;
}

// The same from the pinned mirror (valid once the solver's event has completed).
void read_info_mirror(ie_solver s, ie_solve_info *info, int *done) {
    const int S = s->S;
    const int *st = s->h_st;
    if (done) *done = st[1] == 0;
    if (!info) return;
    int it = 0;
    double rr = 0;
    bool conv = true;
    for (int q = 0; q < S; ++q) {
        it = std::max(it, st[2 + 3 * S + q]);
        rr = std::max(rr, s->h_rel[q]);
        if (s->h_rel[q] > s->tol) conv = false;
    }
    info->iterations = it;
    info->relres = rr;
    info->converged = conv ? 1 : 0;
    const int64_t body = st[3 + 4 * S];
    info->matvecs = (int)(s->use_while ? body + s->cycles_run : (int64_t)s->cycles_run * s->matvecs_per_cycle);
    if (s->use_while && body > s->body_runs_seen) {
        count_launches((body - s->body_runs_seen) * s->body_kernels);
        s->body_runs_seen = body;
    }
}

// Enqueue the copy of the status into the pinned mirror and record the solver's event.
ie_status mirror_status(ie_solver s, cudaStream_t st) {
    IE_CK(cudaMemcpyAsync(s->h_st, s->st, (4 + 4 * s->S) * sizeof(int), cudaMemcpyDeviceToHost, st));
    IE_CK(cudaMemcpyAsync(s->h_rel, s->relres, s->S * sizeof(double), cudaMemcpyDeviceToHost, st));
    IE_CK(cudaEventRecord(s->ev, st));
    return IE_OK;
}

// Cycles until every system is done (or the cycle cap), synchronising once per cycle.
ie_status run_cycles(ie_solver s, const ie_solve_opts &o, void *stream, ie_solve_info *inf) {
    cudaStream_t st = (cudaStream_t)stream;
    int done = 0;
    const int max_cycles = (o.max_iters + o.restart - 1) / o.restart + 2;
    for (int cyc = 0; !done && cyc < max_cycles; ++cyc) {
        IE_TRY(ie_solver_advance(s, 1, stream));
        IE_CK(cudaStreamSynchronize(st));
        read_info_mirror(s, inf, &done);     // the advance copied the status to the host
    }
    return read_info(s, inf, &done);
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
    Chunks c = make_chunks(p);
    *bytes = solver_bytes(p->n, nrhs, p->ngroups, o.restart, (int)c.group.size(), c.nblk);
    return IE_OK;
}

ie_status ie_solver_create(ie_plan p, int nrhs, const ie_solve_opts *opts, ie_solver *out) {
    if (!p || !out) return set_error("null argument"), IE_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    *out = nullptr;
    ie_solve_opts o;
    fill_defaults(&o);
    if (opts) o = *opts;
    if (nrhs < 1 || nrhs > p->max_rhs || nrhs > 64) return set_error("bad nrhs %d", nrhs), IE_ERR_INVALID;
    if (o.restart < 1 || o.restart > 64) return set_error("restart must be in [1, 64]"), IE_ERR_INVALID;
    if (o.refine) return set_error("solver objects do not refine; use ie_solve"), IE_ERR_INVALID;
    if ((int64_t)nrhs * p->ngroups > kMaxSystems)
        return set_error("%d right-hand sides x %d scatterers exceed %d systems", nrhs, p->ngroups, kMaxSystems),
               IE_ERR_INVALID;
    if (!(p->prec_mask & IE_PRECMASK(o.prec))) return set_error("precision not in plan"), IE_ERR_UNSUPPORTED;
    ie_solver s = new ie_solver_s();
    auto fail = [&](ie_status st) {
        ie_solver_destroy(s);
        return st;
    };
    s->plan = p;
    s->R = nrhs;
    s->G = p->ngroups;
    s->S = nrhs * p->ngroups;
    s->m = o.restart;
    s->max_iters = o.max_iters;
    s->tol = o.tol;
    s->prec = o.prec;
    s->n = p->n;
    Chunks c = make_chunks(p);
    s->C = (int)c.group.size();
    s->nblk = c.nblk;
    const int R = nrhs, S = s->S, m = o.restart;
    ie_status e;
#define SA(ptr, cnt)                                   \
    do {                                               \
        e = salloc_t(s, &(ptr), (size_t)(cnt));        \
        if (e != IE_OK) return fail(e);                \
    } while (0)
    SA(s->chunk_group, s->C);
    SA(s->chunk_start, s->C);
    SA(s->chunk_local, s->C);
    SA(s->goff, s->G + 1);
    SA(s->nchunk, s->G);
    SA(s->V, (size_t)(m + 1) * R * s->n);
    SA(s->W, (size_t)R * s->n);
    SA(s->Vcur, (size_t)R * s->n);
    SA(s->H, (size_t)S * m * (m + 1));
    SA(s->cs, (size_t)S * m);
    SA(s->sn, (size_t)S * m);
    SA(s->g, (size_t)S * (m + 1));
    SA(s->hbuf, (size_t)S * (m + 1));
    SA(s->partial, (size_t)S * (m + 1) * s->nblk);
    SA(s->bnorm, S);
    SA(s->relres, S);
    SA(s->st, 4 + 4 * S);
#undef SA
    if (cudaMemcpy(s->chunk_group, c.group.data(), s->C * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->chunk_start, c.start.data(), s->C * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->chunk_local, c.local.data(), s->C * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->goff, p->goff.data(), (s->G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->nchunk, c.nchunk.data(), s->G * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->st, 0, (4 + 4 * S) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("solver set-up copies failed");
        return fail(IE_ERR_CUDA);
    }
    // work lists must exist before graph capture (they allocate)
    WorkList *wl = nullptr;
    e = work_list_for(p, o.prec, R, &wl);
    if (e != IE_OK) return fail(e);
    if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
        set_error("stream/event creation failed");
        return fail(IE_ERR_CUDA);
    }
    {
        void *h = nullptr;
        const size_t ib = ((4 + 4 * (size_t)S) * sizeof(int) + 7) / 8 * 8;
        if (cudaMallocHost(&h, ib + S * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_error("pinned status mirror allocation failed");
            return fail(IE_ERR_OOM);
        }
        s->h_st = static_cast<int *>(h);
        s->h_rel = reinterpret_cast<double *>(static_cast<char *>(h) + ib);
        std::fill(s->h_st, s->h_st + 4 + 4 * S, 0);
        std::fill(s->h_rel, s->h_rel + S, 0.0);
    }
    s->matvecs_per_cycle = m + 1;
    *out = s;
    return IE_OK;
}

ie_status ie_solver_destroy(ie_solver s) {
    if (!s) return IE_OK;
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    cudaDeviceSynchronize();
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->ev) cudaEventDestroy(s->ev);
    for (void *q : s->allocs) cudaFree(q);
    if (s->h_st) cudaFreeHost(s->h_st);
    delete s;
    return IE_OK;
}

ie_status ie_solver_start(ie_solver s, const void *v, void *c, void *stream) {
    if (!s || !v || !c) return set_error("null argument"), IE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    s->v = (const float2 *)v;
    s->x = (float2 *)c;
    s->cycles_run = 0;
    const int R = s->R, S = s->S, m = s->m;
    const Seg sg = seg_of(s);
    const dim3 cg(s->C, R);
    IE_CK(cudaMemsetAsync(s->st, 0, (4 + 4 * S) * sizeof(int), st));
    s->body_runs_seen = 0;
    IE_CK(cudaMemsetAsync(s->x, 0, (size_t)R * s->n * sizeof(float2), st));
    residual_kernel<<<cg, kDotThreads, 0, st>>>(s->v, nullptr, s->V, sg, S, 1, s->st);
    dots_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->V, sg, R, S, 0, s->partial, s->nblk, m, s->st, 1, 1);
    begin_cycle_kernel<<<1, kSysThreads, 0, st>>>(s->partial, s->nchunk, s->G, s->nblk, m, S, s->tol, s->max_iters,
                                                  s->bnorm, s->relres, s->g, s->hbuf, 1, s->st);
    scale_v0_kernel<<<cg, kDotThreads, 0, st>>>(s->V, s->Vcur, sg, S, m, s->hbuf, s->st);
    count_launches(3);
    IE_CK_LAUNCH();
    IE_TRY(mirror_status(s, st));
    // the captured cycle reads v and x through fixed pointers: recapture if they moved
    if (s->exec && (s->cap_v != s->v || s->cap_x != s->x)) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    return IE_OK;
}

ie_status ie_solver_advance(ie_solver s, int cycles, void *stream) {
    ie::NvtxRange nvtx_range("ie_solver_advance");
    if (!s || cycles < 0) return set_error("bad argument"), IE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < cycles; ++c) {
        if (!s->exec) {
            std::lock_guard<std::recursive_mutex> lock(device_mutex());
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
    return mirror_status(s, st);
}

ie_status ie_solver_poll(ie_solver s, int *done, ie_solve_info *info) {
    if (!s || !done) return set_error("null argument"), IE_ERR_INVALID;
    cudaError_t q = cudaEventQuery(s->ev);
    if (q == cudaErrorNotReady) {
        *done = 0;
        return IE_OK;
    }
    IE_CK(q);
    read_info_mirror(s, info, done);
    return IE_OK;
}

ie_status ie_solver_state(ie_solver s, int *state, ie_solve_info *info) {
    if (!s || !state) return set_error("null argument"), IE_ERR_INVALID;
    cudaError_t q = cudaEventQuery(s->ev);
    if (q == cudaErrorNotReady) {
        *state = IE_SOLVER_BUSY;
        return IE_OK;
    }
    IE_CK(q);
    int done = 0;
    read_info_mirror(s, info, &done);
    *state = done ? IE_SOLVER_DONE : IE_SOLVER_IDLE;
    return IE_OK;
}

ie_status ie_solve(ie_plan p, const void *v, void *c, int nrhs, const ie_solve_opts *opts, ie_solve_info *info,
                   void *stream) {
    ie::NvtxRange nvtx_range("ie_solve");
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
        IE_TRY(ie_solver_start(s, v, c, stream));
        IE_TRY(run_cycles(s, o, stream, &inf));
        result = inf.converged ? IE_OK : IE_ERR_NOT_CONVERGED;
    } else {
        // outer refinement: x64 += GMRES_prec(r), r = v - Z_refine(x) in FP64, per system
        if (!(p->prec_mask & IE_PRECMASK(o.refine_prec)) || !(p->prec_mask & IE_PRECMASK(o.prec)))
            return set_error("refinement precisions not in plan"), IE_ERR_UNSUPPORTED;
        ie_solve_opts io = o;
        io.refine = 0;
        io.tol = o.inner_tol;
        ie_solver s = nullptr;
        IE_TRY(cached_solver(p, nrhs, io, &s));
        const int64_t total = (int64_t)nrhs * p->n;
        const int S = s->S, nblk = s->nblk, G = s->G;
        const Seg sg = seg_of(s);
        double2 *x64 = nullptr, *part = nullptr;
        float2 *rv = nullptr, *d = nullptr, *Wz = nullptr;
        IE_CK(cudaMallocAsync(&x64, total * sizeof(double2), st));
        IE_CK(cudaMallocAsync(&rv, total * sizeof(float2), st));
        IE_CK(cudaMallocAsync(&d, total * sizeof(float2), st));
        IE_CK(cudaMallocAsync(&Wz, total * sizeof(float2), st));
        IE_CK(cudaMallocAsync(&part, (size_t)S * nblk * sizeof(double2), st));
        IE_CK(cudaMemsetAsync(part, 0, (size_t)S * nblk * sizeof(double2), st));
        ref_accumulate_kernel<<<vec_grid(total), 256, 0, st>>>(x64, nullptr, (float2 *)c, total, 1);
        count_launches(1);
        std::vector<double2> hp((size_t)S * nblk);
        std::vector<int> nch(G);
        for (int g = 0; g < G; ++g) nch[g] = (int)((p->goff[g + 1] - p->goff[g] + kChunk - 1) / kChunk);
        int outer = 0, inner_iters = 0, mv = 0;
        double worst = 1;
        ie_status e = IE_OK;
        bool reuse = false;     // the inner solver's last product is Z c in refine_prec
        while (e == IE_OK) {
            // r = v - Z x  (FP64 difference of the product); x = 0 on the first step, so r = v
            const float2 *Zc = nullptr;
            if (reuse) {
                Zc = s->W;
            } else if (outer > 0) {
                e = apply(p, IE_FULL, o.refine_prec, (const float2 *)c, Wz, nrhs, st);
                mv++;
                if (e != IE_OK) break;
                Zc = Wz;
            }
            ref_residual_kernel<<<dim3(s->C, nrhs), kDotThreads, 0, st>>>((const float2 *)v, Zc, rv, sg, nblk, part);
            count_launches(1);
            if (cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                set_error("refinement residual copy failed");
                e = IE_ERR_CUDA;
                break;
            }
            worst = 0;
            for (int q = 0; q < S; ++q) {
                double rs = 0, vs = 0;
                for (int b = 0; b < nch[q % G]; ++b) rs += hp[(size_t)q * nblk + b].x, vs += hp[(size_t)q * nblk + b].y;
                worst = std::max(worst, vs > 0 ? std::sqrt(rs / vs) : 0.0);
            }
            if (worst <= o.tol || outer >= o.max_refine || inner_iters >= o.max_iters) break;
            // inner solve Z d = r
            e = ie_solver_start(s, rv, d, stream);
            ie_solve_info ii{};
            if (e == IE_OK) e = run_cycles(s, io, stream, &ii);
            if (e != IE_OK) break;
            inner_iters += ii.iterations;
            mv += ii.matvecs;
            ref_accumulate_kernel<<<vec_grid(total), 256, 0, st>>>(x64, d, (float2 *)c, total, 0);
            count_launches(1);
            // After the first inner solve x = 0 + d exactly (c = d), and the inner solver's
            // restart product W = Z d was taken with the last update of d: when it used the
            // refinement's precision, the next residual reuses it instead of a new product.
            reuse = outer == 0 && ii.iterations > 0 && io.prec == o.refine_prec;
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
    IE_TRY(take_device_error(p, st));   // a translation that gave up a wait voids the solve
    return result;
}

}  // extern "C"
