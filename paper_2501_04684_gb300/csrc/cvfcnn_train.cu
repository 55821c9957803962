// Training of the CVFCNN translation networks (§3), first stage, on the GPU.
//
// One network per canonical displacement c = sorted |d| (192 -> H -> 192, complex,
// Cartesian ReLU on the hidden layer; the network is applied to x / ||x||_inf and its
// output is scaled back, so it learns G_c on the unit l-inf ball).  The paper's first
// training stage: inputs whose real and imaginary parts are uniform in [-1, 1]
// (normalised by their l-inf norm), the DGFA product G_c x as the target, mean square
// error, Adam; the stage ends when the relative l2 error of the outputs on a test set of
// the same distribution, e^u of eq. 171, is below the tolerance (1e-3 in the paper).
// The paper's second stage needs RWG-mapped surface data (absent here) and is not run.
//
// Layout: one CTA per network (persistent over networks), 256 threads; an Adam step
// sums the gradients of `minibatches` minibatches of 32 samples, each held in shared
// memory in turn:
//   X  [192][33]  inputs x / s (column j = sample j; rows padded to 33 against bank
//                 conflicts)
//   R  [192][33]  target G x / (s g) (g = max |G| of the block, so the weights the
//                 optimiser sees are of order one), then the output residual
//   Z  [64][33]   hidden pre-activations, then the back-propagated hidden gradient
//   Hh [64][33]   hidden activations
// Weights and Adam moments live in global memory (L2-resident while the CTA trains):
// W1 [64][192], W2T [64][192] (W2 transposed), b1 [64], b2 [192]; rows h >= H stay zero.
// Per step: x from a counter-based hash (the generator is stated below), s = max |x_u|,
// forward, residual, back-propagation (complex gradients as d/dRe + j d/dIm of the
// real loss; the Cartesian ReLU passes the real and the imaginary part of the hidden
// gradient where the real and the imaginary part of the pre-activation are positive),
// Adam on the real and imaginary parts with a cosine-decayed step size.  Every
// `eval_every` steps e^u is measured on a fixed test set of 64 samples; training of the
// network stops once it is below the tolerance or after `max_steps`.
#include <algorithm>
#include <array>
#include <chrono>
#include <map>
#include <vector>

#include "ie_internal.h"

namespace ie {
namespace {

constexpr int kTB = 32;             // minibatch
constexpr int kTP = kTB + 1;        // padded row length (float2)
constexpr int kTrainThreads = 256;
constexpr int kTestSamples = 64;
constexpr int kWElems = kCvHp * kNU;                    // W1 or W2T
constexpr int kStateElems = 2 * kWElems + kCvHp + kNU;  // W1, W2T, b1, b2
constexpr uint32_t kTestStream = 0xFFFFFFFFu;           // step index of the test set

struct SmemTrain {
    float2 X[kNU][kTP];
    float2 R[kNU][kTP];
    float2 Z[kCvHp][kTP];
    float2 Hh[kCvHp][kTP];
    float inv_s[kTB];
    float red[kTrainThreads / 32];
    float err[kTB];
    float enorm[kTB];
};

// splitmix64 finaliser: the counter-based generator of the training inputs
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// two uniforms in [-1, 1) from one draw
__device__ __forceinline__ float2 uniform2(uint64_t seed, uint32_t net, uint32_t step, uint32_t idx) {
    const uint64_t r = mix64(seed ^ mix64(((uint64_t)net << 32 | step) ^ mix64(idx)));
    const float a = (float)(r >> 40) * (1.0f / 16777216.0f);             // 24 bits
    const float b = (float)((r >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
    return make_float2(2.f * a - 1.f, 2.f * b - 1.f);
}
// standard normal pair by Box-Muller from one draw
__device__ __forceinline__ float2 normal2(uint64_t seed, uint32_t net, uint32_t idx) {
    const uint64_t r = mix64(seed ^ mix64(((uint64_t)net << 32 | 0xABCDu) ^ mix64(idx)));
    const float u1 = ((float)(r >> 40) + 1.f) * (1.0f / 16777217.0f);
    const float u2 = (float)((r >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
    const float rad = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincosf(6.2831853f * u2, &sn, &cs);
    return make_float2(rad * cs, rad * sn);
}

__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

struct TrainArgs {
    const float2 *C;        // [net][192 k][192 m] FP32 blocks G_c (transposed)
    float2 *state;          // [net][4][kStateElems]: weights, Adam m, Adam v ((re, im) second moments),
                            // gradient sum over the minibatches of a step
    float2 *Wout;           // [net][kCvBlockElems] trained networks in the inference layout
    float *eu;              // [net] final e^u
    int *steps_used;        // [net]
    int64_t nnet;
    int H, max_steps, eval_every, micro;
    float lr, tol;
    uint64_t seed;
};

// Inputs of a minibatch (or half of the test set) into S.X and their 1 / s.
__device__ void make_inputs(SmemTrain &S, const TrainArgs &a, uint32_t net, uint32_t step, int part) {
    const int t = threadIdx.x;
    for (int idx = t; idx < kNU * kTB; idx += kTrainThreads) {
        const int u = idx / kTB, j = idx % kTB;
        S.X[u][j] = uniform2(a.seed, net, step, (uint32_t)((part * kTB + j) * kNU + u));
    }
    __syncthreads();
    // s_j = max_u |x_u|: warp w reduces samples w, w + 8, w + 16, w + 24
    const int w = t >> 5, lane = t & 31;
    for (int j = w; j < kTB; j += kTrainThreads / 32) {
        float m = 0.f;
        for (int u = lane; u < kNU; u += 32) {
            const float2 x = S.X[u][j];
            m = fmaxf(m, x.x * x.x + x.y * x.y);
        }
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) S.inv_s[j] = m > 0.f ? rsqrtf(m) : 0.f;
    }
    __syncthreads();
    for (int idx = t; idx < kNU * kTB; idx += kTrainThreads) {
        const int u = idx / kTB, j = idx % kTB;
        const float q = S.inv_s[j];
        S.X[u][j] = make_float2(S.X[u][j].x * q, S.X[u][j].y * q);
    }
    __syncthreads();
}

// R[m][j] = sum_k G[m][k] X[k][j] / g  (thread: 4 columns, 6 rows)
__device__ void teacher(SmemTrain &S, const float2 *__restrict__ G, float ginv) {
    const int t = threadIdx.x, j0 = 4 * (t & 7), mr = t >> 3;
    float2 acc[6][4];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = make_float2(0.f, 0.f);
    for (int k = 0; k < kNU; ++k) {
        float2 g[6], x[4];
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = __ldg(G + (size_t)k * kNU + mr + 32 * i);
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = S.X[k][j0 + c];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) cfma(acc[i][c], g[i], x[c]);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) S.R[mr + 32 * i][j0 + c] = make_float2(acc[i][c].x * ginv, acc[i][c].y * ginv);
}

// Z = W1 X + b1, Hh = relu(Z) (thread: column j, rows hr + 8 i)
__device__ void forward_hidden(SmemTrain &S, const float2 *__restrict__ W1, const float2 *__restrict__ b1, int H) {
    const int t = threadIdx.x, j = t & 31, hr = t >> 5;
    float2 acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int k = 0; k < kNU; ++k) {
        const float2 x = S.X[k][j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (hr + 8 * i < H) cfma(acc[i], W1[(size_t)(hr + 8 * i) * kNU + k], x);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int h = hr + 8 * i;
        float2 z = make_float2(0.f, 0.f);
        if (h < H) z = make_float2(acc[i].x + b1[h].x, acc[i].y + b1[h].y);
        S.Z[h][j] = z;
        S.Hh[h][j] = make_float2(fmaxf(z.x, 0.f), fmaxf(z.y, 0.f));
    }
}

// out[m][j] = W2 Hh + b2 (thread: 4 columns, 6 rows); mode 0: R = c (out - R);
// mode 1: per-sample |out - R|^2 and |R|^2 into S.err / S.enorm (test set)
__device__ void forward_output(SmemTrain &S, const float2 *__restrict__ W2T, const float2 *__restrict__ b2, int H,
                               float c, int mode) {
    const int t = threadIdx.x, j0 = 4 * (t & 7), mr = t >> 3;
    float2 acc[6][4];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = b2[mr + 32 * i];
    for (int k = 0; k < H; ++k) {
        float2 w[6], h[4];
#pragma unroll
        for (int i = 0; i < 6; ++i) w[i] = W2T[(size_t)k * kNU + mr + 32 * i];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = S.Hh[k][j0 + q];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) cfma(acc[i][q], w[i], h[q]);
    }
    if (mode == 0) {
        __syncthreads();   // every thread has read what it needs before R changes meaning
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 &r = S.R[mr + 32 * i][j0 + q];
                r = make_float2(c * (acc[i][q].x - r.x), c * (acc[i][q].y - r.y));
            }
    } else {
        float e[4] = {0.f, 0.f, 0.f, 0.f}, n[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 r = S.R[mr + 32 * i][j0 + q];
                const float dx = acc[i][q].x - r.x, dy = acc[i][q].y - r.y;
                e[q] += dx * dx + dy * dy;
                n[q] += r.x * r.x + r.y * r.y;
            }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            atomicAdd(&S.err[j0 + q], e[q]);
            atomicAdd(&S.enorm[j0 + q], n[q]);
        }
    }
}

// Adam on one complex parameter (real and imaginary parts separately)
__device__ __forceinline__ void adam(float2 &p, float2 &m, float2 &v, float2 g, float lr_t, float c1, float c2) {
    constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m = make_float2(b1 * m.x + (1.f - b1) * g.x, b1 * m.y + (1.f - b1) * g.y);
    v = make_float2(b2 * v.x + (1.f - b2) * g.x * g.x, b2 * v.y + (1.f - b2) * g.y * g.y);
    p.x -= lr_t * (m.x * c1) / (sqrtf(v.x * c2) + eps);
    p.y -= lr_t * (m.y * c1) / (sqrtf(v.y * c2) + eps);
}

// The gradient of one minibatch: summed into gs, or (last minibatch of the step) the
// sum taken and the Adam step made.
__device__ __forceinline__ void accumulate(float2 &p, float2 &m, float2 &v, float2 &gs, float2 g, bool first, bool last,
                                           float lr_t, float c1, float c2) {
    if (!first) g = make_float2(g.x + gs.x, g.y + gs.y);
    if (last)
        adam(p, m, v, g, lr_t, c1, c2);
    else
        gs = g;
}

__global__ void __launch_bounds__(kTrainThreads, 1) cvfcnn_train_kernel(const TrainArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemTrain &S = *reinterpret_cast<SmemTrain *>(smem_raw);
    const int t = threadIdx.x;
    const int H = a.H;
    for (int64_t net = blockIdx.x; net < a.nnet; net += gridDim.x) {
        const float2 *G = a.C + (size_t)net * kNU * kNU;
        float2 *P = a.state + (size_t)net * 4 * kStateElems;
        float2 *M = P + kStateElems, *V = M + kStateElems, *Gs = V + kStateElems;
        float2 *W1 = P, *W2T = P + kWElems, *b1 = P + 2 * kWElems, *b2 = b1 + kCvHp;
        // g = max |G_c|
        float gm = 0.f;
        for (int i = t; i < kNU * kNU; i += kTrainThreads) {
            const float2 v = G[i];
            gm = fmaxf(gm, v.x * v.x + v.y * v.y);
        }
        for (int o = 16; o; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if ((t & 31) == 0) S.red[t >> 5] = gm;
        __syncthreads();
        float g2 = 0.f;
        for (int w = 0; w < kTrainThreads / 32; ++w) g2 = fmaxf(g2, S.red[w]);
        const float gscale = g2 > 0.f ? sqrtf(g2) : 1.f, ginv = 1.f / gscale;
        // initial weights: W1 ~ CN(0, 1/192), W2 ~ CN(0, 1/H), biases 0; moments 0
        for (int i = t; i < kStateElems; i += kTrainThreads) {
            float2 w = make_float2(0.f, 0.f);
            if (i < kWElems) {
                if (i / kNU < H) {
                    const float2 z = normal2(a.seed, (uint32_t)net, (uint32_t)i);
                    const float sd = rsqrtf(2.f * kNU);
                    w = make_float2(z.x * sd, z.y * sd);
                }
            } else if (i < 2 * kWElems) {
                if ((i - kWElems) / kNU < H) {
                    const float2 z = normal2(a.seed, (uint32_t)net, (uint32_t)i);
                    const float sd = rsqrtf(2.f * H);
                    w = make_float2(z.x * sd, z.y * sd);
                }
            }
            P[i] = w;
            M[i] = make_float2(0.f, 0.f);
            V[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        float eu = 1.f;
        int step = 0;
        const float cres = 2.f / (kTB * kNU);
        for (; step < a.max_steps; ++step) {
            if (a.eval_every > 0 && step % a.eval_every == 0 && step > 0) {
                // e^u on the test set (two halves of 32)
                float acc = 0.f;
                for (int part = 0; part < kTestSamples / kTB; ++part) {
                    make_inputs(S, a, (uint32_t)net, kTestStream, part);
                    teacher(S, G, ginv);
                    if (t < kTB) S.err[t] = S.enorm[t] = 0.f;
                    __syncthreads();
                    forward_hidden(S, W1, b1, H);
                    __syncthreads();
                    forward_output(S, W2T, b2, H, 0.f, 1);
                    __syncthreads();
                    if (t < 32) {
                        float v = S.enorm[t] > 0.f ? sqrtf(S.err[t] / S.enorm[t]) : 0.f;
                        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (t == 0) S.red[0] = v;
                    }
                    __syncthreads();
                    acc += S.red[0];
                    __syncthreads();
                }
                eu = acc / kTestSamples;
                if (eu < a.tol) break;
            }
            const float lr_t = a.lr * (0.02f + 0.98f * 0.5f * (1.f + cospif((float)step / (float)a.max_steps)));
            const float c1 = 1.f / (1.f - powf(0.9f, (float)(step + 1)));
            const float c2 = 1.f / (1.f - powf(0.999f, (float)(step + 1)));
            // one Adam step on the gradient summed over `micro` minibatches of 32, all
            // taken with the weights of the start of the step
            for (int mbt = 0; mbt < a.micro; ++mbt) {
            const bool first = mbt == 0, last = mbt == a.micro - 1;
            make_inputs(S, a, (uint32_t)net, (uint32_t)(step * a.micro + mbt), 0);
            teacher(S, G, ginv);
            __syncthreads();
            forward_hidden(S, W1, b1, H);
            __syncthreads();
            forward_output(S, W2T, b2, H, cres, 0);
            __syncthreads();
            // hidden gradient with the old W2: dH = W2^H R, then dZ = dH through the ReLU (into Z)
            {
                const int j = t & 31, hr = t >> 5;
                float2 acc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
                for (int m = 0; m < kNU; ++m) {
                    const float2 r = S.R[m][j];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (hr + 8 * i < H) {
                            const float2 w = W2T[(size_t)(hr + 8 * i) * kNU + m];
                            // conj(w) r
                            acc[i].x = fmaf(w.x, r.x, fmaf(w.y, r.y, acc[i].x));
                            acc[i].y = fmaf(w.x, r.y, fmaf(-w.y, r.x, acc[i].y));
                        }
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int h = hr + 8 * i;
                    const float2 z = S.Z[h][j];
                    S.Z[h][j] = make_float2(z.x > 0.f ? acc[i].x : 0.f, z.y > 0.f ? acc[i].y : 0.f);
                }
            }
            // W2 (transposed) and b2: dW2T[k][m] = sum_j R[m][j] conj(Hh[k][j])
            for (int idx = t; idx < H * kNU; idx += kTrainThreads) {
                const int k = idx / kNU, m = idx % kNU;
                float2 g = make_float2(0.f, 0.f);
#pragma unroll 8
                for (int j = 0; j < kTB; ++j) {
                    const float2 r = S.R[m][j], h = S.Hh[k][j];
                    g.x = fmaf(r.x, h.x, fmaf(r.y, h.y, g.x));
                    g.y = fmaf(r.y, h.x, fmaf(-r.x, h.y, g.y));
                }
                accumulate(W2T[idx], M[kWElems + idx], V[kWElems + idx], Gs[kWElems + idx], g, first, last, lr_t, c1,
                           c2);
            }
            for (int m = t; m < kNU; m += kTrainThreads) {
                float2 g = make_float2(0.f, 0.f);
                for (int j = 0; j < kTB; ++j) g = make_float2(g.x + S.R[m][j].x, g.y + S.R[m][j].y);
                const int o = 2 * kWElems + kCvHp + m;
                accumulate(b2[m], M[o], V[o], Gs[o], g, first, last, lr_t, c1, c2);
            }
            __syncthreads();
            // W1 and b1: dW1[h][u] = sum_j dZ[h][j] conj(X[u][j])
            for (int idx = t; idx < H * kNU; idx += kTrainThreads) {
                const int h = idx / kNU, u = idx % kNU;
                float2 g = make_float2(0.f, 0.f);
#pragma unroll 8
                for (int j = 0; j < kTB; ++j) {
                    const float2 d = S.Z[h][j], x = S.X[u][j];
                    g.x = fmaf(d.x, x.x, fmaf(d.y, x.y, g.x));
                    g.y = fmaf(d.y, x.x, fmaf(-d.x, x.y, g.y));
                }
                accumulate(W1[idx], M[idx], V[idx], Gs[idx], g, first, last, lr_t, c1, c2);
            }
            for (int h = t; h < H; h += kTrainThreads) {
                float2 g = make_float2(0.f, 0.f);
                for (int j = 0; j < kTB; ++j) g = make_float2(g.x + S.Z[h][j].x, g.y + S.Z[h][j].y);
                accumulate(b1[h], M[2 * kWElems + h], V[2 * kWElems + h], Gs[2 * kWElems + h], g, first, last, lr_t,
                           c1, c2);
            }
            __syncthreads();
            }
        }
        // e^u of the final weights (if the loop ran out before a check)
        if (step >= a.max_steps) {
            float acc = 0.f;
            for (int part = 0; part < kTestSamples / kTB; ++part) {
                make_inputs(S, a, (uint32_t)net, kTestStream, part);
                teacher(S, G, ginv);
                if (t < kTB) S.err[t] = S.enorm[t] = 0.f;
                __syncthreads();
                forward_hidden(S, W1, b1, H);
                __syncthreads();
                forward_output(S, W2T, b2, H, 0.f, 1);
                __syncthreads();
                if (t < 32) {
                    float v = S.enorm[t] > 0.f ? sqrtf(S.err[t] / S.enorm[t]) : 0.f;
                    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (t == 0) S.red[0] = v;
                }
                __syncthreads();
                acc += S.red[0];
                __syncthreads();
            }
            eu = acc / kTestSamples;
        }
        // the network in the inference layout: W1^T [192][64], b1, W2^T [64][192] and b2 times g
        float2 *O = a.Wout + (size_t)net * kCvBlockElems;
        for (int idx = t; idx < kWElems; idx += kTrainThreads) {
            const int h = idx / kNU, u = idx % kNU;
            O[kCvW1 + (size_t)u * kCvHp + h] = W1[idx];
            const float2 w2 = W2T[idx];
            O[kCvW2 + idx] = make_float2(w2.x * gscale, w2.y * gscale);
        }
        for (int h = t; h < kCvHp; h += kTrainThreads) O[kCvB1 + h] = b1[h];
        for (int m = t; m < kNU; m += kTrainThreads) O[kCvB2 + m] = make_float2(b2[m].x * gscale, b2[m].y * gscale);
        if (t == 0) {
            a.eu[net] = eu;
            a.steps_used[net] = step;
        }
        __syncthreads();
    }
}

}  // namespace

ie_status launch_cvfcnn_train(ie_plan p, const ie_cvfcnn_train_opts &o, ie_cvfcnn_train_info *info, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    // canonical displacements of the plan's far groups, and each group's block and frame
    std::vector<int32_t> canon, gcanon(p->n_far_disp), gsigma(p->n_far_disp);
    {
        std::map<std::array<int32_t, 3>, int32_t> index;
        for (int64_t d = 0; d < p->n_far_disp; ++d) {
            int32_t c[3];
            gsigma[d] = canon_of_disp(&p->h_disp[3 * d], c);
            auto ins = index.emplace(std::array<int32_t, 3>{c[0], c[1], c[2]}, (int32_t)index.size());
            if (ins.second) canon.insert(canon.end(), c, c + 3);
            gcanon[d] = ins.first->second;
        }
    }
    const int64_t ncanon = (int64_t)canon.size() / 3;
    if (info) *info = ie_cvfcnn_train_info{};
    if (ncanon == 0) return IE_OK;
    // with the symmetric store the stored blocks are these canonical ones, in this order
    if (p->sym && ncanon != p->n_blocks) return set_error("canonical blocks do not match the store"), IE_ERR_CUDA;
    int32_t *d_canon = nullptr, *d_gc = nullptr, *d_gs = nullptr, *d_steps = nullptr;
    float2 *C = nullptr, *state = nullptr, *Wc = nullptr;
    float *d_eu = nullptr;
    uint16_t *d_map = nullptr;
    std::vector<uint16_t> map;
    symmetry_map_host(map);
    ie_status s = IE_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && s == IE_OK) {
            cudaGetLastError();
            set_error("CVFCNN training %s: %s", what, cudaGetErrorString(e));
            s = e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
        }
    };
    ck(cudaMallocAsync(&d_canon, canon.size() * sizeof(int32_t), st), "scratch");
    ck(cudaMallocAsync(&C, (size_t)ncanon * kNU * kNU * sizeof(float2), st), "scratch");
    ck(cudaMallocAsync(&state, (size_t)ncanon * 4 * kStateElems * sizeof(float2), st), "scratch");
    ck(cudaMallocAsync(&d_eu, (size_t)ncanon * sizeof(float), st), "scratch");
    ck(cudaMallocAsync(&d_steps, (size_t)ncanon * sizeof(int), st), "scratch");
    if (!p->sym) {
        ck(cudaMallocAsync(&Wc, (size_t)ncanon * kCvBlockElems * sizeof(float2), st), "scratch");
        ck(cudaMallocAsync(&d_gc, gcanon.size() * sizeof(int32_t), st), "scratch");
        ck(cudaMallocAsync(&d_gs, gsigma.size() * sizeof(int32_t), st), "scratch");
        ck(cudaMallocAsync(&d_map, map.size() * sizeof(uint16_t), st), "scratch");
    }
    if (s == IE_OK) {
        ck(cudaMemcpyAsync(d_canon, canon.data(), canon.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
        if (!p->sym) {
            ck(cudaMemcpyAsync(d_gc, gcanon.data(), gcanon.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
            ck(cudaMemcpyAsync(d_gs, gsigma.data(), gsigma.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
            ck(cudaMemcpyAsync(d_map, map.data(), map.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st), "copy");
        }
    }
    if (s == IE_OK) s = launch_coupling_simt(p, d_canon, ncanon, C, false, st);   // G_c, FP64 -> FP32, [k][m]
    if (s == IE_OK) {
        TrainArgs a;
        a.C = C;
        a.state = state;
        a.Wout = p->sym ? p->d_cvW : Wc;
        a.eu = d_eu;
        a.steps_used = d_steps;
        a.nnet = ncanon;
        a.H = p->cv_hidden;
        a.max_steps = o.max_steps;
        a.eval_every = o.eval_every;
        a.micro = o.minibatches;
        a.lr = (float)o.lr;
        a.tol = (float)o.tol;
        a.seed = o.seed;
        int dev = 0, sms = 0;
        ck(cudaGetDevice(&dev), "device");
        ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
        if (s == IE_OK) {
            const int grid = (int)std::min<int64_t>(ncanon, sms);
            cvfcnn_train_kernel<<<grid, kTrainThreads, sizeof(SmemTrain), st>>>(a);
            count_launches(1);
            ck(cudaGetLastError(), "launch");
        }
    }
    if (s == IE_OK && !p->sym) {
        launch_cvfcnn_expand(Wc, d_gc, d_gs, d_map, p->n_blocks, p->d_cvW, st);
        ck(cudaGetLastError(), "expansion");
    }
    if (s == IE_OK) s = build_cvfcnn_images(p, st);
    std::vector<float> eu(ncanon);
    std::vector<int> steps(ncanon);
    if (s == IE_OK) {
        ck(cudaMemcpyAsync(eu.data(), d_eu, ncanon * sizeof(float), cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaMemcpyAsync(steps.data(), d_steps, ncanon * sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "sync");
    }
    for (void *ptr : {(void *)d_canon, (void *)C, (void *)state, (void *)d_eu, (void *)d_steps, (void *)Wc, (void *)d_gc,
                      (void *)d_gs, (void *)d_map})
        if (ptr) cudaFreeAsync(ptr, st);
    if (s != IE_OK) return s;
    if (info) {
        info->networks = ncanon;
        double mx = 0, mean = 0;
        int below = 0, smax = 0;
        for (int64_t i = 0; i < ncanon; ++i) {
            mx = std::max(mx, (double)eu[i]);
            mean += eu[i];
            below += eu[i] < o.tol ? 1 : 0;
            smax = std::max(smax, steps[i]);
        }
        info->eu_max = mx;
        info->eu_mean = mean / ncanon;
        info->converged = below;
        info->steps_max = smax;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    p->cv_trained = 1;
    return IE_OK;
}

ie_status prepare_cvfcnn_train() {
    IE_CK(cudaFuncSetAttribute(cvfcnn_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(SmemTrain)));
    return IE_OK;
}

}  // namespace ie

using namespace ie;

extern "C" void ie_cvfcnn_train_opts_default(ie_cvfcnn_train_opts *o) {
    if (!o) return;
    o->max_steps = 8000;
    o->minibatches = 4;
    o->eval_every = 250;
    o->lr = 4e-3;
    o->tol = 1e-3;
    o->seed = 20250108;
}

extern "C" ie_status ie_cvfcnn_train(ie_plan p, const ie_cvfcnn_train_opts *opts, ie_cvfcnn_train_info *info,
                                     void *stream) {
    ie::NvtxRange nvtx_range("ie_cvfcnn_train");
    if (!p) return set_error("null plan"), IE_ERR_INVALID;
    if (!p->d_cvW) return set_error("the plan holds no CVFCNN surrogates"), IE_ERR_UNSUPPORTED;
    ie_cvfcnn_train_opts o;
    ie_cvfcnn_train_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_steps < 0 || o.max_steps > 1000000 || o.minibatches < 1 || o.minibatches > 64 || o.eval_every < 0 ||
        !(o.lr > 0) || !(o.tol > 0))
        return set_error("bad training options"), IE_ERR_INVALID;
    IE_TRY(prepare_cvfcnn_train());
    return launch_cvfcnn_train(p, o, info, (cudaStream_t)stream);
}
