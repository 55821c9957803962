// CVFCNN translation networks (§3) evaluated on the tensor cores (IE_PREC_CVFCNN).
//
// A network replaces G_d x in Alg. 2 by s (W2 relu(W1 x / s + b1) + b2), s = ||x||_inf,
// relu the Cartesian ReLU.  Both layers are complex GEMMs in the real form of the
// block product (translate_tc.cu): A rows 2r, 2r+1 hold Re and Im of a weight row, B
// rows 2j, 2j+1 the real and imaginary parts of column j, and the epilogue combines
// the four real products of each complex product with one lane exchange.
//   layer 1: D1 = A1 B^T, A1 = W1 in real form (2H <= 128 rows, K = 192), B the item's
//            gathered fp16 inputs (the same split input as the block product's);
//   layer 2: D2 = A2 H^T, A2 = W2 in real form (384 rows in three M-blocks, K = 64, the
//            hidden width padded with zero rows), H the hidden activations written back
//            to shared memory by the epilogue of layer 1 as the B operand of layer 2.
// The operands are fp16 (single products, FP32 accumulation): the networks' own error
// (e^u ~ 1e-3, eq. 171) is far above fp16 rounding, so the hi/lo split of the block
// product would buy nothing.  Per stored network the weights are kept as twelve 8 KB
// fp16 images (6 K-chunks of A1, 3 M-blocks x 2 K-chunks of A2) in the 64-byte-swizzled
// K-major layout of tcgen05.mma, each layer with a power-of-two scale.
//
// Work item = (displacement, run of <= 80 complex columns).  The MMA thread runs the
// layers one item apart: layer 1 of item i + 1 is issued before layer 2 of item i, so
// the tensor cores work while the hidden-layer warps turn item i + 1's layer 1 into its
// hidden operand (two hidden buffers alternate).  TMEM: layer 1 in columns [0, 160),
// layer 2 in two alternating slots [160, 320) and [320, 480).  608 threads, roles:
//   warp 0     weight producer (one thread): per item the 6 layer-1 images of item i + 1
//              and the 6 layer-2 images of item i (the MMA order), one bulk copy each
//              into a 4-deep ring (`afull` / `aempty`).
//   warp 1     MMA issuer (one thread).
//   warp 2     signaller: per input chunk, proxy fence after the gathers, `bfull`.
//   warps 3-6  gatherers of the inputs (as in translate_tc.cu), plus per column the
//              target offset, the layer-1 scale 2^(e_x + e_1) / s and the output scale s.
//   warps 7-10 hidden layer (one per TMEM lane quarter): z = D1 x scale + b1,
//              h = relu(z), written as fp16 into the hidden operand (rows 2j, 2j+1 of
//              column j, K = hidden index), proxy fence, `hready`.
//   warps 11-18 output (two per lane quarter, alternating 32-column chunks): y =
//              s (2^e_2 D2 + b2), one 8-byte red.global.add per complex result into the
//              slab d mod 8 (mapped row and sign for the symmetric store).
// Every wait is bounded as in the block product; a role that gives up raises the abort
// flag and the device error word, drains what it issued, and reaches the final barrier.
#include <algorithm>

#include "ie_internal.h"

namespace ie {
namespace {

constexpr int kCvTileCols = 80;                  // complex columns per item (N <= 160)
constexpr int kN = 2 * kCvTileCols;
constexpr int kAStages = 4;
constexpr int kGathWarps = 4;
constexpr int kGath = 32 * kGathWarps;
constexpr int kMidWarps = 4, kOutWarps = 8;
constexpr int kWarpGath0 = 3, kWarpMid0 = kWarpGath0 + kGathWarps, kWarpOut0 = kWarpMid0 + kMidWarps;
constexpr int kThreads = 32 * (kWarpOut0 + kOutWarps);          // 608
constexpr int kLines = (kCvTileCols + kGath / 8 - 1) / (kGath / 8);   // input lines per gatherer thread and chunk
constexpr int kImgBytes = 128 * kTcK * 2;                       // 8 KB image
constexpr int kImages = kTcKChunks + 3 * 2;                     // 12 per network
constexpr int kBPlane = kN * kTcK * 2;                          // 10 KB: one chunk of the inputs (hi only)
constexpr int kBBytes = kTcKChunks * kBPlane;                   // 60 KB
constexpr int kHChunks = kCvHp / kTcK;                          // 2 K-chunks of the hidden operand
constexpr int kHBytes = kHChunks * kBPlane;                     // 20 KB per hidden buffer
constexpr int kRing = 8;
constexpr int kEpiBytes = kRing * kCvTileCols * (8 + 4 + 4 + 2) + kRing * 16;   // per column: target, scales, Q
static_assert(kRing * kCvTileCols * (8 + 4 + 4 + 2) % 16 == 0, "item headers 16-byte aligned");
constexpr int kColBytes = 2 * kCvTileCols * 8;
constexpr int kBars = 2 * kAStages + 3 * kTcKChunks + 2 + 4 * 2 + kRing + 1;
constexpr int kSmemBytes = kAStages * kImgBytes + kBBytes + 2 * kHBytes + kEpiBytes + kColBytes + 8 * kBars + 16 + 1024;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kD2Col0 = 160;                               // TMEM columns of the layer-2 slots:
__device__ __forceinline__ uint32_t d2col(int slot) { return kD2Col0 + 160u * (uint32_t)slot; }   // 160, 320
constexpr long long kWaitCycles = 1ll << 31;
static_assert(kBPlane % 512 == 0, "operand planes hold whole 8-row groups");
static_assert(kGath >= kCvTileCols, "one gatherer thread per column of an item");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(kCvHp == 64, "two K-chunks of hidden units");
static_assert(kMidWarps % 4 == 0 && kOutWarps % 4 == 0, "whole TMEM lane quarters per role");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
template <bool SLEEP = true>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    const long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) break;
        if (SLEEP) __nanosleep(64);   // a waiting warp leaves the issue slots to the working ones
    }
    *abort_flag = 1;
    return false;
}
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void named_sync_gatherers() { asm volatile("bar.sync 1, %0;" ::"n"(kGath) : "memory"); }
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}
// kind::f16, fp16 A and B, FP32 accumulate, K-major, M = 128, N = n
__device__ __forceinline__ uint32_t f16_idesc(int n) {
    uint32_t d = 0;
    d |= 1u << 4;
    d |= (uint32_t)(n >> 3) << 17;
    d |= (uint32_t)(128 >> 4) << 24;
    return d;
}
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void red_add_v2(float *addr, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// ---------------------------------------------------------------- weight images
// One CTA per stored network: the 12 fp16 images (layer-1 K-chunks, then layer-2
// (M-block, K-chunk)) and the two power-of-two scales, from the complex64 weights in
// the SIMT layout (W1^T [192][64], b1 [64], W2^T [64][192], b2 [192]).
__global__ void cvfcnn_images_kernel(const float2 *__restrict__ W, uint16_t *__restrict__ img, int32_t *__restrict__ exps) {
    const float2 *w = W + (size_t)blockIdx.x * kCvBlockElems;
    uint16_t *out = img + (size_t)blockIdx.x * kImages * kTcImageElems;
    __shared__ float red[2][8];
    __shared__ float sc[2];
    float m1 = 0.f, m2 = 0.f;
    for (int i = threadIdx.x; i < kNU * kCvHp; i += blockDim.x) {
        const float2 a = w[kCvW1 + i], b = w[kCvW2 + i];
        m1 = fmaxf(m1, fmaxf(fabsf(a.x), fabsf(a.y)));
        m2 = fmaxf(m2, fmaxf(fabsf(b.x), fabsf(b.y)));
    }
    for (int o = 16; o; o >>= 1) {
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = m1, red[1][threadIdx.x >> 5] = m2;
    __syncthreads();
    if (threadIdx.x < 2) {
        float m = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[threadIdx.x][k]);
        int e = 0;
        if (m > 0.f) {
            frexpf(m, &e);
            e -= 14;            // m 2^-e < 2^14
        }
        exps[2 * blockIdx.x + threadIdx.x] = e;
        sc[threadIdx.x] = ldexpf(1.f, -e);
    }
    __syncthreads();
    // 12 images x 128 rows x 4 chunks of 16 bytes
    for (int t = threadIdx.x; t < kImages * 128 * 4; t += blockDim.x) {
        const int c = t & 3, r = (t >> 2) & 127, im = t >> 9;
        uint16_t vals[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float x;
            if (im < kTcKChunks) {      // layer 1: row r = 2h + part, K = input unknown
                const int h = r >> 1, k = kTcK * im + 8 * c + e;
                const float2 v = w[kCvW1 + (size_t)k * kCvHp + h];
                x = (r & 1 ? v.y : v.x) * sc[0];
            } else {                    // layer 2: (M-block, K-chunk), row 2m + part, K = hidden unit
                const int q = im - kTcKChunks, mb = q >> 1, kc = q & 1;
                const int R = 128 * mb + r, m = R >> 1, k = kTcK * kc + 8 * c + e;
                const float2 v = w[kCvW2 + (size_t)k * kNU + m];
                x = (R & 1 ? v.y : v.x) * sc[1];
            }
            vals[e] = __half_as_ushort(__float2half_rn(x));
        }
        uint4 pk;
        pk.x = vals[0] | ((uint32_t)vals[1] << 16);
        pk.y = vals[2] | ((uint32_t)vals[3] << 16);
        pk.z = vals[4] | ((uint32_t)vals[5] << 16);
        pk.w = vals[6] | ((uint32_t)vals[7] << 16);
        *reinterpret_cast<uint4 *>(out + (size_t)im * kTcImageElems + r * kTcK + 8 * (c ^ ((r >> 1) & 3))) = pk;
    }
}

struct CvArgs {
    const WorkItem *items;
    int64_t n_items;
    const uint16_t *img;        // [block][12 images]
    const int32_t *wexp;        // [block][2]
    const float2 *W;            // [block][kCvBlockElems] (biases)
    const int32_t *Xexp;        // [col]
    const float *Xinf;          // [col] ||x||_inf of the unpermuted column
    const uint16_t *Xtc;        // split inputs (hi planes used)
    int64_t plane;
    const int32_t *src, *dst;
    float *Yslab;
    size_t slab_stride;
    int nbox;
    int *err;
    const int *gate;
    const int32_t *gcanon, *gsigma;
    const uint16_t *symmap;
    int64_t sig_stride;
    const int32_t *pgroup;      // [pair] group of each pair (null: the item's own group)
};

// SYM: symmetric store (the output maps each column's rows by its Q); one instantiation per
// store mode keeps the other mode's code out of the output loop
template <bool SYM>
__global__ void __launch_bounds__(kThreads, 1) cvfcnn_tc_kernel(const CvArgs a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = smem;                                                // [kAStages][8 KB]
    unsigned char *sB = sA + kAStages * kImgBytes;                           // [6][10 KB]
    unsigned char *sH = sB + kBBytes;                                        // [2 buffers][2][10 KB]
    int64_t *ep_off = reinterpret_cast<int64_t *>(sH + 2 * kHBytes);        // [kRing][80] target (floats)
    float *ep_sc1 = reinterpret_cast<float *>(ep_off + kRing * kCvTileCols); // [kRing][80] layer-1 scale
    float *ep_s = ep_sc1 + kRing * kCvTileCols;                              // [kRing][80] ||x||_inf
    uint16_t *ep_sig = reinterpret_cast<uint16_t *>(ep_s + kRing * kCvTileCols);   // [kRing][80] input copy Q
    int4 *ep_head = reinterpret_cast<int4 *>(ep_sig + kRing * kCvTileCols);  // ncols, disp, -, block
    const uint16_t **colptr = reinterpret_cast<const uint16_t **>(ep_head + kRing);
    uint64_t *afull = reinterpret_cast<uint64_t *>(colptr + 2 * kCvTileCols);
    uint64_t *aempty = afull + kAStages;
    uint64_t *blanded = aempty + kAStages;
    uint64_t *bfull = blanded + kTcKChunks;
    uint64_t *bfree = bfull + kTcKChunks;
    uint64_t *d1full = bfree + kTcKChunks;       // [1]
    uint64_t *d1empty = d1full + 1;              // [1]
    uint64_t *d2full = d1empty + 1;              // [2]
    uint64_t *d2empty = d2full + 2;              // [2]
    uint64_t *hready = d2empty + 2;              // [2]
    uint64_t *hfree = hready + 2;                // [2]
    uint64_t *staged = hfree + 2;                // [kRing]
    uint64_t *mdone = staged + kRing;            // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; ++s) {
            mbar_init(smem_u32(&afull[s]), 1);
            mbar_init(smem_u32(&aempty[s]), 1);
        }
        for (int k = 0; k < kTcKChunks; ++k) {
            mbar_init(smem_u32(&blanded[k]), kGath);
            mbar_init(smem_u32(&bfull[k]), 1);
            mbar_init(smem_u32(&bfree[k]), 1);
        }
        mbar_init(smem_u32(d1full), 1);
        mbar_init(smem_u32(d1empty), kMidWarps);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&d2full[b]), 1);
            mbar_init(smem_u32(&d2empty[b]), kOutWarps);
            mbar_init(smem_u32(&hready[b]), kMidWarps);
            mbar_init(smem_u32(&hfree[b]), 1);
        }
        for (int b = 0; b < kRing; ++b) mbar_init(smem_u32(&staged[b]), kGath);
        mbar_init(smem_u32(mdone), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t first = blockIdx.x, step = gridDim.x;
    // items of this CTA: first + il * step, il < nil
    const int64_t nil = first < a.n_items ? (a.n_items - 1 - first) / step + 1 : 0;
    auto item = [&](int64_t il) { return a.items[first + il * step]; };
    auto block_of = [&](int disp) { return a.gcanon ? __ldg(a.gcanon + disp) : disp; };

    if (warp == 0) {
        // ---------------- weight producer (lane 0): the MMA's order, L1(0), then
        // L1(i + 1), L2(i) for i = 0 .. nil - 1
        if (lane == 0) {
            bool ok = true;
            int64_t g = 0;
            auto images = [&](int64_t il, int q0) {
                const uint16_t *im0 = a.img + (size_t)block_of(item(il).disp) * kImages * kTcImageElems;
                for (int q = q0; q < q0 + 6 && ok; ++q, ++g) {
                    const int s = (int)(g % kAStages);
                    if (!mbar_wait(smem_u32(&aempty[s]), (uint32_t)(((g / kAStages) & 1) ^ 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&afull[s]);
                    mbar_arrive_expect_tx(fb, kImgBytes);
                    bulk_g2s(smem_u32(sA + s * kImgBytes), im0 + (size_t)q * kTcImageElems, kImgBytes, fb);
                }
            };
            if (nil > 0) images(0, 0);
            for (int64_t il = 0; il < nil && ok; ++il) {
                if (il + 1 < nil) images(il + 1, 0);
                images(il, kTcKChunks);
            }
            if (!ok) {
                atomicExch(a.err, 1);
                for (int64_t gg = g > kAStages ? g - kAStages : 0; gg < g; ++gg) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(smem_u32(&afull[gg % kAStages]), (uint32_t)((gg / kAStages) & 1)) &&
                           clock64() - t0 < kWaitCycles) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (lane 0)
        if (lane == 0) {
            const uint64_t da = sw64_desc(smem_u32(sA)), db = sw64_desc(smem_u32(sB)), dh = sw64_desc(smem_u32(sH));
            int64_t g = 0;
            bool ok = true;
            auto idesc_of = [&](int64_t il) {
                const WorkItem it = item(il);
                return f16_idesc((2 * it.npairs * it.nr + 15) & ~15);
            };
            // layer 1 of item il into TMEM columns [0, 160)
            auto layer1 = [&](int64_t il) {
                const uint32_t idesc = idesc_of(il);
                if (!mbar_wait<false>(smem_u32(d1empty), (uint32_t)((il & 1) ^ 1), abort_flag)) return false;
                tc_fence_after();
                for (int kc = 0; kc < kTcKChunks; ++kc, ++g) {
                    const int s = (int)(g % kAStages);
                    if (!mbar_wait<false>(smem_u32(&afull[s]), (uint32_t)((g / kAStages) & 1), abort_flag) ||
                        !mbar_wait<false>(smem_u32(&bfull[kc]), (uint32_t)(il & 1), abort_flag))
                        return false;
                    tc_fence_after();
                    const uint64_t ad = da + (uint64_t)(s * (kImgBytes >> 4));
                    const uint64_t bd = db + (uint64_t)(kc * (kBPlane >> 4));
                    umma(tmem_base, ad, bd, idesc, kc ? 1u : 0u);
                    umma(tmem_base, ad + 2, bd + 2, idesc, 1u);
                    umma_commit(smem_u32(&aempty[s]));
                    umma_commit(smem_u32(&bfree[kc]));
                }
                umma_commit(smem_u32(d1full));
                return true;
            };
            // layer 2 of item il: one product per M-block into the alternating slots
            auto layer2 = [&](int64_t il) {
                const uint32_t idesc = idesc_of(il);
                const int hb = (int)(il & 1);
                if (!mbar_wait<false>(smem_u32(&hready[hb]), (uint32_t)((il >> 1) & 1), abort_flag)) return false;
                for (int mb = 0; mb < 3; ++mb) {
                    const int64_t u = il * 3 + mb;
                    const int sl = (int)(u & 1);
                    if (!mbar_wait<false>(smem_u32(&d2empty[sl]), (uint32_t)(((u >> 1) & 1) ^ 1), abort_flag))
                        return false;
                    tc_fence_after();
                    const uint32_t dt = tmem_base + d2col(sl);
                    for (int kc = 0; kc < kHChunks; ++kc, ++g) {
                        const int s = (int)(g % kAStages);
                        if (!mbar_wait<false>(smem_u32(&afull[s]), (uint32_t)((g / kAStages) & 1), abort_flag))
                            return false;
                        tc_fence_after();
                        const uint64_t ad = da + (uint64_t)(s * (kImgBytes >> 4));
                        const uint64_t hd = dh + (uint64_t)((hb * kHBytes + kc * kBPlane) >> 4);
                        umma(dt, ad, hd, idesc, kc ? 1u : 0u);
                        umma(dt, ad + 2, hd + 2, idesc, 1u);
                        umma_commit(smem_u32(&aempty[s]));
                    }
                    umma_commit(smem_u32(&d2full[sl]));
                }
                umma_commit(smem_u32(&hfree[hb]));       // layer 2 has read this hidden buffer
                return true;
            };
            if (nil > 0) ok = layer1(0);
            for (int64_t il = 0; il < nil && ok; ++il) {
                if (il + 1 < nil) ok = layer1(il + 1);
                if (ok) ok = layer2(il);
            }
            if (!ok) atomicExch(a.err, 1);
            umma_commit(smem_u32(mdone));
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(mdone), 0) && clock64() - t0 < kWaitCycles) {
            }
        }
        __syncwarp();
    } else if (warp == 2) {
        // ---------------- signaller (lane 0)
        if (lane == 0) {
            bool ok = true;
            for (int64_t il = 0; il < nil && ok; ++il) {
                for (int kc = 0; kc < kTcKChunks; ++kc) {
                    if (!mbar_wait<false>(smem_u32(&blanded[kc]), (uint32_t)(il & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();
                    mbar_arrive(smem_u32(&bfull[kc]));
                }
            }
            if (!ok) atomicExch(a.err, 1);
        }
        __syncwarp();
    } else if (warp < kWarpMid0) {
        // ---------------- input gatherers (warps 3-6)
        const int tid = threadIdx.x - 32 * kWarpGath0;
        bool ok = true;
        // each column carries its own group (slab, and with the symmetric store its input
        // copy Q and output map): a symmetric-store item spans the groups of its block
        struct Meta {
            int src, dst, rr, sig, slab, ncols, disp, blk;
            float sc1, s;
        };
        auto meta_issue = [&](const WorkItem &w, bool valid) {
            Meta m{0, 0, 0, 0, 0, 0, 0, 0, 0.f, 0.f};
            if (!valid) return m;
            m.ncols = w.npairs * w.nr;
            m.disp = w.disp;
            m.blk = block_of(w.disp);
            if (tid >= m.ncols) return m;
            const int p = w.pair0 + (w.nr == 1 ? tid : tid / w.nr);
            m.rr = w.nr == 1 ? 0 : tid % w.nr;
            const int grp = a.pgroup ? __ldg(a.pgroup + p) : w.disp;
            m.slab = grp % kSlabs;
            m.sig = a.gcanon ? __ldg(a.gsigma + grp) : 0;
            m.src = __ldg(a.src + p);
            m.dst = __ldg(a.dst + p);
            return m;
        };
        // column scales (they depend on the boxes): loaded a few chunks after meta_issue
        auto meta_scales = [&](Meta &m) {
            if (tid < m.ncols) {
                const int64_t col = (int64_t)m.rr * a.nbox + m.src;
                m.s = __ldg(a.Xinf + col);
                const int e = __ldg(a.Xexp + col) + __ldg(a.wexp + 2 * m.blk);
                m.sc1 = m.s > 0.f ? ldexpf(1.f, e) / m.s : 0.f;
            }
        };
        auto publish = [&](const Meta &m, int64_t il) {
            const bool on = tid < m.ncols;
            const int rb = (int)(il % kRing);
            if (tid < kCvTileCols) {
                colptr[(il & 1) * kCvTileCols + tid] =
                    on ? a.Xtc + (int64_t)m.sig * a.sig_stride + ((int64_t)m.rr * a.nbox + m.src) * (2 * kNU) : nullptr;
                if (SYM)   // float offset of the column's target, its slab included
                    ep_off[rb * kCvTileCols + tid] =
                        on ? (int64_t)m.slab * (2 * (int64_t)a.slab_stride) + 2 * ((int64_t)m.rr * a.nbox + m.dst) * kNU
                           : 0;
                else       // complex offset inside the item's slab (32 bits, in the same buffer)
                    reinterpret_cast<int32_t *>(ep_off)[rb * kCvTileCols + tid] = on ? (m.rr * a.nbox + m.dst) * kNU : 0;
                ep_sig[rb * kCvTileCols + tid] = (uint16_t)(on ? m.sig : 0);
                ep_sc1[rb * kCvTileCols + tid] = on ? m.sc1 : 0.f;
                ep_s[rb * kCvTileCols + tid] = on ? m.s : 0.f;
            }
            if (tid == 0) ep_head[rb] = make_int4(m.ncols, m.disp, 0, m.blk);
            mbar_arrive(smem_u32(&staged[rb]));
        };
        if (nil > 0) {
            WorkItem w_nxt = nil > 1 ? item(1) : WorkItem{0, 0, 0, 0, 1};
            Meta m_cur = meta_issue(item(0), true);
            meta_scales(m_cur);
            publish(m_cur, 0);
            named_sync_gatherers();
            const int sub = tid & 7, lg = tid >> 3, part = sub >> 2, c = sub & 3;
            for (int64_t il = 0; il < nil; ++il) {
                const bool has_next = il + 1 < nil;
                const WorkItem w_nn = il + 2 < nil ? item(il + 2) : WorkItem{0, 0, 0, 0, 1};
                Meta m_nxt = meta_issue(w_nxt, has_next);
                const int ncols = m_cur.ncols;
                const uint16_t *const *cols = colptr + (il & 1) * kCvTileCols;
                uint32_t loff[kLines];
                const uint16_t *lsrc[kLines];
#pragma unroll
                for (int k = 0; k < kLines; ++k) {
                    const int j = lg + (kGath / 8) * k;           // one line per column (hi only)
                    lsrc[k] = nullptr;
                    loff[k] = 0;
                    if (j < ncols) {
                        const int n = 2 * j + part;
                        loff[k] = (uint32_t)((n >> 3) * 512 + (n & 7) * 64 + ((c ^ ((n >> 1) & 3)) << 4));
                        lsrc[k] = cols[j] + part * kTcK + c * 8;
                    }
                }
                for (int kc = 0; kc < kTcKChunks && ok; ++kc) {
                    if (kc == 2) meta_scales(m_nxt);
                    if (!warp_wait(smem_u32(&bfree[kc]), (uint32_t)((il & 1) ^ 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sb = smem_u32(sB + kc * kBPlane);
#pragma unroll
                    for (int k = 0; k < kLines; ++k)
                        if (lsrc[k]) cp_async16(sb + loff[k], lsrc[k] + kc * (2 * kTcK));
                    cp_async_arrive_noinc(smem_u32(&blanded[kc]));
                }
                if (ok && has_next) publish(m_nxt, il + 1);
                named_sync_gatherers();
                if (*abort_flag) ok = false;
                if (!ok) break;
                w_nxt = w_nn;
                m_cur = m_nxt;
            }
        }
        cp_async_wait_all();
        if (!ok && tid == 0) atomicExch(a.err, 1);
    } else if (warp < kWarpOut0) {
        // ---------------- hidden layer, warps 7-10 (TMEM lane quarter = warp mod 4)
        const int q = warp & 3;
        const int half = (warp - kWarpMid0) >> 2;     // 0: one warp per quarter takes every chunk
        const bool odd = lane & 1;
        const int h = 16 * q + (lane >> 1);                 // hidden unit of this lane pair
        const int kc2 = h >> 5, kk = h & 31, grp = kk >> 3, el = kk & 7;
        const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16);
        for (int64_t il = 0; il < nil; ++il) {
            const int rb = (int)(il % kRing), hb = (int)(il & 1);
            if (!warp_wait(smem_u32(&staged[rb]), (uint32_t)((il / kRing) & 1), abort_flag) ||
                !warp_wait(smem_u32(d1full), (uint32_t)(il & 1), abort_flag) ||
                !warp_wait(smem_u32(&hfree[hb]), (uint32_t)(((il >> 1) & 1) ^ 1), abort_flag))
                break;
            tc_fence_after();
            const int4 hd = ep_head[rb];
            const int ncols = hd.x, blk = hd.w;
            const float *sc1 = ep_sc1 + rb * kCvTileCols;
            const float2 bias = __ldg(a.W + (size_t)blk * kCvBlockElems + kCvB1 + h);
            unsigned char *hbase = sH + hb * kHBytes + kc2 * kBPlane;
            for (int c0 = 32 * half; c0 < 2 * ncols; c0 += 32 * (kMidWarps / 4)) {
                uint32_t r[32];
                tmem_ld32(tbase + (uint32_t)c0, r);
                tmem_wait_ld();
                const int jb = c0 >> 1;
#pragma unroll
                for (int pk = 0; pk < 8; ++pk) {
                    const float a0 = __uint_as_float(r[4 * pk]), a1 = __uint_as_float(r[4 * pk + 1]);
                    const float b0 = __uint_as_float(r[4 * pk + 2]), b1 = __uint_as_float(r[4 * pk + 3]);
                    const float g0 = __shfl_xor_sync(0xffffffffu, odd ? a0 : b0, 1);
                    const float g1 = __shfl_xor_sync(0xffffffffu, odd ? a1 : b1, 1);
                    const float re = odd ? g0 - b1 : a0 - g1;
                    const float im = odd ? b0 + g1 : g0 + a1;
                    const int j = jb + 2 * pk + (odd ? 1 : 0);
                    if (j < ncols) {
                        const float sc = sc1[j];
                        const float zr = fmaf(re, sc, bias.x), zi = fmaf(im, sc, bias.y);
                        const int n0 = 2 * j, n1 = n0 + 1;   // rows of column j: re, im
                        unsigned char *p0 = hbase + (n0 >> 3) * 512 + (n0 & 7) * 64 + ((grp ^ ((n0 >> 1) & 3)) << 4) +
                                            2 * el;
                        unsigned char *p1 = hbase + (n1 >> 3) * 512 + (n1 & 7) * 64 + ((grp ^ ((n1 >> 1) & 3)) << 4) +
                                            2 * el;
                        *reinterpret_cast<__half *>(p0) = __float2half_rn(fmaxf(zr, 0.f));
                        *reinterpret_cast<__half *>(p1) = __float2half_rn(fmaxf(zi, 0.f));
                    }
                }
            }
            fence_proxy_async();            // generic-proxy writes -> the tensor core
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(smem_u32(&hready[hb]));
                mbar_arrive(smem_u32(d1empty));
            }
        }
    } else {
        // ---------------- output, warps 15-22 (TMEM lane quarter = warp mod 4)
        const int q = warp & 3;
        const int half = (warp - kWarpOut0) >> 2;
        const bool odd = lane & 1;
        bool ok = true;
        for (int64_t il = 0; il < nil && ok; ++il) {
            const int rb = (int)(il % kRing);
            if (!warp_wait(smem_u32(&staged[rb]), (uint32_t)((il / kRing) & 1), abort_flag)) break;
            const int4 hd = ep_head[rb];
            const int ncols = hd.x, blk = hd.w, slab = hd.y % kSlabs;   // the item's slab (full store)
            const int64_t *offs = ep_off + rb * kCvTileCols;
            const int32_t *offs32 = reinterpret_cast<const int32_t *>(ep_off) + rb * kCvTileCols;
            const float *sx = ep_s + rb * kCvTileCols;
            const uint16_t *sigs = ep_sig + rb * kCvTileCols;
            const float2 *Wb = a.W + (size_t)blk * kCvBlockElems;
            const float s2 = ldexpf(1.f, __ldg(a.wexp + 2 * blk + 1));
            for (int mb = 0; mb < 3; ++mb) {
                const int64_t u = il * 3 + mb;
                const int sl = (int)(u & 1);
                if (!warp_wait(smem_u32(&d2full[sl]), (uint32_t)((u >> 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + d2col(sl);
                const int mrow = 64 * mb + 16 * q + (lane >> 1);
                const float2 bias = __ldg(Wb + kCvB2 + mrow);   // canonical row (frame of the block)
                // the row itself without the symmetric store (one slab per item)
                float *const Yrow = a.Yslab + (int64_t)slab * (2 * (int64_t)a.slab_stride) + 2 * mrow;
                for (int c0 = 32 * half; c0 < 2 * ncols; c0 += 32 * (kOutWarps / 4)) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)c0, r);
                    tmem_wait_ld();
                    const int jb = c0 >> 1;
#pragma unroll
                    for (int pk = 0; pk < 8; ++pk) {
                        const float a0 = __uint_as_float(r[4 * pk]), a1 = __uint_as_float(r[4 * pk + 1]);
                        const float b0 = __uint_as_float(r[4 * pk + 2]), b1 = __uint_as_float(r[4 * pk + 3]);
                        const float g0 = __shfl_xor_sync(0xffffffffu, odd ? a0 : b0, 1);
                        const float g1 = __shfl_xor_sync(0xffffffffu, odd ? a1 : b1, 1);
                        const float re = odd ? g0 - b1 : a0 - g1;
                        const float im = odd ? b0 + g1 : g0 + a1;
                        const int j = jb + 2 * pk + (odd ? 1 : 0);
                        if (j < ncols) {
                            float s = sx[j];
                            float *y = Yrow + 2 * (int64_t)offs32[j];
                            if (SYM) {   // the row mapped by the column's Q
                                const uint16_t e = __ldg(a.symmap + sigs[j] * kNU + mrow);
                                y = a.Yslab + offs[j] + 2 * (e & 0xFF);
                                if (e & 0x100) s = -s;
                            }
                            red_add_v2(y, s * fmaf(re, s2, bias.x), s * fmaf(im, s2, bias.y));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&d2empty[sl]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols));
    }
}

}  // namespace

ie_status prepare_cvfcnn_tc() {
    IE_CK(cudaFuncSetAttribute(cvfcnn_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    IE_CK(cudaFuncSetAttribute(cvfcnn_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    return IE_OK;
}

size_t cvfcnn_image_elems() { return (size_t)kImages * kTcImageElems; }

ie_status build_cvfcnn_images(ie_plan p, cudaStream_t st) {
    if (!p->d_cvW || !p->d_cvimg || p->n_blocks == 0) return IE_OK;
    cvfcnn_images_kernel<<<(unsigned)p->n_blocks, 256, 0, st>>>(p->d_cvW, p->d_cvimg, p->d_cvexp);
    IE_CK_LAUNCH();
    return IE_OK;
}

int cvfcnn_tc_tile_columns() { return kCvTileCols; }

ie_status launch_translate_cvfcnn_tc(ie_plan p, float2 *Yslab, int nrhs, cudaStream_t st, const int *gate) {
    if (!p->d_cvimg) return set_error("the plan holds no tensor-core network images"), IE_ERR_UNSUPPORTED;
    if ((int64_t)p->max_rhs * p->nbox * kNU > (int64_t)INT32_MAX)
        return set_error("plan too large for the tensor-core networks' 32-bit offsets"), IE_ERR_UNSUPPORTED;
    WorkList *wl = nullptr;
    IE_TRY(work_list_for(p, IE_PREC_CVFCNN, nrhs, &wl));
    if (wl->n == 0) return IE_OK;
    CvArgs a;
    a.items = wl->d_items;
    a.n_items = wl->n;
    a.img = p->d_cvimg;
    a.wexp = p->d_cvexp;
    a.W = p->d_cvW;
    a.Xexp = p->d_Xexp;
    a.Xinf = p->d_Xinf;
    a.Xtc = p->d_Xtc;
    a.plane = (int64_t)nrhs * p->nbox * 2 * kNU;
    a.src = p->d_src;
    a.dst = p->d_dst;
    a.Yslab = reinterpret_cast<float *>(Yslab);
    a.slab_stride = slab_stride(p);
    a.nbox = p->nbox;
    a.err = p->d_err;
    a.gate = gate;
    a.gcanon = p->sym ? p->d_gcanon : nullptr;
    a.gsigma = p->sym ? p->d_gsigma : nullptr;
    a.symmap = p->sym ? p->d_symmap : nullptr;
    a.sig_stride = 2 * a.plane;
    a.pgroup = p->sym ? p->d_pgroup : nullptr;   // the symmetric store's items are packed
    const int grid = (int)std::min<int64_t>(wl->n, p->tc_sms > 0 ? p->tc_sms : 148);
    if (p->sym)
        cvfcnn_tc_kernel<true><<<grid, kThreads, kSmemBytes, st>>>(a);
    else
        cvfcnn_tc_kernel<false><<<grid, kThreads, kSmemBytes, st>>>(a);
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie
