// K3 (tensor-core path): translation stage (Alg. 2) on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in TMEM), sm_103a.
//
// Complex GEMM in real form.  For one displacement d the coupling block G = Gr + j Gi
// (192 x 192, eq. 13) is stored as a 384 x 192 real matrix A with row 2m = Gr[m][:],
// row 2m+1 = Gi[m][:]; a source vector x = xr + j xi becomes two B rows (xr and xi).
// The product A B^T then holds Gr xr, Gr xi, Gi xr, Gi xi in adjacent TMEM lanes /
// columns, and the epilogue forms y = (Gr xr - Gi xi) + j (Gr xi + Gi xr) with one lane
// exchange.  Split precision: every operand is hi + lo in 16 bits (bf16 or fp16), and
// D = Ahi Bhi + Ahi Blo + Alo Bhi is accumulated in FP32 (X1 forms: Ahi Bhi only).
//
// Work item = (displacement, run of <= 96 complex columns).  The item's gathered inputs
// B (192 real rows x K = 192, hi and lo) stay in shared memory while the three M-blocks
// of 128 real rows of A stream past them, so every input line is gathered once per
// column tile (not once per M-block) and every M-block's product is one TMEM
// accumulator of N <= 192 columns; two accumulators alternate, so the epilogue of one
// M-block overlaps the MMAs of the next.  Persistent CTAs walk the items round-robin.
// 480 threads, roles:
//   warp 0     A producer (one thread): per (M-block, K-chunk of 32) one bulk copy of
//              the pre-swizzled hi (and lo) images into a 4-deep ring (TMA engine,
//              complete_tx on `afull`).
//   warp 1     MMA issuer (one thread): tcgen05.mma M=128, N<=192, K=16, three products
//              (hi*hi, hi*lo, lo*hi) per K-step for X3; commits free each A stage, free
//              each B chunk after the last M-block used it, and hand each accumulator to
//              the epilogue.
//   warp 2     signaller (one thread): per B chunk, waits for its gathers (`blanded`),
//              issues the proxy fence that makes rows written by cp.async visible to the
//              tensor core, arrives on `bfull`.
//   warps 3-6  B gatherers.  Per item thread t < columns owns column t: the pair's boxes,
//              the block and input copy (symmetric store) are loaded one item ahead, the
//              fp16 scales halfway through the item before, so no dependent global load
//              stalls a chunk.  The column's gather base goes to shared memory; its target
//              offset and scale go to a 4-deep ring for the epilogue (`staged`).  Per
//              K-chunk, once the previous item's last M-block has released it (`bfree`),
//              every (column, hi/lo) line of the chunk-major input (128 bytes: re and im
//              rows) is copied by 8 lanes with 16-byte cp.async into the 64-byte-swizzled
//              K-major layout (chunk c of row n at c ^ ((n / 2) mod 4)), at addresses
//              computed once per item; the threads arrive on `blanded`.
//   warps 7-14 epilogue (two warps per TMEM lane quarter, alternating 32-column chunks):
//              lanes 2m' and 2m'+1 (Re and Im rows of complex row m') exchange two values
//              per column pair, then each adds one complex result (fp16 rescaled) with an
//              8-byte red.global.add into the slab d mod 8, at the mapped row with the
//              map's sign for the symmetric store.
// Every wait is bounded: a role that gives up raises the CTA's abort flag and the device
// error word.  The A producer then waits (bounded) for its armed stages' bytes (`afull`
// depends on nothing else), the gatherers for their cp.async, the MMA thread for its
// issued MMAs; every role reaches the final barrier, which frees TMEM.
#include <algorithm>

#include "ie_internal.h"

namespace ie {
namespace {

constexpr int kTcTileCols = 96;                  // complex columns per work item (N <= 192)
constexpr int kN = 2 * kTcTileCols;              // real B rows of a full item
constexpr int kAStages = 4;
constexpr int kAcc = 2;                          // TMEM accumulators
constexpr uint32_t kAccCols = 256;               // TMEM columns of one accumulator slot (>= kN)
constexpr int kCtasPerSm = 1;                    // resident CTAs per SM (shared memory, TMEM, registers)
constexpr int kGathWarps = 4;
constexpr int kGath = 32 * kGathWarps;
constexpr int kEpiWarps = 8;
constexpr int kWarpGath0 = 3, kWarpEpi0 = kWarpGath0 + kGathWarps;
constexpr int kThreadsTc = 32 * (kWarpEpi0 + kEpiWarps);        // 480
constexpr int kLines = (2 * kTcTileCols) / (kGath / 8);         // B lines per gatherer thread and chunk (<=)
constexpr int kImgBytes = 128 * kTcK * 2;        // 8 KB A image
constexpr int kAStageBytes = 2 * kImgBytes;      // hi + lo
constexpr int kBPlane = kN * kTcK * 2;           // 12 KB: one chunk, one of hi / lo (192 rows x 64 B)
constexpr int kBChunkBytes = 2 * kBPlane;
constexpr int kBBytes = kTcKChunks * kBChunkBytes;              // 144 KB
constexpr int kRing = 4;                         // epilogue metadata buffers
constexpr int kEpiBytes = kRing * kTcTileCols * (8 + 4 + 2) + kRing * 16;   // per column: target, scale, Q
static_assert(kRing * kTcTileCols * (8 + 4 + 2) % 16 == 0, "item headers 16-byte aligned");
constexpr int kColBytes = 2 * kTcTileCols * 8;                  // gather base of each column, 2 items
constexpr int kSmemBytes = kAStages * kAStageBytes + kBBytes + kEpiBytes + kColBytes + 512 /*barriers*/ +
                           1024 /*alignment*/;
constexpr uint32_t kTmemCols = kAcc * kAccCols;
constexpr long long kWaitCycles = 1ll << 31;     // bounded waits give up after ~1 s of SM clock
// diagnostics (ie_diag_wait_limit): a shorter give-up limit for the pipeline's waits, so that
// a test can drive a real launch through its abort path; the drains keep kWaitCycles
__device__ long long g_wait_limit = 0;
static_assert(kAStages * kAStageBytes % 1024 == 0 && kBChunkBytes % 1024 == 0, "operand tiles 1 KB aligned");
static_assert(kSmemBytes <= 227 * 1024 && kCtasPerSm * (kSmemBytes + 1024) <= 228 * 1024, "shared memory");
static_assert(kN <= (int)kAccCols && kCtasPerSm * kTmemCols <= 512, "tensor memory");
static_assert(kEpiWarps % 4 == 0, "whole TMEM lane quarters per epilogue warp group");
static_assert(kGath >= kTcTileCols, "one gatherer thread per column of an item");

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
// Bounded wait by one thread: false when `limit` SM cycles pass without the phase
// completing (then the CTA's abort flag is raised) or the CTA already gave up.
// SLEEP = false for the latency-critical single threads (MMA issuer, signaller): they
// rely on try_wait's own suspension instead of backing off.
template <bool SLEEP = true>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          long long limit = kWaitCycles) {
    const long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) break;
        if (SLEEP && i > 32) __nanosleep(64);
    }
    *abort_flag = 1;
    return false;
}
// Whole warp: lane 0 waits, the outcome is broadcast.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          long long limit = kWaitCycles) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, limit) ? 1 : 0;
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
// Arrive on `bar` once every earlier cp.async of this thread has landed (no pending-count increment).
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);     // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;             // stride byte offset
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)4 << 61;                      // 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B both bf16 or both fp16,
// both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t f16_idesc(int n, bool fp16) {
    uint32_t d = 0;
    d |= 1u << 4;                        // D: F32
    d |= (fp16 ? 0u : 1u) << 7;          // A: F16 = 0, BF16 = 1
    d |= (fp16 ? 0u : 1u) << 10;         // B
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
// The same with A kept in the collector buffer for the next MMA (fill), or read from it
// for the last time (lastuse).
__device__ __forceinline__ void umma_fill(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_last(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
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

struct TcArgs {
    const WorkItem *items;
    int64_t n_items;
    const uint16_t *C;          // [block][36 images]
    const int32_t *Cexp;        // [block] or null
    const int32_t *Xexp;        // [col]
    const uint16_t *Xtc;        // [hl][col][chunk][reim][32]
    int64_t plane;              // elements per hl plane of Xtc
    const int32_t *src, *dst;
    float *Yslab;               // float view of the complex64 slabs
    size_t slab_stride;         // complex elements between slabs
    int nbox, nrhs;
    int *err;
    const int *gate;
    // symmetry-compressed store (null gcanon: one block per displacement)
    const int32_t *gcanon;      // [disp] stored block
    const int32_t *gsigma;      // [disp] input copy Q
    const uint16_t *symmap;     // [48][192] output map u -> U_Q(u) | 0x100 when negated
    int64_t sig_stride;         // elements between the input copies of Xtc
    // with the symmetric store an item's columns may come from several groups of its block
    const int32_t *pgroup;      // [pair] group of each pair (null: the item's own group)
};

// SYM: symmetric store (the epilogue maps each column's rows by its Q); one instantiation per
// store mode keeps the other mode's code out of the epilogue loop
template <bool FP16, bool X3, bool SYM>
__global__ void __launch_bounds__(kThreadsTc, kCtasPerSm)
translate_tc_kernel(const TcArgs a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sAbase = smem;                                                        // [kAStages][16 KB]
    unsigned char *sBbase = smem + kAStages * kAStageBytes;                              // [6][hi, lo][12 KB]
    int64_t *ep_off = reinterpret_cast<int64_t *>(sBbase + kBBytes);                    // [kRing][96] target (floats)
    float *ep_scale = reinterpret_cast<float *>(ep_off + kRing * kTcTileCols);          // [kRing][96]
    uint16_t *ep_sig = reinterpret_cast<uint16_t *>(ep_scale + kRing * kTcTileCols);    // [kRing][96] input copy Q
    int4 *ep_head = reinterpret_cast<int4 *>(ep_sig + kRing * kTcTileCols);             // [kRing] ncols, disp
    const uint16_t **colptr = reinterpret_cast<const uint16_t **>(ep_head + kRing);    // [2][96]
    uint64_t *afull = reinterpret_cast<uint64_t *>(colptr + 2 * kTcTileCols);           // [kAStages]
    uint64_t *aempty = afull + kAStages;                                                 // [kAStages]
    uint64_t *blanded = aempty + kAStages;                                               // [6]
    uint64_t *bfull = blanded + kTcKChunks;                                              // [6]
    uint64_t *bfree = bfull + kTcKChunks;                                                // [6]
    uint64_t *accfull = bfree + kTcKChunks;                                              // [kAcc]
    uint64_t *accempty = accfull + kAcc;                                                 // [kAcc]
    uint64_t *staged = accempty + kAcc;                                                  // [kRing]
    uint64_t *mdone = staged + kRing;                                                    // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long lim = g_wait_limit > 0 ? g_wait_limit : kWaitCycles;   // give-up limit of the pipeline's waits
    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; ++s) {
            mbar_init(smem_u32(&afull[s]), 1);              // the A producer's expect_tx arrive
            mbar_init(smem_u32(&aempty[s]), 1);
        }
        for (int k = 0; k < kTcKChunks; ++k) {
            mbar_init(smem_u32(&blanded[k]), kGath);
            mbar_init(smem_u32(&bfull[k]), 1);
            mbar_init(smem_u32(&bfree[k]), 1);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(smem_u32(&accfull[b]), 1);
            mbar_init(smem_u32(&accempty[b]), kEpiWarps);
        }
        for (int b = 0; b < kRing; ++b) mbar_init(smem_u32(&staged[b]), kGath);
        mbar_init(smem_u32(&mdone[0]), 1);
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
    if (warp == 0) {
        // ---------------- A producer (lane 0)
        if (lane == 0) {
            bool ok = true;
            int64_t g = 0;                  // A stages issued
            int64_t i = first;
            int blk = 0;
            if (i < a.n_items) {
                const int d0 = a.items[i].disp;
                blk = a.gcanon ? __ldg(a.gcanon + d0) : d0;
            }
            for (; i < a.n_items && ok; i += step) {
                // the next item's block, in flight during this item
                int blk_n = 0;
                if (i + step < a.n_items) {
                    const int dn = a.items[i + step].disp;
                    blk_n = a.gcanon ? __ldg(a.gcanon + dn) : dn;
                }
                const uint16_t *Cd = a.C + (int64_t)blk * kTcDispElems;
                for (int q = 0; q < 3 * kTcKChunks; ++q, ++g) {      // q = mb * 6 + kc
                    const int s = (int)(g % kAStages);
                    const uint32_t ph = (uint32_t)((g / kAStages) & 1);
                    if (!mbar_wait(smem_u32(&aempty[s]), ph ^ 1, abort_flag, lim)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&afull[s]);
                    mbar_arrive_expect_tx(fb, X3 ? 2 * kImgBytes : kImgBytes);
                    // images of (mb, kc) are (mb * 6 + kc) * 2 + hl: hi and lo adjacent
                    bulk_g2s(smem_u32(sAbase + s * kAStageBytes), Cd + (int64_t)(2 * q) * kTcImageElems,
                             X3 ? 2 * kImgBytes : kImgBytes, fb);
                }
                blk = blk_n;
            }
            if (!ok) {
                atomicExch(a.err, 1);
                // drain: the last stages armed complete once their bytes land (no other role involved)
                for (int64_t gg = g > kAStages ? g - kAStages : 0; gg < g; ++gg) {
                    const uint32_t ph = (uint32_t)((gg / kAStages) & 1);
                    const long long t0 = clock64();
                    while (!mbar_try_wait(smem_u32(&afull[gg % kAStages]), ph) && clock64() - t0 < kWaitCycles) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (lane 0)
        if (lane == 0) {
            const uint64_t da = sw64_desc(smem_u32(sAbase));      // A stage s: + s * kAStageBytes / 16
            const uint64_t db = sw64_desc(smem_u32(sBbase));      // B chunk kc: + kc * kBChunkBytes / 16
            int64_t il = 0, g = 0;
            bool ok = true, issued = false;
            WorkItem nxt = first < a.n_items ? a.items[first] : WorkItem{0, 0, 0, 0, 1};
            for (int64_t i = first; i < a.n_items && ok; i += step, ++il) {
                const WorkItem it = nxt;
                if (i + step < a.n_items) nxt = a.items[i + step];   // in flight during this item
                const int ncols = it.npairs * it.nr;
                const int nmma = (2 * ncols + 15) & ~15;
                const uint32_t idesc = f16_idesc(nmma, FP16);
                const uint32_t bph = (uint32_t)(il & 1);
                for (int mb = 0; mb < 3 && ok; ++mb) {
                    const int64_t qa = il * 3 + mb;          // accumulator use
                    const int buf = (int)(qa % kAcc);
                    if (!mbar_wait<false>(smem_u32(&accempty[buf]), (uint32_t)(((qa / kAcc) & 1) ^ 1), abort_flag, lim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)buf * kAccCols;
                    for (int kc = 0; kc < kTcKChunks; ++kc, ++g) {
                        const int s = (int)(g % kAStages);
                        if (!mbar_wait<false>(smem_u32(&afull[s]), (uint32_t)((g / kAStages) & 1), abort_flag, lim) ||
                            (mb == 0 && !mbar_wait<false>(smem_u32(&bfull[kc]), bph, abort_flag, lim))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        // descriptors of this K-chunk; +2 advances the start address by 32 B (K = 16)
                        const uint64_t ah = da + (uint64_t)(s * (kAStageBytes >> 4));
                        const uint64_t al = ah + (uint64_t)(kImgBytes >> 4);
                        const uint64_t bh = db + (uint64_t)(kc * (kBChunkBytes >> 4));
                        const uint64_t bl = bh + (uint64_t)(kBPlane >> 4);
                        // X3: hi*hi then hi*lo keep A (hi) in the collector buffer, so it is
                        // read from shared memory once for the two products
                        if (X3) {
                            umma_fill(dt, ah, bh, idesc, kc ? 1u : 0u);
                            umma_last(dt, ah, bl, idesc, 1u);
                            umma(dt, al, bh, idesc, 1u);
                            umma_fill(dt, ah + 2, bh + 2, idesc, 1u);
                            umma_last(dt, ah + 2, bl + 2, idesc, 1u);
                            umma(dt, al + 2, bh + 2, idesc, 1u);
                        } else {
                            umma(dt, ah, bh, idesc, kc ? 1u : 0u);
                            umma(dt, ah + 2, bh + 2, idesc, 1u);
                        }
                        issued = true;
                        umma_commit(smem_u32(&aempty[s]));
                        if (mb == 2) umma_commit(smem_u32(&bfree[kc]));
                        if (kc == kTcKChunks - 1) umma_commit(smem_u32(&accfull[buf]));
                    }
                }
            }
            if (!ok) {
                atomicExch(a.err, 1);
                // the MMAs already issued still read shared memory and TMEM: wait for them
                if (issued) {
                    umma_commit(smem_u32(&mdone[0]));
                    const long long t0 = clock64();
                    while (!mbar_try_wait(smem_u32(&mdone[0]), 0) && clock64() - t0 < kWaitCycles) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 2) {
        // ---------------- signaller (lane 0)
        if (lane == 0) {
            int64_t il = 0;
            bool ok = true;
            for (int64_t i = first; i < a.n_items && ok; i += step, ++il) {
                for (int kc = 0; kc < kTcKChunks; ++kc) {
                    if (!mbar_wait<false>(smem_u32(&blanded[kc]), (uint32_t)(il & 1), abort_flag, lim)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();     // gathered rows (generic proxy) -> tensor core (async proxy)
                    mbar_arrive(smem_u32(&bfull[kc]));
                }
            }
            if (!ok) atomicExch(a.err, 1);
        }
        __syncwarp();
    } else if (warp < kWarpEpi0) {
        // ---------------- B gatherers (warps 3-6)
        const int tid = threadIdx.x - 32 * kWarpGath0;       // 0 .. kGath-1
        bool ok = true;
        // Per item, thread t owns column t: its gather base (input copy, rhs, source box)
        // and the epilogue's target offset and fp16 scale.  The metadata of an item is
        // fetched over the item before it (boxes and copy at its start, fp16 scales at
        // its third chunk), so no dependent global load stalls a chunk.
        // Each column carries its own group (its slab d mod 8, and with the symmetric store
        // its input copy Q and output map): a symmetric-store item spans the groups of its block.
        struct Meta {
            int src, dst, rr, sig, slab, ed, xe, ncols, disp;
        };
        auto meta_issue = [&](const WorkItem &w, bool valid) {
            Meta m{0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (!valid) return m;
            m.ncols = w.npairs * w.nr;
            m.disp = w.disp;
            if (tid >= m.ncols) return m;
            int p;
            if (w.nr == 1) {
                p = w.pair0 + tid;
            } else {
                p = w.pair0 + tid / w.nr;
                m.rr = tid % w.nr;
            }
            const int grp = a.pgroup ? __ldg(a.pgroup + p) : w.disp;
            m.slab = grp % kSlabs;
            m.sig = a.gcanon ? __ldg(a.gsigma + grp) : 0;
            m.src = __ldg(a.src + p);
            m.dst = __ldg(a.dst + p);
            return m;
        };
        auto meta_scales = [&](Meta &m) {
            if (FP16 && tid < m.ncols) {
                const int blk = a.gcanon ? __ldg(a.gcanon + m.disp) : m.disp;
                m.ed = __ldg(a.Cexp + blk);
                m.xe = __ldg(a.Xexp + (int64_t)m.rr * a.nbox + m.src);
            }
        };
        // publish item il's column data: gather bases and the epilogue ring
        auto publish = [&](const Meta &m, int64_t il) {
            const bool on = tid < m.ncols;
            const int rb = (int)(il % kRing);
            if (tid < kTcTileCols) {
                colptr[(il & 1) * kTcTileCols + tid] =
                    on ? a.Xtc + (int64_t)m.sig * a.sig_stride + ((int64_t)m.rr * a.nbox + m.src) * (2 * kNU) : nullptr;
                if (SYM)   // float offset of the column's target, its slab included
                    ep_off[rb * kTcTileCols + tid] =
                        on ? (int64_t)m.slab * (2 * (int64_t)a.slab_stride) + 2 * ((int64_t)m.rr * a.nbox + m.dst) * kNU
                           : 0;
                else       // complex offset inside the item's slab (32 bits, in the same buffer)
                    reinterpret_cast<int32_t *>(ep_off)[rb * kTcTileCols + tid] = on ? (m.rr * a.nbox + m.dst) * kNU : 0;
                ep_scale[rb * kTcTileCols + tid] = (FP16 && on) ? ldexpf(1.f, m.ed + m.xe) : 1.f;
                ep_sig[rb * kTcTileCols + tid] = (uint16_t)(on ? m.sig : 0);
            }
            if (tid == 0) ep_head[rb] = make_int4(m.ncols, m.disp, 0, 0);
            mbar_arrive(smem_u32(&staged[rb]));      // release: the epilogue reads after its wait
        };
        WorkItem w_nxt = first + step < a.n_items ? a.items[first + step] : WorkItem{0, 0, 0, 0, 1};
        Meta m_cur = meta_issue(a.items[first], true);
        meta_scales(m_cur);
        publish(m_cur, 0);
        named_sync_gatherers();
        // line layout of a chunk: each (column, hi/lo) K-chunk is 128 contiguous bytes
        // (re 32 + im 32 values), fetched by 8 lanes: lanes 0-3 the re row, 4-7 the im row
        const int sub = tid & 7, lg = tid >> 3, part = sub >> 2, c = sub & 3;
        int64_t il = 0;
        for (int64_t i = first; i < a.n_items; i += step, ++il) {
            const bool has_next = i + step < a.n_items;
            const WorkItem w_nn = i + 2 * step < a.n_items ? a.items[i + 2 * step] : WorkItem{0, 0, 0, 0, 1};
            Meta m_nxt = meta_issue(w_nxt, has_next);
            const int ncols = m_cur.ncols;
            const int nl = X3 ? 2 * ncols : ncols;
            const uint16_t *const *cols = colptr + (il & 1) * kTcTileCols;
            // this thread's lines of the item (<= kLines): offset inside a chunk and source
            // of K-chunk 0, computed once per item; a chunk then costs one add per copy
            uint32_t loff[kLines];
            const uint16_t *lsrc[kLines];
#pragma unroll
            for (int k = 0; k < kLines; ++k) {
                const int L = lg + (kGath / 8) * k;
                lsrc[k] = nullptr;
                loff[k] = 0;
                if (L < nl) {
                    const int j = X3 ? (L >> 1) : L;
                    const int hl = X3 ? (L & 1) : 0;
                    const int n = 2 * j + part;
                    loff[k] = (uint32_t)((n >> 3) * 512 + (n & 7) * 64 + ((c ^ ((n >> 1) & 3)) << 4)) +
                              (hl ? (uint32_t)kBPlane : 0u);
                    lsrc[k] = cols[j] + (hl ? a.plane : 0) + part * kTcK + c * 8;
                }
            }
            for (int kc = 0; kc < kTcKChunks && ok; ++kc) {
                if (kc == 2) meta_scales(m_nxt);
                // the previous item's last M-block has finished with this chunk
                if (!warp_wait(smem_u32(&bfree[kc]), (uint32_t)((il & 1) ^ 1), abort_flag, lim)) {
                    ok = false;
                    break;
                }
                const uint32_t sB = smem_u32(sBbase + kc * kBChunkBytes);
#pragma unroll
                for (int k = 0; k < kLines; ++k)
                    if (lsrc[k]) cp_async16(sB + loff[k], lsrc[k] + kc * (2 * kTcK));
                cp_async_arrive_noinc(smem_u32(&blanded[kc]));
            }
            // every gatherer warp reaches this once per item, also after a timeout
            if (ok && has_next) publish(m_nxt, il + 1);
            named_sync_gatherers();
            if (*abort_flag) ok = false;
            if (!ok) break;
            w_nxt = w_nn;
            m_cur = m_nxt;
        }
        cp_async_wait_all();
        if (!ok && tid == 0) atomicExch(a.err, 1);
    } else {
        // ---------------- epilogue warps 7-14 (TMEM lane quarter = warp mod 4)
        const int q = warp & 3;
        const int half = (warp - kWarpEpi0) >> 2;          // which alternate 32-column chunks
        const bool odd = lane & 1;
        int64_t il = 0;
        bool ok = true;
        for (int64_t i = first; i < a.n_items && ok; i += step, ++il) {
            const int rb = (int)(il % kRing);
            if (!warp_wait(smem_u32(&staged[rb]), (uint32_t)((il / kRing) & 1), abort_flag, lim)) break;
            const int ncols = ep_head[rb].x, slab = ep_head[rb].y % kSlabs;   // the item's slab (full store)
            const int64_t *offs = ep_off + rb * kTcTileCols;
            const int32_t *offs32 = reinterpret_cast<const int32_t *>(ep_off) + rb * kTcTileCols;
            const float *scl = ep_scale + rb * kTcTileCols;
            const uint16_t *sigs = ep_sig + rb * kTcTileCols;
            for (int mb = 0; mb < 3; ++mb) {
                const int64_t qa = il * 3 + mb;
                const int buf = (int)(qa % kAcc);
                if (!warp_wait(smem_u32(&accfull[buf]), (uint32_t)((qa / kAcc) & 1), abort_flag, lim)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int mrow = 64 * mb + 16 * q + (lane >> 1);   // this lane's complex row
                // its target row without the symmetric store (one slab per item)
                float *const Yrow = a.Yslab + (int64_t)slab * (2 * (int64_t)a.slab_stride) + 2 * mrow;
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * kAccCols;
                // 32 TMEM columns = 16 complex columns per load.  Lanes 2m', 2m'+1 hold the Re G
                // and Im G rows of complex row m'; per pair of columns (k, k+1) they exchange
                // two values, then the even lane owns the complex result of column k and the
                // odd lane that of column k+1.
                for (int c0 = 32 * half; c0 < 2 * ncols; c0 += 32 * (kEpiWarps / 4)) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)c0, r);
                    tmem_wait_ld();
                    const int jb = c0 >> 1;
#pragma unroll
                    for (int pk = 0; pk < 8; ++pk) {
                        const float a0 = __uint_as_float(r[4 * pk]), a1 = __uint_as_float(r[4 * pk + 1]);
                        const float b0 = __uint_as_float(r[4 * pk + 2]), b1 = __uint_as_float(r[4 * pk + 3]);
                        // even lane (Re G row) sends column k+1's values, odd lane (Im G row) column k's
                        const float g0 = __shfl_xor_sync(0xffffffffu, odd ? a0 : b0, 1);
                        const float g1 = __shfl_xor_sync(0xffffffffu, odd ? a1 : b1, 1);
                        // even: y_k = (Gr xr - Gi xi, Gi xr + Gr xi) with Gi from the partner
                        // odd:  y_{k+1} with Gr from the partner
                        const float re = odd ? g0 - b1 : a0 - g1;
                        const float im = odd ? b0 + g1 : g0 + a1;
                        const int j = jb + 2 * pk + (odd ? 1 : 0);
                        if (j < ncols) {
                            float sc = FP16 ? scl[j] : 1.f;
                            float *y = Yrow + 2 * (int64_t)offs32[j];
                            if (SYM) {   // the row mapped by the column's Q
                                const uint16_t e = __ldg(a.symmap + sigs[j] * kNU + mrow);
                                y = a.Yslab + offs[j] + 2 * (e & 0xFF);
                                if (e & 0x100) sc = -sc;
                            }
                            red_add_v2(y, sc * re, sc * im);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&accempty[buf]));
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

template <bool FP16, bool X3>
ie_status set_attr() {
    IE_CK(cudaFuncSetAttribute(translate_tc_kernel<FP16, X3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemBytes));
    IE_CK(cudaFuncSetAttribute(translate_tc_kernel<FP16, X3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemBytes));
    return IE_OK;
}

template <bool FP16, bool X3>
void launch_tc(const TcArgs &a, int grid, bool sym, cudaStream_t st) {
    if (sym)
        translate_tc_kernel<FP16, X3, true><<<grid, kThreadsTc, kSmemBytes, st>>>(a);
    else
        translate_tc_kernel<FP16, X3, false><<<grid, kThreadsTc, kSmemBytes, st>>>(a);
}

}  // namespace

int tc_tile_columns() { return kTcTileCols; }

namespace {
// One thread waits, with the translation kernels' bounded wait, on an mbarrier that
// nothing arrives on; the wait must give up and report it.
__global__ void bounded_wait_selftest_kernel(long long limit, int *out) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, limit);
    out[0] = ok ? 0 : 1;
    out[1] = abort_flag;
}
}  // namespace

ie_status bounded_wait_selftest(double limit_ms, cudaStream_t st) {
    int *d = nullptr;
    IE_CK(cudaMallocAsync(&d, 2 * sizeof(int), st));
    const long long limit = (long long)(limit_ms * 2.0e6);   // SM cycles at ~2 GHz
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(limit, d);
    IE_CK_LAUNCH();
    int h[2] = {0, 0};
    IE_CK(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    IE_CK(cudaStreamSynchronize(st));
    IE_CK(cudaFreeAsync(d, st));
    if (h[0] == 1 && h[1] == 1) return set_error("bounded wait gave up as designed"), IE_ERR_TIMEOUT;
    return set_error("bounded wait self-test: the wait did not report a timeout"), IE_ERR_CUDA;
}

ie_status prepare_translate_tc() {
    IE_TRY((set_attr<false, true>()));
    IE_TRY((set_attr<true, true>()));
    IE_TRY((set_attr<false, false>()));
    IE_TRY((set_attr<true, false>()));
    return IE_OK;
}

ie_status launch_translate_tc(ie_plan p, int prec, float2 *Yslab, int nrhs, cudaStream_t st, const int *gate) {
    const bool fp16 = is_fp16(prec);
    const uint16_t *C = fp16 ? p->d_Cfp16 : p->d_Cbf16;
    if (!C) return set_error("tensor-core coupling store for precision %d not built", prec), IE_ERR_UNSUPPORTED;
    if ((int64_t)p->max_rhs * p->nbox * kNU > (int64_t)INT32_MAX)
        return set_error("plan too large for the tensor-core translation's 32-bit offsets"), IE_ERR_UNSUPPORTED;
    WorkList *wl = nullptr;
    IE_TRY(work_list_for(p, prec, nrhs, &wl));
    if (wl->n == 0) return IE_OK;
    TcArgs a;
    a.items = wl->d_items;
    a.n_items = wl->n;
    a.C = C;
    a.Cexp = fp16 ? p->d_Cexp16 : nullptr;
    a.Xexp = p->d_Xexp;
    a.Xtc = p->d_Xtc;
    a.plane = (int64_t)nrhs * p->nbox * 2 * kNU;
    a.src = p->d_src;
    a.dst = p->d_dst;
    a.Yslab = reinterpret_cast<float *>(Yslab);
    a.slab_stride = slab_stride(p);
    a.nbox = p->nbox;
    a.nrhs = nrhs;
    a.err = p->d_err;
    a.gate = gate;
    a.gcanon = p->sym ? p->d_gcanon : nullptr;
    a.gsigma = p->sym ? p->d_gsigma : nullptr;
    a.symmap = p->sym ? p->d_symmap : nullptr;
    a.sig_stride = 2 * a.plane;
    a.pgroup = p->sym ? p->d_pgroup : nullptr;   // the symmetric store's items are packed
    int grid = (int)std::min<int64_t>(wl->n, (int64_t)kCtasPerSm * (p->tc_sms > 0 ? p->tc_sms : 148));
    if (prec == IE_PREC_BF16X3)
        launch_tc<false, true>(a, grid, p->sym, st);
    else if (prec == IE_PREC_FP16X3)
        launch_tc<true, true>(a, grid, p->sym, st);
    else if (prec == IE_PREC_BF16X1)
        launch_tc<false, false>(a, grid, p->sym, st);
    else if (prec == IE_PREC_FP16X1)
        launch_tc<true, false>(a, grid, p->sym, st);
    else
        return set_error("not a tensor-core precision: %d", prec), IE_ERR_INVALID;
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie

extern "C" ie_status ie_diag_wait_limit(int64_t cycles) {
    if (cycles < 0) return ie::set_error("negative wait limit"), IE_ERR_INVALID;
    const long long v = (long long)cycles;
    IE_CK(cudaMemcpyToSymbol(ie::g_wait_limit, &v, sizeof(v)));
    return IE_OK;
}
