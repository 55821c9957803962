// K3 (tensor-core path): translation stage (Alg. 2) on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in TMEM), sm_103a.
//
// Complex GEMM in real form.  For one displacement d the coupling block G = Gr + j Gi
// (192 x 192, eq. 13) is stored as a 384 x 192 real matrix A with row 2m = Gr[m][:],
// row 2m+1 = Gi[m][:]; a source vector x = xr + j xi becomes two B rows (xr and xi).
// The product A B^T then holds Gr xr, Gr xi, Gi xr, Gi xi in adjacent TMEM lanes /
// columns, and the epilogue forms y = (Gr xr - Gi xi) + j (Gr xi + Gi xr) with one lane
// exchange.  Split precision: every operand is hi + lo in 16 bits (bf16 or fp16), and
// D = Ahi Bhi + Ahi Blo + Alo Bhi is accumulated in FP32 (BF16X1: Ahi Bhi only).
//
// Work item = (displacement, M-block of 128 real rows, run of <= 128 complex columns).
// Persistent CTAs walk the size-sorted item list round-robin.  576 threads, roles:
//   warps 0-7  producers.  Per item, thread t < columns owns column t: the pair's boxes,
//              the block and input copy (symmetric store) are fetched one item ahead,
//              the fp16 scales at that item's third stage, the work item two ahead, so
//              no dependent global load stalls a stage.  The column's gather base goes
//              to shared memory for the copies; its target offset and scale go to a
//              4-deep ring for the epilogue, released through the `staged` mbarrier.
//              Per K-chunk of 32 (a stage): one thread bulk-copies the two pre-swizzled
//              8 KB A images (TMA engine, complete_tx on `full`); every (column, hi/lo)
//              chunk of B is one 128-byte line of the chunk-major input (re and im rows
//              adjacent), copied by 8 lanes with 16-byte cp.async into the 64-byte-
//              swizzled K-major layout (chunk c of row n at c ^ ((n / 2) mod 4)); the
//              copy addresses are computed once per item.  Threads arrive on `landed`
//              when their copies complete (cp.async.mbarrier.arrive.noinc).
//   warp 9     signaller (one thread): per stage, waits for `landed`, issues the proxy
//              fence that makes the gathered rows visible to the tensor core, arrives on
//              `full`.  48 KB stages, 4-deep ring.
//   warp 8     MMA issuer (one thread): tcgen05.mma M=128, N<=256, K=16 with
//              descriptors derived from one base, into one of two TMEM accumulators
//              (2 x 256 columns); the next work item is prefetched.
//   warps 10-17 epilogue (two warps per TMEM lane quarter, alternating 16-column chunks,
//              two chunks per TMEM wait): lanes 2m' and 2m'+1 (Re and Im rows of complex
//              row m') exchange two values per column pair, then each adds one complex
//              result (fp16 rescaled) with an 8-byte red.global.add into the slab d mod 8,
//              at the mapped row with the map's sign for the symmetric store.
// Every wait is bounded and each role decides on a timeout uniformly (lane-0 wait +
// shuffle, or a named barrier + abort flag), so no lane is ever left at a barrier; a
// timeout sets the device error word, drains the CTA's copies, frees TMEM, returns.
#include <algorithm>

#include "ie_internal.h"

namespace ie {
namespace {

constexpr int kTcTileCols = 128;                 // complex columns per work item (N <= 256)
constexpr int kStages = 4;
constexpr int kAcc = 2;                          // TMEM accumulators of 256 columns
constexpr int kProducers = 256;
constexpr int kProdWarps = kProducers / 32;
constexpr int kMmaWarp = kProdWarps, kSigWarp = kProdWarps + 1;
constexpr int kLines = 2 * kTcTileCols / (kProducers / 8);      // B lines per producer thread and stage (<=)
constexpr int kEpilogue = 256;
constexpr int kThreadsTc = kProducers + 32 + 32 + kEpilogue;  // producers, MMA, signaller, epilogue
constexpr int kEpiFirst = kProducers + 64;                    // first epilogue thread
constexpr int kImgBytes = 128 * kTcK * 2;        // 8 KB A image
constexpr int kBBytes = 256 * kTcK * 2;          // 16 KB B plane (256 rows x 64 B)
constexpr int kStageBytes = 2 * kImgBytes + 2 * kBBytes;     // 48 KB
constexpr int kRing = 4;                         // epilogue metadata buffers (producers stay < 3 items ahead)
constexpr int kEpiBytes = kRing * kTcTileCols * (8 + 4) + kRing * 16;   // column offsets + scales + item header
constexpr int kColBytes = 2 * kTcTileCols * 8;                 // gather base pointer of each column, 2 items
constexpr int kSmemBytes = kStages * kStageBytes + kEpiBytes + kColBytes + 512 /*barriers*/ + 1024 /*alignment*/;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitCycles = 1ll << 31;     // bounded waits give up after ~1 s of SM clock

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
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void named_sync_epilogue() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void named_sync_producers() { asm volatile("bar.sync 2, %0;" ::"n"(kProducers) : "memory"); }

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
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t r[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct TcArgs {
    const WorkItem *items;
    int64_t n_items;
    const uint16_t *C;          // [disp][36 images]
    const int32_t *Cexp;        // [disp] or null
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
};

template <bool FP16, bool X3>
__global__ void __launch_bounds__(kThreadsTc, 1)
translate_tc_kernel(const TcArgs a) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    int64_t *ep_off = reinterpret_cast<int64_t *>(smem + kStages * kStageBytes);      // [kRing][128]
    float *ep_scale = reinterpret_cast<float *>(ep_off + kRing * kTcTileCols);          // [kRing][128]
    int4 *ep_head = reinterpret_cast<int4 *>(ep_scale + kRing * kTcTileCols);           // [kRing] ncols, disp, mb
    const uint16_t **colptr = reinterpret_cast<const uint16_t **>(ep_head + kRing);    // [2][128]
    uint64_t *full = reinterpret_cast<uint64_t *>(colptr + 2 * kTcTileCols);            // [kStages]
    uint64_t *empty = full + kStages;                                                    // [kStages]
    uint64_t *landed = empty + kStages;                                                  // [kStages]
    uint64_t *accfull = landed + kStages;                                                // [kAcc]
    uint64_t *accempty = accfull + kAcc;                                                 // [kAcc]
    uint64_t *staged = accempty + kAcc;                                                  // [kRing]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(staged + kRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 2);               // signaller + the A copies' expect_tx arrive
            mbar_init(smem_u32(&empty[s]), 1);
            mbar_init(smem_u32(&landed[s]), kProducers);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(smem_u32(&accfull[b]), 1);
            mbar_init(smem_u32(&accempty[b]), kEpilogue);
        }
        for (int b = 0; b < kRing; ++b) mbar_init(smem_u32(&staged[b]), kProducers);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int64_t first = blockIdx.x, step = gridDim.x;
    if (warp < kProdWarps) {
        // ---------------- producers (warps 0-7)
        const int tid = threadIdx.x;
        int64_t armed[kStages];
        for (int s = 0; s < kStages; ++s) armed[s] = -1;
        bool ok = true;
        // Per item, thread t owns column t: its gather base (input copy, rhs, source box)
        // and the epilogue's target offset and fp16 scale.  No dependent global load may
        // stall a stage, so the metadata of an item is fetched in steps over the items
        // before it: the work item two items ahead; its pair's boxes and the block and
        // input copy at the start of the item before; the fp16 scales at that item's
        // third stage; the result is published at its end.
        struct Meta {
            int src, dst, rr, blk, sig, ed, xe, ncols, disp, mb;
        };
        auto meta_issue = [&](const WorkItem &w, bool valid) {
            Meta m{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (!valid) return m;
            m.ncols = w.npairs * w.nr;
            m.disp = w.disp;
            m.mb = w.mb;
            m.blk = a.gcanon ? __ldg(a.gcanon + w.disp) : w.disp;
            m.sig = a.gcanon ? __ldg(a.gsigma + w.disp) : 0;
            if (tid >= m.ncols) return m;
            int p;
            if (w.nr == 1) {
                p = w.pair0 + tid;
            } else {
                p = w.pair0 + tid / w.nr;
                m.rr = tid % w.nr;
            }
            m.src = __ldg(a.src + p);
            m.dst = __ldg(a.dst + p);
            return m;
        };
        auto meta_scales = [&](Meta &m) {
            if (FP16 && tid < m.ncols) {
                m.ed = __ldg(a.Cexp + m.blk);
                m.xe = __ldg(a.Xexp + (int64_t)m.rr * a.nbox + m.src);
            }
        };
        // publish item il's column data: gather bases (producers) and the epilogue ring
        auto publish = [&](const Meta &m, int64_t il) {
            const bool on = tid < m.ncols;
            const int rb = (int)(il % kRing);
            if (tid < kTcTileCols) {
                colptr[(il & 1) * kTcTileCols + tid] =
                    on ? a.Xtc + (int64_t)m.sig * a.sig_stride + ((int64_t)m.rr * a.nbox + m.src) * (2 * kNU) : nullptr;
                ep_off[rb * kTcTileCols + tid] = on ? ((int64_t)m.rr * a.nbox + m.dst) * (2 * kNU) : 0;
                ep_scale[rb * kTcTileCols + tid] = (FP16 && on) ? ldexpf(1.f, m.ed + m.xe) : 1.f;
            }
            if (tid == 0) ep_head[rb] = make_int4(m.ncols, m.disp, m.mb, m.sig);
            mbar_arrive(smem_u32(&staged[rb]));      // release: the epilogue reads after its wait
        };
        WorkItem w_cur = a.items[first];
        WorkItem w_nxt = first + step < a.n_items ? a.items[first + step] : WorkItem{0, 0, 0, 0, 1};
        Meta m_cur = meta_issue(w_cur, true);
        meta_scales(m_cur);
        publish(m_cur, 0);
        named_sync_producers();
        // line layout of a stage: each (column, hi/lo) K-chunk is 128 contiguous bytes
        // (re 32 + im 32 values), fetched by 8 lanes: lanes 0-3 the re row, 4-7 the im row
        const int sub = tid & 7, lg = tid >> 3, part = sub >> 2, c = sub & 3;
        int64_t g = 0;                 // stages issued by this CTA
        int64_t il = 0;
        for (int64_t i = first; i < a.n_items; i += step, ++il) {
            const WorkItem it = w_cur;
            const int blk = m_cur.blk;
            const bool has_next = i + step < a.n_items;
            const WorkItem w_nn = i + 2 * step < a.n_items ? a.items[i + 2 * step] : WorkItem{0, 0, 0, 0, 1};
            Meta m_nxt = meta_issue(w_nxt, has_next);
            const int ncols = it.npairs * it.nr;
            const int nl = X3 ? 2 * ncols : ncols;
            const uint16_t *const *cols = colptr + (il & 1) * kTcTileCols;
            const uint16_t *Cd = a.C + (int64_t)blk * kTcDispElems;
            // this thread's lines of the item (<= kLines): offset inside a stage and source
            // of K-chunk 0, computed once per item; a stage then costs one add per copy
            uint32_t loff[kLines];
            const uint16_t *lsrc[kLines];
#pragma unroll
            for (int k = 0; k < kLines; ++k) {
                const int L = lg + (kProducers / 8) * k;
                lsrc[k] = nullptr;
                loff[k] = 0;
                if (L < nl) {
                    const int j = X3 ? (L >> 1) : L;
                    const int hl = X3 ? (L & 1) : 0;
                    const int n = 2 * j + part;
                    loff[k] = (uint32_t)((n >> 3) * 512 + (n & 7) * 64 + ((c ^ ((n >> 1) & 3)) << 4)) +
                              (hl ? (uint32_t)kBBytes : 0u);
                    lsrc[k] = cols[j] + (hl ? a.plane : 0) + part * kTcK + c * 8;
                }
            }
            for (int kc = 0; kc < kTcKChunks && ok; ++kc, ++g) {
                const int s = (int)(g % kStages);
                const uint32_t ph = (uint32_t)((g / kStages) & 1);
                if (kc == 2) meta_scales(m_nxt);
                if (!warp_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                unsigned char *st = smem + s * kStageBytes;
                const uint32_t sA = smem_u32(st), sB = smem_u32(st + 2 * kImgBytes);
                const uint32_t fb = smem_u32(&full[s]);
                if (tid == 0) {
                    mbar_arrive_expect_tx(fb, X3 ? 2 * kImgBytes : kImgBytes);
                    armed[s] = g;
                    const uint16_t *img = Cd + (int64_t)((it.mb * kTcKChunks + kc) * 2) * kTcImageElems;
                    bulk_g2s(sA, img, kImgBytes, fb);
                    if (X3) bulk_g2s(sA + kImgBytes, img + kTcImageElems, kImgBytes, fb);
                }
#pragma unroll
                for (int k = 0; k < kLines; ++k)
                    if (lsrc[k]) cp_async16(sB + loff[k], lsrc[k] + kc * (2 * kTcK));
                cp_async_arrive_noinc(smem_u32(&landed[s]));
            }
            // every producer warp reaches this once per item, also after a timeout
            if (ok && has_next) publish(m_nxt, il + 1);
            named_sync_producers();
            if (*abort_flag) ok = false;
            if (!ok) break;
            w_cur = w_nxt;
            w_nxt = w_nn;
            m_cur = m_nxt;
        }
        cp_async_wait_all();
        if (!ok) {
            if (tid == 0) {
                atomicExch(a.err, 1);
                // drain: every stage this CTA armed completes once its bulk bytes land
                for (int s = 0; s < kStages; ++s) {
                    if (armed[s] < 0) continue;
                    const uint32_t ph = (uint32_t)((armed[s] / kStages) & 1);
                    const long long t0 = clock64();
                    while (!mbar_try_wait(smem_u32(&full[s]), ph) && clock64() - t0 < kWaitCycles) __nanosleep(64);
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer (lane 0)
        if (lane == 0) {
            const uint64_t d0 = sw64_desc(smem_u32(smem));   // stage s: + s * kStageBytes / 16
            int64_t il = 0;
            bool ok = true;
            WorkItem nxt = first < a.n_items ? a.items[first] : WorkItem{0, 0, 0, 0, 1};
            for (int64_t i = first; i < a.n_items && ok; i += step, ++il) {
                const WorkItem it = nxt;
                if (i + step < a.n_items) nxt = a.items[i + step];   // in flight during this item
                const int ncols = it.npairs * it.nr;
                const int nmma = (2 * ncols + 15) & ~15;
                const uint32_t idesc = f16_idesc(nmma, FP16);
                const int buf = (int)(il % kAcc);
                const uint32_t aph = (uint32_t)((il / kAcc) & 1);
                if (!mbar_wait<false>(smem_u32(&accempty[buf]), aph ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(buf * 256);
                for (int kc = 0; kc < kTcKChunks; ++kc) {
                    const int64_t g = il * kTcKChunks + kc;
                    const int s = (int)(g % kStages);
                    const uint32_t ph = (uint32_t)((g / kStages) & 1);
                    if (!mbar_wait<false>(smem_u32(&full[s]), ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // descriptors of this stage; +2 advances the start address by 32 B (K = 16)
                    const uint64_t ah = d0 + (uint64_t)(s * (kStageBytes >> 4));
                    const uint64_t bh = ah + (uint64_t)((2 * kImgBytes) >> 4);
                    const uint64_t al = ah + (uint64_t)(kImgBytes >> 4), bl = bh + (uint64_t)(kBBytes >> 4);
                    umma(dt, ah, bh, idesc, kc ? 1u : 0u);
                    if (X3) {
                        umma(dt, ah, bl, idesc, 1u);
                        umma(dt, al, bh, idesc, 1u);
                    }
                    umma(dt, ah + 2, bh + 2, idesc, 1u);
                    if (X3) {
                        umma(dt, ah + 2, bl + 2, idesc, 1u);
                        umma(dt, al + 2, bh + 2, idesc, 1u);
                    }
                    umma_commit(smem_u32(&empty[s]));
                    if (kc == kTcKChunks - 1) umma_commit(smem_u32(&accfull[buf]));
                }
            }
            if (!ok) atomicExch(a.err, 1);
        }
    } else if (warp == kSigWarp) {
        // ---------------- signaller (lane 0)
        if (lane == 0) {
            int64_t g = 0;
            for (int64_t i = first; i < a.n_items; i += step) {
                bool ok = true;
                for (int kc = 0; kc < kTcKChunks; ++kc, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t ph = (uint32_t)((g / kStages) & 1);
                    if (!mbar_wait<false>(smem_u32(&landed[s]), ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();     // gathered rows (generic proxy) -> tensor core (async proxy)
                    mbar_arrive(smem_u32(&full[s]));
                }
                if (!ok) {
                    atomicExch(a.err, 1);
                    break;
                }
            }
        }
    } else {
        // ---------------- epilogue warps 6-13 (TMEM lane quarter = warp mod 4)
        const int q = warp & 3;
        const int half = (warp - kEpiFirst / 32) >> 2;     // which alternate 8-column chunks
        const int64_t slab_f = (int64_t)a.slab_stride * 2;
        int64_t il = 0;
        for (int64_t i = first; i < a.n_items; i += step, ++il) {
            const int buf = (int)(il % kAcc);
            const uint32_t aph = (uint32_t)((il / kAcc) & 1);
            const int rb = (int)(il % kRing);
            bool ok = true;
            if (lane == 0) {
                ok = mbar_wait(smem_u32(&staged[rb]), (uint32_t)((il / kRing) & 1), abort_flag) &&
                     mbar_wait(smem_u32(&accfull[buf]), aph, abort_flag);
            }
            named_sync_epilogue();               // makes the abort decision uniform
            if (*abort_flag) break;
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            const int4 hd = ep_head[rb];
            const int ncols = hd.x, disp = hd.y, mb = hd.z, sig = hd.w;
            const int64_t *offs = ep_off + rb * kTcTileCols;
            const float *scl = ep_scale + rb * kTcTileCols;
            const int m0 = 64 * mb + 16 * q;       // first complex row of this warp
            float *Ys = a.Yslab + (int64_t)(disp % kSlabs) * slab_f + 2 * m0 + lane;
            float sgn = 1.f;
            if (a.gcanon) {                        // output row of this lane in the frame of d
                const uint16_t e = __ldg(a.symmap + sig * kNU + m0 + (lane >> 1));
                Ys = a.Yslab + (int64_t)(disp % kSlabs) * slab_f + 2 * (e & 0xFF) + (lane & 1);
                sgn = (e & 0x100) ? -1.f : 1.f;
            }
            const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256);
            // two 16-column chunks per TMEM wait (this warp's chunks are 32 columns apart).
            // Lanes 2m', 2m'+1 hold Re G and Im G rows of complex row m'; per pair of
            // columns (k, k+1) they exchange two values, then the even lane owns the
            // complex result of column k and the odd lane that of column k+1, added with
            // one 8-byte reduction each.
            const bool odd = lane & 1;
            float *Yrow = Ys - (lane & 1);               // float offset of complex row m' (or U(m'))
            for (int c0 = 16 * half; c0 < 2 * ncols; c0 += 64) {
                uint32_t r[32];
                const bool two = c0 + 32 < 2 * ncols;   // warp-uniform
                tmem_ld16_nowait(tbase + (uint32_t)c0, r);
                if (two) {
                    tmem_ld16_nowait(tbase + (uint32_t)(c0 + 32), r + 16);
                } else {
#pragma unroll
                    for (int k = 16; k < 32; ++k) r[k] = 0u;
                }
                tmem_wait_ld();
                const int jb = c0 >> 1;
#pragma unroll
                for (int pk = 0; pk < 8; ++pk) {
                    const int k = 2 * pk;                // columns k, k+1 of the 16 (k even)
                    const float a0 = __uint_as_float(r[2 * k]), a1 = __uint_as_float(r[2 * k + 1]);
                    const float b0 = __uint_as_float(r[2 * k + 2]), b1 = __uint_as_float(r[2 * k + 3]);
                    // even lane (Re G row) sends column k+1's values, odd lane (Im G row) column k's
                    const float g0 = __shfl_xor_sync(0xffffffffu, odd ? a0 : b0, 1);
                    const float g1 = __shfl_xor_sync(0xffffffffu, odd ? a1 : b1, 1);
                    // even: y_k = (Gr xr - Gi xi, Gi xr + Gr xi) with Gi from the partner
                    // odd:  y_{k+1} with Gr from the partner
                    float re = odd ? g0 - b1 : a0 - g1;
                    float im = odd ? b0 + g1 : g0 + a1;
                    const int kk = k + (odd ? 1 : 0);
                    const int j = jb + (kk & 7) + 16 * (kk >> 3);
                    if (j < ncols) {
                        float sc = sgn;
                        if (FP16) sc *= scl[j];
                        atomicAdd(reinterpret_cast<float2 *>(Yrow + offs[j]), make_float2(sc * re, sc * im));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&accempty[buf]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols));
    }
}

template <bool FP16, bool X3>
ie_status set_attr() {
    IE_CK(cudaFuncSetAttribute(translate_tc_kernel<FP16, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    return IE_OK;
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
    WorkList *wl = nullptr;
    IE_TRY(work_list(p, true, nrhs, &wl));
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
    int grid = (int)std::min<int64_t>(wl->n, p->tc_sms > 0 ? p->tc_sms : 148);
    if (prec == IE_PREC_BF16X3)
        translate_tc_kernel<false, true><<<grid, kThreadsTc, kSmemBytes, st>>>(a);
    else if (prec == IE_PREC_FP16X3)
        translate_tc_kernel<true, true><<<grid, kThreadsTc, kSmemBytes, st>>>(a);
    else if (prec == IE_PREC_BF16X1)
        translate_tc_kernel<false, false><<<grid, kThreadsTc, kSmemBytes, st>>>(a);
    else if (prec == IE_PREC_FP16X1)
        translate_tc_kernel<true, false><<<grid, kThreadsTc, kSmemBytes, st>>>(a);
    else
        return set_error("not a tensor-core precision: %d", prec), IE_ERR_INVALID;
    IE_CK_LAUNCH();
    return IE_OK;
}

}  // namespace ie
