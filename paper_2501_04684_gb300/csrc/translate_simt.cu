// K3 (plain path): translation stage (Alg. 2) in FP32 on the SIMT cores.
//
// Far pairs are grouped by box displacement d (Alg. 2 with eq. 13's matrix shared
// by every pair of the group), so each group is one dense complex GEMM
//     Y[:, dst_p] += G_d X[:, src_p]   for the pairs p of the group,
// with M = K = 192 and N = pairs x rhs.  A work item is one group's run of at most
// 64 columns (with the symmetry-compressed store: a run of columns over all the groups
// that share one stored block); one CTA computes its full 192 x 64 output tile over
// K = 192 in chunks of 16 (cp.async double buffering) and scatter-adds the tile into
// the target boxes.
//
// Accuracy: each tile sums 192 complex products in FP32 registers.  Contributions
// of different displacements meet in one of kSlabs FP32 partial fields (slab =
// d mod kSlabs, red.global.add.v4.f32), and the slabs are added in FP64 by the
// inverse-mapping kernel, so no FP32 sum runs over more than ~N_far/kSlabs terms.
#include <mutex>

#include "ie_internal.h"

namespace ie {

constexpr int kTileN = 64;
constexpr int kKC = 16;
constexpr int kThreads = 256;
constexpr int kAVec = kKC * kNU / 2 / kThreads;   // 16-byte copies of A per thread and chunk
constexpr int kBPer = kKC * kTileN / kThreads;    // consecutive k of one B column per thread and chunk
static_assert(kKC * kNU % (2 * kThreads) == 0 && kKC * kTileN % kThreads == 0 && kThreads % kTileN == 0,
              "loader shapes");

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

struct SmemSimt {
    float2 A[2][kKC][kNU];      // A^T chunk: [k][m]
    float2 B[2][kKC][kTileN];   // B chunk:   [k][col]
};

namespace {

// Symmetry-compressed store: the block of displacement d is G_c (c canonical) and
// G_d = S G_c S^T, so the tile reads G_c, takes its input from the signed-permuted
// copy Q of X, and adds output row u at U_Q(u) with the map's sign.  Items are packed:
// the groups of one stored block are contiguous in the pair list, and an item's columns
// may come from several of them, each column with its own group (pgroup), hence its own
// input copy, slab and output map.
struct SymArgs {
    const int32_t *gcanon = nullptr;     // [disp] stored block (null: no symmetry)
    const int32_t *gsigma = nullptr;     // [disp] copy Q of the input
    const int32_t *pgroup = nullptr;     // [pair] group of the pair (packed items)
    const uint16_t *map = nullptr;       // [48][192]
    size_t stride = 0;                   // complex elements between input copies
};

// One work item: the 192 x (npairs * nrhs) output tile of displacement it.disp,
// scatter-added into slab (disp mod kSlabs).
__device__ __forceinline__ void simt_tile(const WorkItem it, const float2 *__restrict__ C,
                                          const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                          const float2 *__restrict__ X, float2 *__restrict__ Yslab,
                                          size_t slab_stride, int nbox, int nrhs, const SymArgs sy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemSimt &S = *reinterpret_cast<SmemSimt *>(smem_raw);
    const int tid = threadIdx.x;
    const int ncols = it.npairs * it.nr;
    const float2 *Cd = C + (int64_t)(sy.gcanon ? sy.gcanon[it.disp] : it.disp) * kNU * kNU;
    auto group_of = [&](int pair) { return sy.pgroup ? __ldg(sy.pgroup + pair) : it.disp; };

    // B loader: thread -> (column, kBPer consecutive k)
    const int lcol = tid % kTileN;
    const int lkq = tid / kTileN;
    int lc = lcol < ncols ? lcol : 0;
    const int lpair = it.pair0 + lc / it.nr;
    const int lr = lc % it.nr;
    const float2 *xcol = X + ((int64_t)lr * nbox + src[lpair]) * kNU;
    if (sy.gcanon) xcol += (size_t)__ldg(sy.gsigma + group_of(lpair)) * sy.stride;

    auto load_chunk = [&](int kc, int buf) {
        // A: kKC x 192 float2 in 16-byte copies, kAVec per thread
        const float4 *ga = reinterpret_cast<const float4 *>(Cd + (int64_t)kc * kKC * kNU);
        float4 *sa = reinterpret_cast<float4 *>(&S.A[buf][0][0]);
#pragma unroll
        for (int t = 0; t < kAVec; ++t) cp_async16(sa + tid + t * kThreads, ga + tid + t * kThreads);
#pragma unroll
        for (int t = 0; t < kBPer; ++t) {
            int kk = lkq * kBPer + t;
            cp_async8(&S.B[buf][kk][lcol], xcol + kc * kKC + kk);
        }
        cp_commit();
    };

    const int tm = tid >> 3;     // 0..31: rows {2tm, 2tm+1} + 64 j
    const int tn = tid & 7;      // 0..7:  cols {2tn, 2tn+1} + 16 j
    float2 acc[6][8];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);

    constexpr int nK = kNU / kKC;   // 12
    load_chunk(0, 0);
    for (int kc = 0; kc < nK; ++kc) {
        int buf = kc & 1;
        if (kc + 1 < nK) {
            load_chunk(kc + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        // not unrolled: one K-step is ~200 instructions (192 FMAs), and a fully unrolled chunk
        // overflows the instruction cache (measured: 5% slower, "no instruction" stalls)
#pragma unroll 1
        for (int kk = 0; kk < kKC; ++kk) {
            float2 a[6], b[8];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float4 v = *reinterpret_cast<const float4 *>(&S.A[buf][kk][2 * tm + 64 * j]);
                a[2 * j] = make_float2(v.x, v.y);
                a[2 * j + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float4 v = *reinterpret_cast<const float4 *>(&S.B[buf][kk][2 * tn + 16 * j]);
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

#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int col = 2 * tn + 16 * (j >> 1) + (j & 1);
        if (col >= ncols) continue;
        int pair = it.pair0 + col / it.nr;
        int r = col % it.nr;
        const int grp = group_of(pair);
        float2 *ycol = Yslab + (size_t)(grp % kSlabs) * slab_stride + ((int64_t)r * nbox + dst[pair]) * kNU;
        if (sy.gcanon) {
            const uint16_t *map = sy.map + __ldg(sy.gsigma + grp) * kNU;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const uint16_t e = __ldg(map + 2 * tm + 64 * (i >> 1) + (i & 1));
                const float sg = (e & 0x100) ? -1.f : 1.f;
                atomicAdd(ycol + (e & 0xFF), make_float2(sg * acc[i][j].x, sg * acc[i][j].y));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float4 v = make_float4(acc[2 * i][j].x, acc[2 * i][j].y, acc[2 * i + 1][j].x, acc[2 * i + 1][j].y);
                atomicAdd(reinterpret_cast<float4 *>(ycol + 2 * tm + 64 * i), v);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
translate_simt_kernel(const WorkItem *__restrict__ items, const float2 *__restrict__ C,
                      const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                      const float2 *__restrict__ X, float2 *__restrict__ Yslab, size_t slab_stride,
                      int nbox, int nrhs, const SymArgs sy, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    simt_tile(items[blockIdx.x], C, src, dst, X, Yslab, slab_stride, nbox, nrhs, sy);
}

}  // namespace

size_t slab_stride(const ie_plan p) { return (size_t)p->max_rhs * p->nbox * kNU; }

ie_status prepare_translate_simt() {
    IE_CK(cudaFuncSetAttribute(translate_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(SmemSimt)));
    return IE_OK;
}

ie_status launch_translate_simt(ie_plan p, const float2 *X, float2 *Yslab, int nrhs, cudaStream_t st,
                                const int *gate) {
    WorkList *wl = nullptr;
    IE_TRY(work_list_for(p, IE_PREC_FP32, nrhs, &wl));
    if (wl->n == 0) return IE_OK;
    if (!p->d_Csimt) return set_error("the plan holds no FP32 coupling store"), IE_ERR_UNSUPPORTED;
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
    translate_simt_kernel<<<(unsigned)wl->n, kThreads, sizeof(SmemSimt), st>>>(
        wl->d_items, p->d_Csimt, p->d_src, p->d_dst, X, Yslab, slab_stride(p), p->nbox, nrhs, sy, gate);
    IE_CK_LAUNCH();
    return IE_OK;
}

int simt_tile_columns() { return kTileN; }

}  // namespace ie

// ---------------------------------------------------------------------------------
// ie_translate_noalloc: the FP32 translation with its scratch in a fixed device area.
//
// For callers that cannot allocate device memory when they run the product: code
// whose device memory is owned by another allocator (a framework pool that forbids
// raw cudaMalloc), or a latency-critical loop where cudaMalloc / cudaFree could
// block or synchronise the device.  ie_translate needs the plan's scratch slabs
// and, on the first call for a new number of right-hand sides, allocates a work
// list; this variant allocates nothing.  Its scratch is the file-scope array below,
// held by every GPU that loads the library until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Same tile as translate_simt_kernel; the work item comes from the group offsets
// (blockIdx.x = displacement group, blockIdx.y = run of `per` pairs inside it).
__global__ void __launch_bounds__(ie::kThreads, 1)
translate_simt_grouped_kernel(const int64_t *__restrict__ gstart, const float2 *__restrict__ C,
                              const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                              const float2 *__restrict__ X, float2 *__restrict__ Yslab, size_t slab_stride,
                              int nbox, int nrhs, int per) {
    int64_t d = blockIdx.x;
    int64_t s = gstart[d], e = gstart[d + 1];
    int64_t q = s + (int64_t)blockIdx.y * per;
    if (q >= e) return;
    ie::WorkItem it{(int32_t)d, (int32_t)q, (int32_t)(e - q < per ? e - q : per), 0, nrhs};
    ie::simt_tile(it, C, src, dst, X, Yslab, slab_stride, nbox, nrhs, ie::SymArgs());
}

// Device address of the scratch area on the current device (looked up once per
// device; the kernel attribute is set at the same time).
ie_status noalloc_scratch(void **out) {
    int dev = 0;
    IE_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return ie::set_error("device %d out of range", dev), IE_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        IE_CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        IE_CK(cudaFuncSetAttribute(translate_simt_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(ie::SmemSimt)));
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return IE_OK;
}

}  // namespace

extern "C" ie_status ie_translate_noalloc(ie_plan p, const void *X, void *Y, int nrhs, void *stream) {
    using namespace ie;
    if (!p || !X || !Y) return set_error("null argument"), IE_ERR_INVALID;
    if (nrhs < 1 || nrhs > p->max_rhs || nrhs > kTileN)
        return set_error("nrhs %d outside [1, %d]", nrhs, p->max_rhs < kTileN ? p->max_rhs : kTileN), IE_ERR_INVALID;
    if (!(p->prec_mask & IE_PRECMASK(IE_PREC_FP32)) || p->sym || !p->gnrhs.empty())
        return set_error("ie_translate_noalloc runs the FP32 translation over a full block store; this plan has "
                         "no FP32 store or a symmetry-compressed one"),
               IE_ERR_UNSUPPORTED;
    size_t stride = (size_t)nrhs * p->nbox * kNU;                 // float2 per slab
    size_t need = (size_t)kSlabs * stride * sizeof(float2);
    if (need > kNoAllocScratchBytes)
        return set_error("ie_translate_noalloc needs %zu bytes of scratch for %d boxes x %d rhs; the fixed area "
                         "holds %zu bytes (use ie_translate)", need, p->nbox, nrhs, kNoAllocScratchBytes),
               IE_ERR_INVALID;
    int per = kTileN / nrhs;
    int64_t maxg = 0;
    for (int64_t d = 0; d < p->n_far_disp; ++d) maxg = std::max<int64_t>(maxg, p->h_gstart[d + 1] - p->h_gstart[d]);
    int64_t runs = (maxg + per - 1) / per;
    if (runs > 65535) return set_error("displacement group too large for ie_translate_noalloc"), IE_ERR_INVALID;
    void *base = nullptr;
    IE_TRY(noalloc_scratch(&base));
    cudaStream_t st = (cudaStream_t)stream;
    float2 *slabs = reinterpret_cast<float2 *>(base);
    // the area keeps the previous call's contents: the slabs must start at zero
    IE_TRY(launch_zero(slabs, (size_t)kSlabs * stride * sizeof(float2), st));
    if (p->n_far_disp > 0) {
        // group offsets: the plan's device copy, uploaded once when the plan was built
        translate_simt_grouped_kernel<<<dim3((unsigned)p->n_far_disp, (unsigned)runs), kThreads, sizeof(SmemSimt),
                                        st>>>(p->d_gstart, p->d_Csimt, p->d_src, p->d_dst, (const float2 *)X, slabs,
                                              stride, p->nbox, nrhs, per);
        IE_CK_LAUNCH();
    }
    return launch_sum_slabs(p, slabs, kSlabs, stride, (float2 *)Y, nrhs, st);
}
