// Coupling-block stores shared by plans.
//
// The far translation G_d (eq. 13) depends on k, eta, the box edge and d only, so one
// set of blocks serves every scatterer discretised with the same boxes (end of §2); with
// the lattice symmetry of §2.2 only the canonical c = sorted |d| need storing.  A store
// holds G_c for every canonical far c with c2 <= max_disp: plans of any shape whose far
// displacements stay within that reach index into it (ie_plan_create_shared) instead of
// generating blocks.  Blocks are generated as in a plan (FP64 site sums rounded to FP32,
// the 16-bit split images cut from them), ordered by c0, then c1, then c2.
#include <algorithm>
#include <chrono>

#include "ie_internal.h"

namespace ie {
namespace {

constexpr unsigned kBlockPrecs = IE_PRECMASK(IE_PREC_FP32) | IE_PRECMASK(IE_PREC_BF16X3) |
                                 IE_PRECMASK(IE_PREC_FP16X3) | IE_PRECMASK(IE_PREC_BF16X1) |
                                 IE_PRECMASK(IE_PREC_FP16X1);
constexpr unsigned kBf16Mask = IE_PRECMASK(IE_PREC_BF16X3) | IE_PRECMASK(IE_PREC_BF16X1);
constexpr unsigned kFp16Mask = IE_PRECMASK(IE_PREC_FP16X3) | IE_PRECMASK(IE_PREC_FP16X1);

ie_status check_spec(const ie_store_spec *sp) {
    if (!sp) return set_error("null store spec"), IE_ERR_INVALID;
    if (sp->lattice != kLattice) return set_error("lattice must be 4 (got %d)", sp->lattice), IE_ERR_INVALID;
    if (!(sp->k > 0) || !(sp->eta > 0) || !(sp->box_edge > 0))
        return set_error("k, eta and box_edge must be positive"), IE_ERR_INVALID;
    if (sp->max_disp < 2 || sp->max_disp > 1024)
        return set_error("max_disp %d outside [2, 1024]", sp->max_disp), IE_ERR_INVALID;
    if (sp->prec_mask == 0 || (sp->prec_mask & ~kBlockPrecs))
        return set_error("a store holds coupling-block precisions only (FP32, BF16X3/X1, FP16X3/X1)"),
               IE_ERR_INVALID;
    return IE_OK;
}

// canonical far triples c0 <= c1 <= c2 <= D, c2 >= 2
int64_t canon_count(int D) {
    const int64_t m = D + 1;
    return m * (m + 1) * (m + 2) / 6 - 4;   // all sorted triples minus the 4 with c2 <= 1
}

size_t store_bytes(const ie_store_spec *sp) {
    const int64_t nb = canon_count(sp->max_disp);
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
    add((size_t)nb * 3 * sizeof(int32_t));
    if (sp->prec_mask & IE_PRECMASK(IE_PREC_FP32))
        add((size_t)nb * kNU * kNU * sizeof(float2));
    else   // staging of the 16-bit images, freed before the store returns
        add((size_t)std::min<int64_t>(nb, kCouplingChunk) * kNU * kNU * sizeof(float2));
    if (sp->prec_mask & kBf16Mask) add((size_t)nb * kTcDispElems * sizeof(uint16_t));
    if (sp->prec_mask & kFp16Mask) {
        add((size_t)nb * kTcDispElems * sizeof(uint16_t));
        add((size_t)nb * sizeof(int32_t));
    }
    return b;
}

void store_free(ie_store s) {
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    cudaDeviceSynchronize();
    for (void *q : s->allocs) cudaFree(q);
    delete s;
}

template <class T>
ie_status salloc(ie_store s, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return IE_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    }
    s->allocs.push_back(*ptr);
    s->bytes += count * sizeof(T);
    return IE_OK;
}

}  // namespace

void store_retain(ie_store s) { s->refs.fetch_add(1); }

void store_release(ie_store s) {
    if (s->refs.fetch_sub(1) == 1) store_free(s);
}

}  // namespace ie

using namespace ie;

extern "C" {

ie_status ie_store_footprint(const ie_store_spec *spec, size_t *bytes) {
    IE_TRY(check_spec(spec));
    if (!bytes) return set_error("null bytes"), IE_ERR_INVALID;
    *bytes = store_bytes(spec);
    return IE_OK;
}

ie_status ie_store_create(const ie_store_spec *spec, void *stream, ie_store *out) {
    ie::NvtxRange nvtx_range("ie_store_create");
    auto t0 = std::chrono::steady_clock::now();
    if (!out) return set_error("null out"), IE_ERR_INVALID;
    *out = nullptr;
    IE_TRY(check_spec(spec));
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    cudaStream_t st = (cudaStream_t)stream;
    ie_store s = new ie_store_s();
    auto fail = [&](ie_status e) {
        store_free(s);
        return e;
    };
    s->k = spec->k;
    s->eta = spec->eta;
    s->a = spec->box_edge;
    s->max_disp = spec->max_disp;
    s->prec_mask = spec->prec_mask;
    const int D = spec->max_disp;
    s->index.assign((size_t)(D + 1) * (D + 1) * (D + 1), -1);
    for (int c0 = 0; c0 <= D; ++c0)
        for (int c1 = c0; c1 <= D; ++c1)
            for (int c2 = std::max(c1, 2); c2 <= D; ++c2) {
                s->index[((size_t)c0 * (D + 1) + c1) * (D + 1) + c2] = (int32_t)(s->canon.size() / 3);
                s->canon.insert(s->canon.end(), {c0, c1, c2});
            }
    s->n_blocks = (int64_t)s->canon.size() / 3;
    const int64_t nb = s->n_blocks;
    int32_t *d_canon = nullptr;
    ie_status e;
    if ((e = salloc(s, &d_canon, s->canon.size())) != IE_OK) return fail(e);
    if (cudaMemcpyAsync(d_canon, s->canon.data(), s->canon.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
        cudaGetLastError();
        set_error("store: upload of the canonical displacements failed");
        return fail(IE_ERR_CUDA);
    }
    if (s->prec_mask & IE_PRECMASK(IE_PREC_FP32))
        if ((e = salloc(s, &s->d_Csimt, (size_t)nb * kNU * kNU)) != IE_OK) return fail(e);
    if (s->prec_mask & kBf16Mask)
        if ((e = salloc(s, &s->d_Cbf16, (size_t)nb * kTcDispElems)) != IE_OK) return fail(e);
    if (s->prec_mask & kFp16Mask) {
        if ((e = salloc(s, &s->d_Cfp16, (size_t)nb * kTcDispElems)) != IE_OK) return fail(e);
        if ((e = salloc(s, &s->d_Cexp16, (size_t)nb)) != IE_OK) return fail(e);
    }
    if ((e = generate_blocks(s->k, s->eta, s->a, d_canon, nb, s->d_Csimt, s->d_Cbf16, s->d_Cfp16, s->d_Cexp16, st)) !=
        IE_OK)
        return fail(e);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        set_error("store: block generation failed");
        return fail(IE_ERR_CUDA);
    }
    s->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = s;
    return IE_OK;
}

ie_status ie_store_info(ie_store s, int64_t *n_blocks, size_t *bytes) {
    if (!s) return set_error("null store"), IE_ERR_INVALID;
    if (n_blocks) *n_blocks = s->n_blocks;
    if (bytes) *bytes = s->bytes;
    return IE_OK;
}

ie_status ie_store_release(ie_store s) {
    if (!s) return IE_OK;
    store_release(s);
    return IE_OK;
}

}  // extern "C"
