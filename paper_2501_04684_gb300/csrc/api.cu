// libie C ABI: plan construction (geometry, one-box-buffer split, displacement
// grouping, coupling-block and near-block generation) and the products.
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <atomic>
#include <unordered_set>

#include "ie_internal.h"

namespace ie {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char *last_error() { return g_err; }

static std::atomic<int64_t> g_launches{0};
static thread_local int g_capture_depth = 0;
void count_launches(int64_t n) {
    if (g_capture_depth == 0) g_launches += n;
}
void capture_begin() { g_capture_depth++; }
void capture_end() { g_capture_depth--; }

ie_status dalloc(ie_plan p, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return IE_OK;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    }
    p->allocs.push_back(*ptr);
    p->bytes += bytes;
    return IE_OK;
}

ie_status prepare_translate_simt();
ie_status prepare_translate_tc();
ie_status prepare_translate_cvfcnn();
ie_status prepare_cvfcnn_tc();

std::recursive_mutex &device_mutex() {
    static std::recursive_mutex mu;
    return mu;
}

ie_status prepare_kernels() {
    IE_TRY(prepare_translate_simt());
    IE_TRY(prepare_translate_tc());
    IE_TRY(prepare_translate_cvfcnn());
    IE_TRY(prepare_cvfcnn_tc());
    return IE_OK;
}

namespace {

bool wants_tc(unsigned mask) {
    return mask & (IE_PRECMASK(IE_PREC_BF16X3) | IE_PRECMASK(IE_PREC_FP16X3) | IE_PRECMASK(IE_PREC_BF16X1) |
                   IE_PRECMASK(IE_PREC_FP16X1));
}
bool wants_bf16(unsigned mask) {
    return mask & (IE_PRECMASK(IE_PREC_BF16X3) | IE_PRECMASK(IE_PREC_BF16X1));
}
bool wants_fp16(unsigned mask) { return mask & (IE_PRECMASK(IE_PREC_FP16X3) | IE_PRECMASK(IE_PREC_FP16X1)); }
// networks on the tensor cores (fp16 images) and / or on the SIMT cores (FP32)
bool wants_cvfcnn_tc(unsigned mask) { return mask & IE_PRECMASK(IE_PREC_CVFCNN); }
bool wants_cvfcnn(unsigned mask) { return mask & (IE_PRECMASK(IE_PREC_CVFCNN) | IE_PRECMASK(IE_PREC_CVFCNN_FP32)); }
// FP32 translation inputs are read by the FP32 block and network kernels
bool wants_x32(unsigned mask) { return mask & (IE_PRECMASK(IE_PREC_FP32) | IE_PRECMASK(IE_PREC_CVFCNN_FP32)); }
// split 16-bit translation inputs are read by the tensor-core block and network kernels
bool wants_split(unsigned mask) { return wants_tc(mask) || wants_cvfcnn_tc(mask); }
constexpr int kCvDefaultHidden = 50;   // the paper's H

ie_status validate(const ie_problem *pr) {
    if (!pr) return set_error("null problem"), IE_ERR_INVALID;
    if (pr->lattice != kLattice) return set_error("lattice must be 4 (got %d)", pr->lattice), IE_ERR_INVALID;
    if (pr->n_boxes < 1) return set_error("n_boxes must be >= 1"), IE_ERR_INVALID;
    if (!pr->box_ijk) return set_error("box_ijk is null"), IE_ERR_INVALID;
    if ((pr->P == nullptr) != (pr->nb == nullptr))
        return set_error("P and nb must both be given or both be null"), IE_ERR_INVALID;
    if (pr->max_rhs < 1 || pr->max_rhs > 64) return set_error("max_rhs must be in [1, 64]"), IE_ERR_INVALID;
    if (!(pr->k > 0) || !(pr->box_edge > 0) || !(pr->eta > 0))
        return set_error("k, eta and box_edge must be positive"), IE_ERR_INVALID;
    unsigned known = IE_PRECMASK(IE_PREC_FP32) | IE_PRECMASK(IE_PREC_BF16X3) | IE_PRECMASK(IE_PREC_FP16X3) |
                     IE_PRECMASK(IE_PREC_BF16X1) | IE_PRECMASK(IE_PREC_FP16X1) | IE_PRECMASK(IE_PREC_CVFCNN) |
                     IE_PRECMASK(IE_PREC_CVFCNN_FP32);
    if (pr->prec_mask == 0 || (pr->prec_mask & ~known)) return set_error("bad prec_mask"), IE_ERR_INVALID;
    if (wants_cvfcnn(pr->prec_mask) && (pr->cvfcnn_hidden < 0 || pr->cvfcnn_hidden > kCvHp))
        return set_error("cvfcnn_hidden %d outside [0, %d]", pr->cvfcnn_hidden, kCvHp), IE_ERR_INVALID;
    if (pr->self_box_mode != 0 && pr->self_box_mode != 1) return set_error("self_box_mode must be 0 or 1"), IE_ERR_INVALID;
    if (pr->symmetry != 0 && pr->symmetry != 1) return set_error("symmetry must be 0 or 1"), IE_ERR_INVALID;
    if (pr->group_nrhs) {
        if (!pr->box_group) return set_error("group_nrhs needs box_group"), IE_ERR_INVALID;
        for (int g = 0; g < pr->n_groups; ++g)
            if (pr->group_nrhs[g] < 1 || pr->group_nrhs[g] > pr->max_rhs)
                return set_error("group_nrhs[%d] = %d outside [1, %d]", g, pr->group_nrhs[g], pr->max_rhs),
                       IE_ERR_INVALID;
    }
    if (pr->nb)
        for (int b = 0; b < pr->n_boxes; ++b)
            if (pr->nb[b] < 1 || pr->nb[b] > kNU)
                return set_error("nb[%d] = %d outside [1,192]", b, pr->nb[b]), IE_ERR_INVALID;
    for (int b = 0; b < pr->n_boxes; ++b)
        for (int c = 0; c < 3; ++c) {
            int v = pr->box_ijk[3 * b + c];
            if (v < -(1 << 20) || v > (1 << 20)) return set_error("box index out of range"), IE_ERR_INVALID;
        }
    if (pr->box_group) {
        if (pr->n_groups < 1 || !pr->group_alpha)
            return set_error("box_group needs n_groups >= 1 and group_alpha"), IE_ERR_INVALID;
        for (int b = 0; b < pr->n_boxes; ++b) {
            int g = pr->box_group[b];
            if (g < 0 || g >= pr->n_groups) return set_error("box_group[%d] = %d out of range", b, g), IE_ERR_INVALID;
            if (b > 0 && g < pr->box_group[b - 1]) return set_error("box_group must be non-decreasing"), IE_ERR_INVALID;
        }
    } else if (pr->n_groups > 1) {
        return set_error("n_groups > 1 needs box_group"), IE_ERR_INVALID;
    }
    return IE_OK;
}

int group_of(const ie_problem *pr, int b) { return pr->box_group ? pr->box_group[b] : 0; }
int n_groups_of(const ie_problem *pr) { return pr->box_group ? pr->n_groups : 1; }

// Dense lookup of the occupied boxes over their bounding box, one layer per scatterer.
struct BoxGrid {
    int lo[3], ext[3];
    size_t cells = 0;
    std::vector<int32_t> slot;
    int at(int g, int x, int y, int z) const {
        x -= lo[0], y -= lo[1], z -= lo[2];
        if (x < 0 || y < 0 || z < 0 || x >= ext[0] || y >= ext[1] || z >= ext[2]) return -1;
        return slot[(size_t)g * cells + ((size_t)x * ext[1] + y) * ext[2] + z];
    }
};

ie_status build_grid(const ie_problem *pr, BoxGrid &g) {
    for (int c = 0; c < 3; ++c) {
        int lo = pr->box_ijk[c], hi = lo;
        for (int b = 0; b < pr->n_boxes; ++b) {
            lo = std::min(lo, (int)pr->box_ijk[3 * b + c]);
            hi = std::max(hi, (int)pr->box_ijk[3 * b + c]);
        }
        g.lo[c] = lo;
        g.ext[c] = hi - lo + 1;
    }
    g.cells = (size_t)g.ext[0] * g.ext[1] * g.ext[2];
    size_t ng = (size_t)n_groups_of(pr);
    if (g.cells * ng > ((size_t)1 << 28)) return set_error("box bounding grid too large"), IE_ERR_INVALID;
    g.slot.assign(g.cells * ng, -1);
    for (int b = 0; b < pr->n_boxes; ++b) {
        const int32_t *q = pr->box_ijk + 3 * b;
        size_t i = (size_t)group_of(pr, b) * g.cells +
                   ((size_t)(q[0] - g.lo[0]) * g.ext[1] + (q[1] - g.lo[1])) * g.ext[2] + (q[2] - g.lo[2]);
        if (g.slot[i] != -1) return set_error("duplicate box (%d,%d,%d)", q[0], q[1], q[2]), IE_ERR_INVALID;
        g.slot[i] = b;
    }
    return IE_OK;
}

// Far pairs (Chebyshev distance >= 2) by counting sort on the displacement.
// ---- symmetry of the cell-centred lattice (§2.2: blocks of displacements with the
// same sorted |d| are one matrix up to a signed permutation of the unknowns)
// Q = 8 * p + s: (Q c)_i = (-1)^{bit i of s} c_{kPerm[p][i]}.
const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Canonical c = |d| sorted ascending and the Q with Q c = d.
int canon_of(const int32_t d[3], int32_t c[3]) {
    const int ad[3] = {std::abs(d[0]), std::abs(d[1]), std::abs(d[2])};
    int ord[3] = {0, 1, 2};
    std::stable_sort(ord, ord + 3, [&](int x, int y) { return ad[x] < ad[y]; });
    int pi[3];
    for (int k = 0; k < 3; ++k) {
        c[k] = ad[ord[k]];
        pi[ord[k]] = k;
    }
    int pidx = 0;
    while (pidx < 5 && !(kPerm[pidx][0] == pi[0] && kPerm[pidx][1] == pi[1] && kPerm[pidx][2] == pi[2])) ++pidx;
    return 8 * pidx + (d[0] < 0 ? 1 : 0) + (d[1] < 0 ? 2 : 0) + (d[2] < 0 ? 4 : 0);
}

// map[Q][u], u = 3 site + a in the frame of c: U_Q(u) | 0x100 when negated, so that
// G_{Qc}[U(u)][U(v)] = sign(u) sign(v) G_c[u][v].  Site l maps to l' with
// l'_i = l_{p(i)} (s_i = +1) or 3 - l_{p(i)} (s_i = -1); component a to the axis i
// with p(i) = a, with sign s_i.
void symmetry_map(std::vector<uint16_t> &map) {
    map.assign((size_t)kSym * kNU, 0);
    for (int q = 0; q < kSym; ++q) {
        const int *pi = kPerm[q / 8];
        int sg[3], inv[3];
        for (int i = 0; i < 3; ++i) {
            sg[i] = ((q >> i) & 1) ? -1 : 1;
            inv[pi[i]] = i;
        }
        for (int site = 0; site < kSites; ++site) {
            const int l[3] = {site & 3, (site >> 2) & 3, site >> 4};
            int lp[3];
            for (int i = 0; i < 3; ++i) lp[i] = sg[i] > 0 ? l[pi[i]] : 3 - l[pi[i]];
            const int sp = lp[0] + 4 * lp[1] + 16 * lp[2];
            for (int a = 0; a < 3; ++a) {
                const int ap = inv[a];
                map[(size_t)q * kNU + 3 * site + a] = (uint16_t)((3 * sp + ap) | (sg[ap] < 0 ? 0x100 : 0));
            }
        }
    }
}

struct FarGroups {
    std::vector<int32_t> disp;       // n_d x 3
    std::vector<int64_t> start;      // n_d + 1
    std::vector<int32_t> src, dst;   // sorted by displacement, then source
};

void far_groups(const ie_problem *pr, const BoxGrid &g, bool fill, FarGroups &out, int64_t &npairs, int64_t &nd,
                int64_t *ncanon = nullptr) {
    int span[3] = {2 * g.ext[0] - 1, 2 * g.ext[1] - 1, 2 * g.ext[2] - 1};
    size_t nkeys = (size_t)span[0] * span[1] * span[2];
    std::vector<int64_t> count(nkeys + 1, 0);
    const int32_t *ijk = pr->box_ijk;
    int n = pr->n_boxes;
    // box range of each scatterer (ids are non-decreasing)
    std::vector<int> gend(n);
    for (int b = n - 1; b >= 0; --b) gend[b] = (b + 1 < n && group_of(pr, b + 1) == group_of(pr, b)) ? gend[b + 1] : b + 1;
    std::vector<int> gbeg(n);
    for (int b = 0; b < n; ++b) gbeg[b] = (b > 0 && group_of(pr, b - 1) == group_of(pr, b)) ? gbeg[b - 1] : b;
    auto key = [&](int dx, int dy, int dz) {
        return ((size_t)(dx + g.ext[0] - 1) * span[1] + (dy + g.ext[1] - 1)) * span[2] + (dz + g.ext[2] - 1);
    };
    for (int b = 0; b < n; ++b)
        for (int t = gbeg[b]; t < gend[b]; ++t) {
            int dx = ijk[3 * t] - ijk[3 * b], dy = ijk[3 * t + 1] - ijk[3 * b + 1], dz = ijk[3 * t + 2] - ijk[3 * b + 2];
            int ch = std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz)));
            if (ch >= 2) count[key(dx, dy, dz)]++;
        }
    npairs = 0;
    nd = 0;
    for (size_t k = 0; k < nkeys; ++k)
        if (count[k]) {
            npairs += count[k];
            nd++;
        }
    if (ncanon) {   // distinct sorted |d| among the displacements present
        const int E = std::max(g.ext[0], std::max(g.ext[1], g.ext[2]));
        std::vector<char> seen((size_t)E * E * E, 0);
        *ncanon = 0;
        for (size_t k = 0; k < nkeys; ++k)
            if (count[k]) {
                const int32_t d[3] = {(int32_t)(k / ((size_t)span[2] * span[1])) - (g.ext[0] - 1),
                                      (int32_t)((k / span[2]) % span[1]) - (g.ext[1] - 1),
                                      (int32_t)(k % span[2]) - (g.ext[2] - 1)};
                int32_t c[3];
                canon_of(d, c);
                char &f = seen[((size_t)c[0] * E + c[1]) * E + c[2]];
                if (!f) f = 1, ++*ncanon;
            }
    }
    if (!fill) return;
    out.disp.resize(3 * nd);
    out.start.resize(nd + 1);
    std::vector<int64_t> pos(nkeys, -1);
    int64_t s = 0, di = 0;
    for (size_t k = 0; k < nkeys; ++k)
        if (count[k]) {
            int dz = (int)(k % span[2]) - (g.ext[2] - 1);
            int dy = (int)((k / span[2]) % span[1]) - (g.ext[1] - 1);
            int dx = (int)(k / ((size_t)span[2] * span[1])) - (g.ext[0] - 1);
            out.disp[3 * di] = dx;
            out.disp[3 * di + 1] = dy;
            out.disp[3 * di + 2] = dz;
            out.start[di] = s;
            pos[k] = s;
            s += count[k];
            di++;
        }
    out.start[nd] = s;
    out.src.resize(npairs);
    out.dst.resize(npairs);
    for (int b = 0; b < n; ++b)
        for (int t = gbeg[b]; t < gend[b]; ++t) {
            int dx = ijk[3 * t] - ijk[3 * b], dy = ijk[3 * t + 1] - ijk[3 * b + 1], dz = ijk[3 * t + 2] - ijk[3 * b + 2];
            int ch = std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz)));
            if (ch >= 2) {
                int64_t &p = pos[key(dx, dy, dz)];
                out.src[p] = b;
                out.dst[p] = t;
                p++;
            }
        }
}

// Near pairs per target box a: sources b with Chebyshev distance <= 1.
void near_lists(const ie_problem *pr, const BoxGrid &g, const std::vector<int32_t> &nb, std::vector<int32_t> &start,
                std::vector<int32_t> &src, std::vector<int64_t> &boff, int64_t &elems) {
    int n = pr->n_boxes;
    start.assign(n + 1, 0);
    src.clear();
    boff.clear();
    elems = 0;
    for (int a = 0; a < n; ++a) {
        start[a] = (int32_t)src.size();
        const int32_t *q = pr->box_ijk + 3 * a;
        for (int ex = -1; ex <= 1; ++ex)
            for (int ey = -1; ey <= 1; ++ey)
                for (int ez = -1; ez <= 1; ++ez) {
                    if (pr->self_box_mode == 1 && ex == 0 && ey == 0 && ez == 0) continue;
                    int b = g.at(group_of(pr, a), q[0] - ex, q[1] - ey, q[2] - ez);
                    if (b < 0) continue;
                    src.push_back(b);
                    boff.push_back(elems);
                    elems += (int64_t)nb[a] * nb[b];
                }
    }
    start[n] = (int32_t)src.size();
}

size_t plan_bytes(const ie_problem *pr, int64_t n, int64_t npairs, int64_t nd, int64_t nnear, int64_t near_elems,
                  int64_t nblk, bool shared = false) {
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
    int64_t nbox = pr->n_boxes;
    if (pr->P) add((size_t)n * kNU * sizeof(float2));
    add(nbox * sizeof(int32_t));
    add((nbox + 1) * sizeof(int64_t));
    add(nbox * 3 * sizeof(int32_t));
    add(nd * 3 * sizeof(int32_t));
    add((nd + 1) * sizeof(int64_t));
    add(npairs * sizeof(int32_t));
    add(npairs * sizeof(int32_t));
    const bool sym = pr->symmetry == 1;
    const int64_t ncanon = nblk;   // canonical displacements
    if (!sym) nblk = nd;
    if (sym) {
        add(nd * 2 * sizeof(int32_t));                       // block and Q of each group
        add(npairs * sizeof(int32_t));                       // group of each pair
        add((size_t)kSym * kNU * sizeof(uint16_t));
        add(nblk * 3 * sizeof(int32_t));
        if (wants_x32(pr->prec_mask))                        // permuted FP32 inputs
            add((size_t)kSym * pr->max_rhs * nbox * kNU * sizeof(float2));
    }
    if (!shared) {   // the blocks themselves (a shared store holds them instead)
        if (pr->prec_mask & IE_PRECMASK(IE_PREC_FP32))
            add((size_t)nblk * kNU * kNU * sizeof(float2));
        else   // staging of the 16-bit images, freed before the plan returns
            add((size_t)std::min<int64_t>(nblk, kCouplingChunk) * kNU * kNU * sizeof(float2));
        if (wants_bf16(pr->prec_mask)) add((size_t)nblk * kTcDispElems * sizeof(uint16_t));
        if (wants_fp16(pr->prec_mask)) {
            add((size_t)nblk * kTcDispElems * sizeof(uint16_t));
            add(nblk * sizeof(int32_t));
        }
    }
    if (wants_cvfcnn(pr->prec_mask)) {
        add((size_t)nblk * kCvBlockElems * sizeof(float2));
        if (wants_cvfcnn_tc(pr->prec_mask)) {   // fp16 images and scales of every network
            add((size_t)nblk * cvfcnn_image_elems() * sizeof(uint16_t));
            add((size_t)nblk * 2 * sizeof(int32_t));
        }
        // FP64 fit scratch (block and right singular vectors) and, without the symmetric
        // store, the canonical networks before their expansion: freed before the plan returns
        add((size_t)std::min<int64_t>(ncanon, kCvFitChunk) * 2 * kNU * kNU * sizeof(double2));
        if (!sym) add((size_t)ncanon * kCvBlockElems * sizeof(float2));
    }
    add((nbox + 1) * sizeof(int32_t));
    add(nnear * sizeof(int32_t));
    add(nnear * sizeof(int64_t));
    add(near_elems * sizeof(float2));
    size_t col = (size_t)pr->max_rhs * nbox;
    add(col * kNU * sizeof(float2));                       // X
    add((size_t)kSlabs * col * kNU * sizeof(float2));      // slabs
    if (wants_split(pr->prec_mask)) {
        add((sym ? kSym : 1) * 2 * col * 2 * kNU * sizeof(uint16_t));
        add(col * sizeof(int32_t));
        add(col * sizeof(float));
    }
    add(sizeof(int) * 4);
    add((size_t)pr->max_rhs * n * sizeof(float2));         // tmp
    // work lists (generous: one item per pair per precision family)
    add((size_t)(npairs / 8 + nd + 1) * sizeof(WorkItem) * 4);
    return b;
}

}  // namespace

// Work list of one translation kernel for `nrhs`: every displacement group cut into
// runs of at most (tile columns / nrhs) pairs (the tensor-core kernel runs the three
// M-blocks of a run inside one item).  In order 1 the tensor-core list keeps
// displacement order, so that the tiles of one group (which share the group's coupling
// images) run at the same time on neighbouring CTAs of the persistent kernel's static
// round-robin; order 0 sorts runs by size (largest first).  The tensor-core tile width
// and order come from ie_plan_tune (default: the full tile width, order 1).
ie_status work_list(ie_plan p, bool tc, int nrhs, WorkList **out, int max_cols, bool pack) {
    auto &cache = tc ? p->tc_work : p->simt_work;
    int cols = tc ? tc_tile_columns() : simt_tile_columns(), order = 1;
    if (tc) {
        auto t = p->tc_tuned.find(nrhs);
        if (t != p->tc_tuned.end()) cols = t->second.first, order = t->second.second;
        if (max_cols > 0) cols = std::min(cols, max_cols);
    }
    pack = pack && p->sym && !p->h_pgroup.empty();
    const int key = tc ? ((nrhs * 1024 + cols) * 2 + order) * 2 + (pack ? 1 : 0) : nrhs * 2 + (pack ? 1 : 0);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = &it->second;
        if (tc)
            p->n_work_tc = it->second.n;
        else
            p->n_work_simt = it->second.n;
        return IE_OK;
    }
    if (nrhs > cols) return set_error("nrhs %d exceeds the tile width %d", nrhs, cols), IE_ERR_INVALID;
    if (g_capture_depth > 0)      // building a list allocates and copies synchronously
        return set_error("work list (nrhs %d, %d columns) missing at stream capture", nrhs, cols), IE_ERR_INVALID;
    // right-hand-side columns of a pair: the call's nrhs, or fewer for a scatterer that has fewer
    auto nr_of = [&](int64_t pair) {
        if (p->gnrhs.empty()) return nrhs;
        return std::min(nrhs, (int)p->gnrhs[p->box_group[p->h_src[pair]]]);
    };
    std::vector<WorkItem> items;
    auto emit = [&](int64_t d, int64_t q, int np, int nr) { items.push_back({(int32_t)d, (int32_t)q, np, 0, nr}); };
    // symmetric store, packed: the groups of one stored block are contiguous, and an item's
    // columns may come from several of them (each column carries its own group; `disp` is
    // the group of the item's first pair)
    int64_t d_step = 1;
    for (int64_t d = 0; d < p->n_far_disp; d += d_step) {
        int64_t d1 = d + 1;
        if (pack)
            while (d1 < p->n_far_disp && p->h_gcanon[d1] == p->h_gcanon[d]) ++d1;
        d_step = d1 - d;
        int64_t s = p->h_gstart[d], e = p->h_gstart[d1];
        // runs of pairs with the same column count (pairs of one scatterer are contiguous)
        int64_t q = s;
        while (q < e) {
            const int nr = nr_of(q);
            const int per = cols / nr;
            int np = 0;
            while (q + np < e && np < per && nr_of(q + np) == nr) ++np;
            emit(pack ? p->h_pgroup[q] : d, q, np, nr);
            q += np;
        }
    }
    if (tc && order == 0)
        std::stable_sort(items.begin(), items.end(),
                         [](const WorkItem &a, const WorkItem &b) { return a.npairs * a.nr > b.npairs * b.nr; });
    WorkList wl;
    wl.n = (int64_t)items.size();
    if (wl.n) {
        IE_TRY(dalloc_t(p, &wl.d_items, items.size()));
        IE_CK(cudaMemcpy(wl.d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    }
    if (tc)
        p->n_work_tc = wl.n;
    else
        p->n_work_simt = wl.n;
    cache[key] = wl;
    *out = &cache[key];
    return IE_OK;
}

ie_status generate_blocks(double k, double eta, double a, const int32_t *d_disp, int64_t nd, float2 *C32,
                          uint16_t *bf16, uint16_t *fp16, int32_t *exp16, cudaStream_t st) {
    if (nd <= 0) return IE_OK;
    const bool keep32 = C32 != nullptr;
    const int64_t chunk = keep32 ? nd : std::min<int64_t>(nd, kCouplingChunk);
    float2 *stage = C32;
    if (!keep32) IE_CK(cudaMallocAsync(&stage, (size_t)chunk * kNU * kNU * sizeof(float2), st));
    ie_status cst = IE_OK;
    for (int64_t d0 = 0; d0 < nd && cst == IE_OK; d0 += chunk) {
        const int64_t m = std::min(chunk, nd - d0);
        float2 *blk = keep32 ? C32 + d0 * kNU * kNU : stage;
        cst = launch_coupling_fp32(k, eta, a, d_disp + 3 * d0, m, blk, false, st);
        if (cst == IE_OK && bf16) cst = launch_coupling_tc(blk, m, bf16 + d0 * kTcDispElems, nullptr, false, st);
        if (cst == IE_OK && fp16) cst = launch_coupling_tc(blk, m, fp16 + d0 * kTcDispElems, exp16 + d0, true, st);
    }
    if (!keep32) cudaFreeAsync(stage, st);
    return cst;
}

bool block_prec_only(unsigned mask) { return !wants_cvfcnn(mask); }

ie_status work_list_for(ie_plan p, int prec, int nrhs, WorkList **out) {
    if (prec == IE_PREC_FP32 || prec == IE_PREC_CVFCNN_FP32) return work_list(p, false, nrhs, out, 0, /*pack=*/true);
    if (prec == IE_PREC_CVFCNN) return work_list(p, true, nrhs, out, cvfcnn_tc_tile_columns(), /*pack=*/true);
    return work_list(p, true, nrhs, out, 0, /*pack=*/true);
}

int canon_of_disp(const int32_t d[3], int32_t c[3]) { return canon_of(d, c); }
void symmetry_map_host(std::vector<uint16_t> &map) { symmetry_map(map); }

ie_status translate_timed(ie_plan p, int prec, const float2 *X, float2 *Yslab, int nrhs, cudaStream_t st,
                          const int *gate) {
    bool timed = false;
    if (p->profile) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        IE_CK(cudaStreamIsCapturing(st, &cs));
        timed = cs == cudaStreamCaptureStatusNone;
    }
    if (timed) IE_CK(cudaEventRecord(p->prof_ev[0], st));
    if (prec == IE_PREC_FP32)
        IE_TRY(launch_translate_simt(p, X, Yslab, nrhs, st, gate));
    else if (prec == IE_PREC_CVFCNN_FP32)
        IE_TRY(launch_translate_cvfcnn(p, X, Yslab, nrhs, st, gate));
    else if (prec == IE_PREC_CVFCNN)
        IE_TRY(launch_translate_cvfcnn_tc(p, Yslab, nrhs, st, gate));
    else
        IE_TRY(launch_translate_tc(p, prec, Yslab, nrhs, st, gate));
    if (timed) {
        IE_CK(cudaEventRecord(p->prof_ev[1], st));
        IE_CK(cudaEventSynchronize(p->prof_ev[1]));
        float ms = 0;
        IE_CK(cudaEventElapsedTime(&ms, p->prof_ev[0], p->prof_ev[1]));
        p->translate_ms += ms;
        p->translate_launches++;
    }
    return IE_OK;
}

ie_status far_product(ie_plan p, int prec, const float2 *c, float2 *y, int nrhs, bool accumulate, cudaStream_t st,
                      const int *gate) {
    size_t stride = slab_stride(p);
    IE_TRY(launch_aggregate(p, c, p->d_X, nrhs, st, gate));
    IE_TRY(launch_zero_slabs(p->d_Yslab, kSlabs, stride, (size_t)nrhs * p->nbox * kNU, st, gate));
    if (uses_split(prec)) IE_TRY(launch_split_tc(p, p->d_X, nrhs, is_fp16(prec), st, gate));
    IE_TRY(translate_timed(p, prec, p->d_X, p->d_Yslab, nrhs, st, gate));
    IE_TRY(launch_disaggregate(p, p->d_Yslab, kSlabs, stride, y, nrhs, accumulate, st, gate));
    return IE_OK;
}

ie_status take_device_error(ie_plan p, cudaStream_t st) {
    IE_CK(cudaStreamSynchronize(st));
    int w = 0;
    IE_CK(cudaMemcpy(&w, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (w == 0) return IE_OK;
    IE_CK(cudaMemset(p->d_err, 0, sizeof(int)));
    set_error("a translation kernel gave up a bounded wait (its result is incomplete)");
    return IE_ERR_TIMEOUT;
}

ie_status apply(ie_plan p, int which, int prec, const float2 *c, float2 *y, int nrhs, cudaStream_t st,
                const int *gate) {
    if (which == IE_FAR) return far_product(p, prec, c, y, nrhs, false, st, gate);
    IE_TRY(launch_near(p, c, y, nrhs, st, gate));
    if (which == IE_FULL) IE_TRY(far_product(p, prec, c, y, nrhs, true, st, gate));
    return IE_OK;
}

}  // namespace ie

using namespace ie;

static ie_status check_prec(ie_plan p, int prec) {
    if (prec < IE_PREC_FP32 || prec > IE_PREC_CVFCNN_FP32) return set_error("unknown precision %d", prec), IE_ERR_INVALID;
    if (!(p->prec_mask & IE_PRECMASK(prec)))
        return set_error("precision %d not prepared by this plan", prec), IE_ERR_UNSUPPORTED;
    return IE_OK;
}

static ie_status check_rhs(ie_plan p, int nrhs) {
    if (nrhs < 1 || nrhs > p->max_rhs) return set_error("nrhs %d outside [1, %d]", nrhs, p->max_rhs), IE_ERR_INVALID;
    return IE_OK;
}

extern "C" {

const char *ie_status_str(ie_status s) {
    switch (s) {
        case IE_OK: return "IE_OK";
        case IE_ERR_INVALID: return "IE_ERR_INVALID";
        case IE_ERR_OOM: return "IE_ERR_OOM";
        case IE_ERR_CUDA: return "IE_ERR_CUDA";
        case IE_ERR_NOT_CONVERGED: return "IE_ERR_NOT_CONVERGED";
        case IE_ERR_TIMEOUT: return "IE_ERR_TIMEOUT";
        case IE_ERR_UNSUPPORTED: return "IE_ERR_UNSUPPORTED";
    }
    return "IE_ERR_?";
}

const char *ie_last_error(void) { return last_error(); }
const char *ie_version(void) { return "libie 0.1 (sm_103a)"; }
int64_t ie_kernel_launches(void) { return g_launches.load(); }

ie_status ie_plan_footprint(const ie_problem *pr, size_t *bytes) {
    IE_TRY(validate(pr));
    if (!bytes) return set_error("null bytes"), IE_ERR_INVALID;
    BoxGrid g;
    IE_TRY(build_grid(pr, g));
    std::vector<int32_t> nb(pr->n_boxes);
    int64_t n = 0;
    for (int b = 0; b < pr->n_boxes; ++b) n += (nb[b] = pr->nb ? pr->nb[b] : kNU);
    FarGroups fg;
    int64_t npairs = 0, nd = 0, ncanon = 0;
    far_groups(pr, g, false, fg, npairs, nd,
               (pr->symmetry || wants_cvfcnn(pr->prec_mask)) ? &ncanon : nullptr);
    std::vector<int32_t> st, src;
    std::vector<int64_t> boff;
    int64_t elems = 0;
    near_lists(pr, g, nb, st, src, boff, elems);
    *bytes = plan_bytes(pr, n, npairs, nd, (int64_t)src.size(), elems, ncanon);
    return IE_OK;
}

}  // extern "C"

// What a shared store requires of a problem (before any far group is looked at).
static ie_status check_store(const ie_problem *pr, ie_store store) {
    if (pr->symmetry != 1)
        return set_error("a shared store serves symmetry-compressed plans (symmetry = 1)"), IE_ERR_UNSUPPORTED;
    if (wants_cvfcnn(pr->prec_mask))
        return set_error("the CVFCNN surrogates are fitted per plan: no shared store"), IE_ERR_UNSUPPORTED;
    if (pr->k != store->k || pr->eta != store->eta || pr->box_edge != store->a)
        return set_error("the store was built for another k, eta or box edge"), IE_ERR_INVALID;
    if (pr->prec_mask & ~store->prec_mask)
        return set_error("precisions 0x%x are not in the store (0x%x)", pr->prec_mask, store->prec_mask),
               IE_ERR_INVALID;
    return IE_OK;
}

static ie_status plan_create(const ie_problem *pr, ie_store store, void *stream, ie_plan *out) {
    ie::NvtxRange nvtx_range("ie_plan_create");
    auto t0 = std::chrono::steady_clock::now();
    if (!out) return set_error("null out"), IE_ERR_INVALID;
    *out = nullptr;
    IE_TRY(validate(pr));
    if (store) IE_TRY(check_store(pr, store));
    BoxGrid g;
    IE_TRY(build_grid(pr, g));
    IE_TRY(prepare_kernels());
    cudaStream_t st = (cudaStream_t)stream;

    ie_plan p = new ie_plan_s();
    if (store) {
        store_retain(store);
        p->store = store;
    }
    auto fail = [&](ie_status s) {
        ie_plan_destroy(p);
        return s;
    };
    p->k = pr->k;
    p->eta = pr->eta;
    p->a = pr->box_edge;
    p->alpha = pr->alpha;
    p->G = pr->grid_n;
    p->nbox = pr->n_boxes;
    p->self_mode = pr->self_box_mode;
    p->max_rhs = pr->max_rhs;
    p->prec_mask = pr->prec_mask;
    p->cv_hidden = wants_cvfcnn(pr->prec_mask) ? (pr->cvfcnn_hidden ? pr->cvfcnn_hidden : kCvDefaultHidden) : 0;
    p->identity = (pr->P == nullptr);
    p->ijk.assign(pr->box_ijk, pr->box_ijk + 3 * (size_t)pr->n_boxes);
    p->nb.resize(p->nbox);
    p->off.resize(p->nbox + 1);
    p->off[0] = 0;
    for (int b = 0; b < p->nbox; ++b) {
        p->nb[b] = pr->nb ? pr->nb[b] : kNU;
        p->off[b + 1] = p->off[b] + p->nb[b];
    }
    p->n = p->off[p->nbox];
    p->ngroups = n_groups_of(pr);
    p->gbox.assign(p->ngroups + 1, 0);
    p->galpha.assign(p->ngroups, pr->alpha);
    for (int b = 0; b < p->nbox; ++b) p->gbox[group_of(pr, b) + 1] = b + 1;
    for (int gi = 1; gi <= p->ngroups; ++gi) p->gbox[gi] = std::max(p->gbox[gi], p->gbox[gi - 1]);
    p->goff.resize(p->ngroups + 1);
    for (int gi = 0; gi <= p->ngroups; ++gi) p->goff[gi] = p->off[p->gbox[gi]];
    if (pr->box_group)
        for (int gi = 0; gi < p->ngroups; ++gi) p->galpha[gi] = pr->group_alpha[gi];
    if (pr->group_nrhs) p->gnrhs.assign(pr->group_nrhs, pr->group_nrhs + p->ngroups);
    p->box_group.resize(p->nbox);
    for (int b = 0; b < p->nbox; ++b) p->box_group[b] = group_of(pr, b);

    FarGroups fg;
    far_groups(pr, g, true, fg, p->n_far_pairs, p->n_far_disp);
    p->h_disp = fg.disp;
    p->h_gstart = fg.start;
    // stored blocks: one per displacement, or one per canonical displacement
    p->sym = pr->symmetry == 1;
    // canonical displacements (the symmetric store, and the networks' fits)
    std::vector<int32_t> gcanon, gsigma, canon_disp;
    if (p->sym || wants_cvfcnn(p->prec_mask)) {
        std::map<std::array<int32_t, 3>, int32_t> index;
        gcanon.resize(p->n_far_disp);
        gsigma.resize(p->n_far_disp);
        const int D = store ? store->max_disp : 0;
        for (int64_t d = 0; d < p->n_far_disp; ++d) {
            int32_t c[3];
            gsigma[d] = canon_of(&fg.disp[3 * d], c);
            if (store) {        // the store's block of c
                if (c[2] > D) {
                    set_error("far displacement |d| = (%d, %d, %d) beyond the store's reach %d", c[0], c[1], c[2], D);
                    return fail(IE_ERR_INVALID);
                }
                gcanon[d] = store->index[((size_t)c[0] * (D + 1) + c[1]) * (D + 1) + c[2]];
                continue;
            }
            auto ins = index.emplace(std::array<int32_t, 3>{c[0], c[1], c[2]}, (int32_t)index.size());
            if (ins.second) canon_disp.insert(canon_disp.end(), c, c + 3);
            gcanon[d] = ins.first->second;
        }
        if (store) canon_disp = store->canon;
    }
    if (p->sym && p->n_far_disp > 1) {
        // groups of one stored block next to each other (displacement order within a block),
        // so that a tensor-core item can take columns from several groups sharing its block
        const int64_t nd = p->n_far_disp;
        std::vector<int64_t> ord(nd);
        for (int64_t d = 0; d < nd; ++d) ord[d] = d;
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return gcanon[x] < gcanon[y]; });
        FarGroups r;
        r.disp.resize(fg.disp.size());
        r.start.resize(nd + 1);
        r.src.resize(fg.src.size());
        r.dst.resize(fg.dst.size());
        std::vector<int32_t> gc(nd), gs(nd);
        int64_t q = 0;
        for (int64_t k = 0; k < nd; ++k) {
            const int64_t d = ord[k];
            for (int c = 0; c < 3; ++c) r.disp[3 * k + c] = fg.disp[3 * d + c];
            r.start[k] = q;
            for (int64_t t = fg.start[d]; t < fg.start[d + 1]; ++t, ++q) {
                r.src[q] = fg.src[t];
                r.dst[q] = fg.dst[t];
            }
            gc[k] = gcanon[d];
            gs[k] = gsigma[d];
        }
        r.start[nd] = q;
        fg = std::move(r);
        gcanon.swap(gc);
        gsigma.swap(gs);
        p->h_disp = fg.disp;
        p->h_gstart = fg.start;
    }
    if (p->sym) {
        p->h_gcanon = gcanon;
        p->h_pgroup.resize(p->n_far_pairs);
        for (int64_t d = 0; d < p->n_far_disp; ++d)
            for (int64_t t = p->h_gstart[d]; t < p->h_gstart[d + 1]; ++t) p->h_pgroup[t] = (int32_t)d;
    }
    p->n_blocks = p->sym ? (int64_t)canon_disp.size() / 3 : p->n_far_disp;
    std::vector<int32_t> nstart, nsrc;
    std::vector<int64_t> nboff;
    near_lists(pr, g, p->nb, nstart, nsrc, nboff, p->near_elems);
    p->n_near_pairs = (int64_t)nsrc.size();

    ie_status s;
#define PT(expr)                   \
    do {                           \
        s = (expr);                \
        if (s != IE_OK) return fail(s); \
    } while (0)
#define PC(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_));     \
            return fail(IE_ERR_CUDA);                                                         \
        }                                                                                     \
    } while (0)

    // geometry and mapping
    PT(dalloc_t(p, &p->d_nb, p->nbox));
    PT(dalloc_t(p, &p->d_off, p->nbox + 1));
    PT(dalloc_t(p, &p->d_ijk, 3 * (size_t)p->nbox));
    PC(cudaMemcpyAsync(p->d_nb, p->nb.data(), p->nbox * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PC(cudaMemcpyAsync(p->d_off, p->off.data(), (p->nbox + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PC(cudaMemcpyAsync(p->d_ijk, p->ijk.data(), 3 * p->nbox * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    {
        std::vector<int32_t> bg(p->nbox);
        std::vector<double> ab(p->nbox);
        for (int b = 0; b < p->nbox; ++b) {
            bg[b] = group_of(pr, b);
            ab[b] = p->galpha[bg[b]];
        }
        PT(dalloc_t(p, &p->d_box_group, p->nbox));
        PT(dalloc_t(p, &p->d_alpha_box, p->nbox));
        PC(cudaMemcpy(p->d_box_group, bg.data(), p->nbox * sizeof(int32_t), cudaMemcpyHostToDevice));
        PC(cudaMemcpy(p->d_alpha_box, ab.data(), p->nbox * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (!p->identity) {
        std::vector<float2> P32((size_t)p->n * kNU);
        for (size_t i = 0; i < P32.size(); ++i) P32[i] = make_float2((float)pr->P[2 * i], (float)pr->P[2 * i + 1]);
        PT(dalloc_t(p, &p->d_P, P32.size()));
        PC(cudaMemcpyAsync(p->d_P, P32.data(), P32.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        PC(cudaStreamSynchronize(st));
    }

    // far groups and coupling blocks
    if (p->n_far_disp) {
        PT(dalloc_t(p, &p->d_disp, fg.disp.size()));
        PT(dalloc_t(p, &p->d_gstart, fg.start.size()));
        PT(dalloc_t(p, &p->d_src, fg.src.size()));
        PT(dalloc_t(p, &p->d_dst, fg.dst.size()));
        PC(cudaMemcpyAsync(p->d_disp, fg.disp.data(), fg.disp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        PC(cudaMemcpyAsync(p->d_gstart, p->h_gstart.data(), p->h_gstart.size() * sizeof(int64_t),
                           cudaMemcpyHostToDevice, st));
        PC(cudaMemcpyAsync(p->d_src, fg.src.data(), fg.src.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        PC(cudaMemcpyAsync(p->d_dst, fg.dst.data(), fg.dst.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        const int32_t *gen_disp = p->d_disp;
        if (p->sym) {
            std::vector<uint16_t> map;
            symmetry_map(map);
            PT(dalloc_t(p, &p->d_gcanon, gcanon.size()));
            PT(dalloc_t(p, &p->d_gsigma, gsigma.size()));
            PT(dalloc_t(p, &p->d_pgroup, p->h_pgroup.size()));
            PC(cudaMemcpy(p->d_pgroup, p->h_pgroup.data(), p->h_pgroup.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice));
            PT(dalloc_t(p, &p->d_symmap, map.size()));
            PT(dalloc_t(p, &p->d_canon_disp, canon_disp.size()));
            PC(cudaMemcpy(p->d_gcanon, gcanon.data(), gcanon.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            PC(cudaMemcpy(p->d_gsigma, gsigma.data(), gsigma.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            PC(cudaMemcpy(p->d_symmap, map.data(), map.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
            PC(cudaMemcpy(p->d_canon_disp, canon_disp.data(), canon_disp.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice));
            gen_disp = p->d_canon_disp;
            p->h_canon_disp = canon_disp;
        }
        const int64_t nd = p->n_blocks;
        if (store) {            // the shared store's blocks (the plan does not own them)
            p->d_Csimt = store->d_Csimt;
            p->d_Cbf16 = store->d_Cbf16;
            p->d_Cfp16 = store->d_Cfp16;
            p->d_Cexp16 = store->d_Cexp16;
        } else {
            if (wants_bf16(p->prec_mask)) PT(dalloc_t(p, &p->d_Cbf16, (size_t)nd * kTcDispElems));
            if (wants_fp16(p->prec_mask)) {
                PT(dalloc_t(p, &p->d_Cfp16, (size_t)nd * kTcDispElems));
                PT(dalloc_t(p, &p->d_Cexp16, (size_t)nd));
            }
            // FP32 blocks: the FP32 store itself, or (FP32 not requested) a bounded
            // staging buffer from which the 16-bit images are cut chunk by chunk
            if (p->prec_mask & IE_PRECMASK(IE_PREC_FP32)) PT(dalloc_t(p, &p->d_Csimt, (size_t)nd * kNU * kNU));
            PT(generate_blocks(p->k, p->eta, p->a, gen_disp, nd, p->d_Csimt, p->d_Cbf16, p->d_Cfp16, p->d_Cexp16,
                               st));
        }
        if (wants_cvfcnn(p->prec_mask)) {
            const int64_t ncanon = (int64_t)canon_disp.size() / 3;
            if (p->sym) {
                PT(launch_cvfcnn_fit(p, p->d_canon_disp, ncanon, nullptr, nullptr, nullptr, st));
            } else {   // fit each canonical displacement once, then turn it into every frame
                std::vector<uint16_t> map;
                symmetry_map(map);
                int32_t *d_cd = nullptr, *d_gc = nullptr, *d_gs = nullptr;
                uint16_t *d_map = nullptr;
                cudaError_t ce = cudaMallocAsync(&d_cd, canon_disp.size() * sizeof(int32_t), st);
                if (ce == cudaSuccess) ce = cudaMallocAsync(&d_gc, gcanon.size() * sizeof(int32_t), st);
                if (ce == cudaSuccess) ce = cudaMallocAsync(&d_gs, gsigma.size() * sizeof(int32_t), st);
                if (ce == cudaSuccess) ce = cudaMallocAsync(&d_map, map.size() * sizeof(uint16_t), st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(d_cd, canon_disp.data(), canon_disp.size() * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(d_gc, gcanon.data(), gcanon.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(d_gs, gsigma.data(), gsigma.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(d_map, map.data(), map.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st);
                ie_status fs = IE_OK;
                if (ce == cudaSuccess) {
                    fs = launch_cvfcnn_fit(p, d_cd, ncanon, d_gc, d_gs, d_map, st);
                } else {
                    cudaGetLastError();
                    set_error("CVFCNN fit set-up: %s", cudaGetErrorString(ce));
                    fs = IE_ERR_CUDA;
                }
                for (void *ptr : {(void *)d_cd, (void *)d_gc, (void *)d_gs, (void *)d_map})
                    if (ptr) cudaFreeAsync(ptr, st);
                PT(fs);
            }
            if (wants_cvfcnn_tc(p->prec_mask)) {
                PT(dalloc_t(p, &p->d_cvimg, (size_t)p->n_blocks * cvfcnn_image_elems()));
                PT(dalloc_t(p, &p->d_cvexp, (size_t)p->n_blocks * 2));
                PT(build_cvfcnn_images(p, st));
            }
        }
    }

    // host copy of the pairs' source boxes: per-scatterer column counts cut the work lists
    if (!p->gnrhs.empty()) {
        PC(cudaStreamSynchronize(st));   // the upload of fg.src has completed
        p->h_src = std::move(fg.src);
    }

    // near blocks
    PT(dalloc_t(p, &p->d_near_start, nstart.size()));
    PC(cudaMemcpyAsync(p->d_near_start, nstart.data(), nstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (p->n_near_pairs) {
        PT(dalloc_t(p, &p->d_near_src, nsrc.size()));
        PT(dalloc_t(p, &p->d_near_boff, nboff.size()));
        PT(dalloc_t(p, &p->d_Nblk, (size_t)p->near_elems));
        PC(cudaMemcpyAsync(p->d_near_src, nsrc.data(), nsrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        PC(cudaMemcpyAsync(p->d_near_boff, nboff.data(), nboff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        PT(launch_near_blocks(p, st));
    }

    // scratch
    size_t col = (size_t)p->max_rhs * p->nbox;
    PT(dalloc_t(p, &p->d_X, col * kNU));
    PT(dalloc_t(p, &p->d_Yslab, (size_t)kSlabs * col * kNU));
    if (wants_split(p->prec_mask)) {
        PT(dalloc_t(p, &p->d_Xtc, (size_t)(p->sym ? kSym : 1) * 2 * col * 2 * kNU));
        PT(dalloc_t(p, &p->d_Xexp, col));
        PT(dalloc_t(p, &p->d_Xinf, col));
    }
    if (p->sym && wants_x32(p->prec_mask)) PT(dalloc_t(p, &p->d_Xsym, (size_t)kSym * col * kNU));
    PT(dalloc_t(p, &p->d_err, 4));
    PC(cudaMemsetAsync(p->d_err, 0, 4 * sizeof(int), st));
    PT(dalloc_t(p, &p->d_tmp, (size_t)p->max_rhs * p->n));
    PC(cudaStreamSynchronize(st));
    PC(cudaGetLastError());
    int dev = 0;
    PC(cudaGetDevice(&dev));
    PC(cudaDeviceGetAttribute(&p->tc_sms, cudaDevAttrMultiProcessorCount, dev));
    p->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return IE_OK;
#undef PT
#undef PC
}

extern "C" {

ie_status ie_sym_canon(const int32_t *d, int32_t *c, int32_t *q) {
    if (!d || !c || !q) return set_error("null argument"), IE_ERR_INVALID;
    *q = canon_of_disp(d, c);
    return IE_OK;
}

ie_status ie_sym_map(uint16_t *out) {
    if (!out) return set_error("null argument"), IE_ERR_INVALID;
    std::vector<uint16_t> map;
    symmetry_map_host(map);
    std::copy(map.begin(), map.end(), out);
    return IE_OK;
}

ie_status ie_plan_create(const ie_problem *pr, void *stream, ie_plan *out) {
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    return plan_create(pr, nullptr, stream, out);
}

ie_status ie_plan_create_shared(const ie_problem *pr, ie_store store, void *stream, ie_plan *out) {
    if (!store) return set_error("null store"), IE_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    return plan_create(pr, store, stream, out);
}

ie_status ie_plan_footprint_shared(const ie_problem *pr, ie_store store, size_t *bytes) {
    if (!store || !bytes) return set_error("null argument"), IE_ERR_INVALID;
    IE_TRY(validate(pr));
    IE_TRY(check_store(pr, store));
    BoxGrid g;
    IE_TRY(build_grid(pr, g));
    std::vector<int32_t> nb(pr->n_boxes);
    int64_t n = 0;
    for (int b = 0; b < pr->n_boxes; ++b) n += (nb[b] = pr->nb ? pr->nb[b] : kNU);
    FarGroups fg;
    int64_t npairs = 0, nd = 0;
    far_groups(pr, g, false, fg, npairs, nd, nullptr);
    std::vector<int32_t> st, src;
    std::vector<int64_t> boff;
    int64_t elems = 0;
    near_lists(pr, g, nb, st, src, boff, elems);
    *bytes = plan_bytes(pr, n, npairs, nd, (int64_t)src.size(), elems, store->n_blocks, true);
    return IE_OK;
}

ie_status ie_plan_tune(ie_plan p, int prec, int nrhs, ie_tune_info *info, void *stream) {
    ie::NvtxRange nvtx_range("ie_plan_tune");
    if (!p) return set_error("null plan"), IE_ERR_INVALID;
    IE_TRY(check_prec(p, prec));
    IE_TRY(check_rhs(p, nrhs));
    if (!is_tc(prec)) return set_error("only the tensor-core translation has a tuned tile"), IE_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    // timing input: zero fields split into the 16-bit planes (the kernel's work does not
    // depend on the values)
    IE_TRY(launch_zero(p->d_X, (size_t)nrhs * p->nbox * kNU * sizeof(float2), st));
    IE_TRY(launch_split_tc(p, p->d_X, nrhs, is_fp16(prec), st));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    IE_CK(cudaEventCreate(&ev[0]));
    IE_CK(cudaEventCreate(&ev[1]));
    const int cands[] = {96, 80, 64, 48};
    std::pair<int, int> best{tc_tile_columns(), 1};
    double best_ms = 1e30, default_ms = 0;
    int tried = 0;
    ie_status e = IE_OK;
    for (int cols : cands) {
        if (cols > tc_tile_columns() || cols < nrhs) continue;
        for (int order = 0; order < 2 && e == IE_OK; ++order) {
            p->tc_tuned[nrhs] = {cols, order};
            e = launch_translate_tc(p, prec, p->d_Yslab, nrhs, st, nullptr);   // builds the list, warms up
            if (e != IE_OK) break;
            if (cudaEventRecord(ev[0], st) != cudaSuccess) e = IE_ERR_CUDA;
            for (int r = 0; r < 2 && e == IE_OK; ++r) e = launch_translate_tc(p, prec, p->d_Yslab, nrhs, st, nullptr);
            float ms = 0;
            if (e == IE_OK && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess))
                e = IE_ERR_CUDA;
            if (e != IE_OK) break;
            ms *= 0.5f;
            ++tried;
            if (cols == tc_tile_columns() && order == 1) default_ms = ms;
            if (ms < best_ms) best_ms = ms, best = {cols, order};
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != IE_OK) {
        p->tc_tuned.erase(nrhs);
        if (e == IE_ERR_CUDA) set_error("ie_plan_tune: timing failed");
        return e;
    }
    p->tc_tuned[nrhs] = best;
    IE_TRY(take_device_error(p, st));
    if (info) {
        info->tile_columns = best.first;
        info->order = best.second;
        info->ms = best_ms;
        info->default_ms = default_ms;
        info->candidates = tried;
    }
    return IE_OK;
}

ie_status ie_plan_check(ie_plan p, void *stream) {
    if (!p) return set_error("null plan"), IE_ERR_INVALID;
    return take_device_error(p, (cudaStream_t)stream);
}

ie_status ie_diag_bounded_wait(double limit_ms, void *stream) {
    if (!(limit_ms > 0) || limit_ms > 10000) return set_error("limit_ms must be in (0, 10000]"), IE_ERR_INVALID;
    return bounded_wait_selftest(limit_ms, (cudaStream_t)stream);
}

ie_status ie_plan_stats_get(ie_plan p, ie_plan_stats *o) {
    if (!p || !o) return set_error("null argument"), IE_ERR_INVALID;
    o->n_boxes = p->nbox;
    o->n = p->n;
    o->n_far_pairs = p->n_far_pairs;
    o->n_far_disp = p->n_far_disp;
    o->n_near_pairs = p->n_near_pairs;
    o->n_work_simt = p->n_work_simt;
    o->n_work_tc = p->n_work_tc;
    o->device_bytes = p->bytes;
    o->plan_seconds = p->plan_seconds;
    o->translate_ms = p->translate_ms;
    o->translate_launches = p->translate_launches;
    o->n_groups = p->ngroups;
    o->max_rhs = p->max_rhs;
    o->n_coupling_blocks = p->n_blocks;
    o->cvfcnn_hidden = p->cv_hidden;
    o->cvfcnn_sweeps = p->cv_sweeps;
    o->cvfcnn_tail = p->cv_tail;
    return IE_OK;
}

ie_status ie_plan_profile(ie_plan p, int enable) {
    if (!p) return set_error("null plan"), IE_ERR_INVALID;
    if (enable && !p->prof_ev[0]) {
        IE_CK(cudaEventCreate(&p->prof_ev[0]));
        IE_CK(cudaEventCreate(&p->prof_ev[1]));
    }
    p->profile = enable ? 1 : 0;
    if (enable) {
        p->translate_ms = 0;
        p->translate_launches = 0;
    }
    return IE_OK;
}

ie_status ie_plan_destroy(ie_plan p) {
    if (!p) return IE_OK;
    std::lock_guard<std::recursive_mutex> lock(device_mutex());
    cudaDeviceSynchronize();
    destroy_cached_solvers(p);
    for (void *q : p->allocs) cudaFree(q);
    for (auto &e : p->prof_ev)
        if (e) cudaEventDestroy(e);
    if (p->store) store_release(p->store);
    delete p;
    return IE_OK;
}

ie_status ie_matvec(ie_plan p, int which, int prec, const void *c, void *y, int nrhs, void *stream) {
    ie::NvtxRange nvtx_range("ie_matvec");
    if (!p || !c || !y) return set_error("null argument"), IE_ERR_INVALID;
    if (which < IE_FAR || which > IE_FULL) return set_error("bad which %d", which), IE_ERR_INVALID;
    IE_TRY(check_rhs(p, nrhs));
    if (which != IE_NEAR) IE_TRY(check_prec(p, prec));
    if (c == y) return set_error("c and y must not alias"), IE_ERR_INVALID;
    return apply(p, which, prec, (const float2 *)c, (float2 *)y, nrhs, (cudaStream_t)stream);
}

ie_status ie_aggregate(ie_plan p, const void *c, void *X, int nrhs, void *stream) {
    if (!p || !c || !X) return set_error("null argument"), IE_ERR_INVALID;
    IE_TRY(check_rhs(p, nrhs));
    return launch_aggregate(p, (const float2 *)c, (float2 *)X, nrhs, (cudaStream_t)stream);
}

ie_status ie_translate(ie_plan p, int prec, const void *X, void *Y, int nrhs, void *stream) {
    ie::NvtxRange nvtx_range("ie_translate");
    if (!p || !X || !Y) return set_error("null argument"), IE_ERR_INVALID;
    IE_TRY(check_rhs(p, nrhs));
    IE_TRY(check_prec(p, prec));
    cudaStream_t st = (cudaStream_t)stream;
    size_t stride = slab_stride(p);
    IE_TRY(launch_zero_slabs(p->d_Yslab, kSlabs, stride, (size_t)nrhs * p->nbox * kNU, st));
    if (uses_split(prec)) IE_TRY(launch_split_tc(p, (const float2 *)X, nrhs, is_fp16(prec), st));
    IE_TRY(translate_timed(p, prec, (const float2 *)X, p->d_Yslab, nrhs, st, nullptr));
    return launch_sum_slabs(p, p->d_Yslab, kSlabs, stride, (float2 *)Y, nrhs, st);
}

ie_status ie_disaggregate(ie_plan p, const void *Y, void *r, int nrhs, void *stream) {
    if (!p || !Y || !r) return set_error("null argument"), IE_ERR_INVALID;
    IE_TRY(check_rhs(p, nrhs));
    return launch_disaggregate(p, (const float2 *)Y, 1, 0, (float2 *)r, nrhs, false, (cudaStream_t)stream);
}

ie_status ie_near(ie_plan p, const void *c, void *y, int nrhs, void *stream) {
    if (!p || !c || !y) return set_error("null argument"), IE_ERR_INVALID;
    IE_TRY(check_rhs(p, nrhs));
    return launch_near(p, (const float2 *)c, (float2 *)y, nrhs, (cudaStream_t)stream);
}

ie_status ie_plan_blocks(ie_plan p, int32_t *disp) {
    if (!p || !disp) return set_error("null argument"), IE_ERR_INVALID;
    const std::vector<int32_t> &src = p->sym ? p->h_canon_disp : p->h_disp;
    std::copy(src.begin(), src.end(), disp);
    return IE_OK;
}

ie_status ie_coupling_blocks(ie_plan p, const int32_t *d, int nd, void *outp, void *stream) {
    if (!p || !d || !outp || nd < 0) return set_error("bad argument"), IE_ERR_INVALID;
    if (nd == 0) return IE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *dd = nullptr;
    IE_CK(cudaMallocAsync(&dd, (size_t)nd * 3 * sizeof(int32_t), st));
    IE_CK(cudaMemcpyAsync(dd, d, (size_t)nd * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    IE_TRY(launch_coupling_simt(p, dd, nd, (float2 *)outp, true, st));
    IE_CK(cudaFreeAsync(dd, st));
    return IE_OK;
}

ie_status ie_rhs_plane_wave(ie_plan p, const double *khat, const double *pol, int nrhs, void *v, void *stream) {
    if (!p || !khat || !pol || !v) return set_error("null argument"), IE_ERR_INVALID;
    if (nrhs < 1 || nrhs > p->max_rhs) return set_error("nrhs %d outside [1, %d]", nrhs, p->max_rhs), IE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    double *dk = nullptr;
    size_t cnt = (size_t)p->ngroups * nrhs * 3;       // [group][rhs][3]
    IE_CK(cudaMallocAsync(&dk, cnt * 2 * sizeof(double), st));
    IE_CK(cudaMemcpyAsync(dk, khat, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
    IE_CK(cudaMemcpyAsync(dk + cnt, pol, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
    IE_TRY(launch_plane_wave(p, dk, dk + cnt, nrhs, (float2 *)v, st));
    IE_CK(cudaFreeAsync(dk, st));
    return IE_OK;
}

}  // extern "C"
