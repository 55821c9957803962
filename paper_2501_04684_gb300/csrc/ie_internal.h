// Internal declarations of libie (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ie.h"

namespace ie {

// Host-side NVTX range for the duration of a scope (seen by Nsight tools; a no-op
// without one attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


constexpr int kLattice = 4;
constexpr int kSites = 64;          // 4^3 dipole sites per box
constexpr int kNU = 192;            // 3 unknowns per site
constexpr int kSlabs = 8;           // FP32 partial-sum slabs of the far field (see translate_simt.cu)
// Precisions whose products read fp16 split inputs (power-of-two column scaling).
inline bool is_fp16(int prec) { return prec == IE_PREC_FP16X3 || prec == IE_PREC_FP16X1 || prec == IE_PREC_CVFCNN; }
// Precisions whose translation is the block product on the tensor cores.
inline bool is_tc(int prec) { return prec >= IE_PREC_BF16X3 && prec <= IE_PREC_FP16X1; }
// Precisions whose translation reads the split 16-bit inputs (block products and networks
// on the tensor cores); their work lists are the tensor-core ones.
inline bool uses_split(int prec) { return is_tc(prec) || prec == IE_PREC_CVFCNN; }
constexpr int kSym = 48;             // signed permutations of the three axes
constexpr int64_t kCouplingChunk = 4096;   // displacements per staging chunk of the 16-bit coupling images

// CVFCNN surrogate weights of one stored block, complex64, hidden width padded to
// kCvHp (padding rows / columns zero): W1^T [192][kCvHp], b1 [kCvHp], W2^T [kCvHp][192],
// b2 [192] (the transposes are the operand layouts of the two SIMT GEMMs).
constexpr int kCvHp = 64;
constexpr size_t kCvW1 = 0;
constexpr size_t kCvB1 = kCvW1 + (size_t)kNU * kCvHp;
constexpr size_t kCvW2 = kCvB1 + kCvHp;
constexpr size_t kCvB2 = kCvW2 + (size_t)kCvHp * kNU;
constexpr size_t kCvBlockElems = kCvB2 + kNU;
constexpr int64_t kCvFitChunk = 512;   // blocks per fit pass (two FP64 192 x 192 scratch matrices each)

// Tensor-core store of one coupling block: 3 M-blocks (128 real-embedded rows) x
// 6 K-chunks (32 source unknowns) x {hi, lo}, each a 128 x 32 16-bit image laid out
// exactly as the 64-byte-swizzled K-major shared-memory operand of tcgen05.mma (8 KB).
constexpr int kTcK = 32;
constexpr int kTcKChunks = kNU / kTcK;                          // 6
constexpr int kTcImageElems = 128 * kTcK;
constexpr int kTcImagesPerDisp = 3 * kTcKChunks * 2;            // 36
constexpr size_t kTcDispElems = (size_t)kTcImageElems * kTcImagesPerDisp;   // 147,456

// D(R) of eq. 5 with psi of eq. 6, FP64.  out[3*i+j] = D_ij.
__device__ inline void dyad_fp64(double k, double eta, double Rx, double Ry, double Rz, double2 out[9]) {
    constexpr double kPi = 3.14159265358979323846;
    double r = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
    double kr = k * r;
    double s, c;
    sincos(kr, &s, &c);
    double sc = k * eta / (4.0 * kPi * r);
    double psi_re = -sc * s, psi_im = -sc * c;          // -j k eta e^{-jkr} / (4 pi r)
    double ikr = 1.0 / kr, ikr2 = ikr * ikr;
    double a_re = 1.0 - ikr2, a_im = -ikr;              // 1 - j/kr - 1/kr^2
    double b_re = 1.0 - 3.0 * ikr2, b_im = -3.0 * ikr;  // 1 - 3j/kr - 3/kr^2
    double rh[3] = {Rx / r, Ry / r, Rz / r};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double t_re = (i == j ? a_re : 0.0) - rh[i] * rh[j] * b_re;
            double t_im = (i == j ? a_im : 0.0) - rh[i] * rh[j] * b_im;
            out[3 * i + j] = make_double2(psi_re * t_re - psi_im * t_im, psi_re * t_im + psi_im * t_re);
        }
}

void set_error(const char *fmt, ...);
const char *last_error();

// Process-wide count of kernels this library has put on the GPU (direct launches
// plus the kernel nodes of every graph replay); captures do not count.
void count_launches(int64_t n);
void capture_begin();
void capture_end();

#define IE_CK(call)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::ie::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return IE_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

#define IE_CK_LAUNCH()                                                                 \
    do {                                                                               \
        ::ie::count_launches(1);                                                       \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            ::ie::set_error("%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            return IE_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

#define IE_TRY(expr)                                                                   \
    do {                                                                               \
        ie_status s_ = (expr);                                                         \
        if (s_ != IE_OK) return s_;                                                    \
    } while (0)

// Work item of the translation kernels: one displacement group, a run of its pairs.
struct WorkItem {
    int32_t disp;        // index of the displacement (coupling block)
    int32_t pair0;       // first pair (global index into src/dst)
    int32_t npairs;      // pairs in this item (x nrhs columns)
    int32_t mb;          // unused (0)
    int32_t nr;          // right-hand-side columns of each pair (the call's nrhs, or fewer for
                         // scatterers with fewer right-hand sides)
};

struct WorkList {
    WorkItem *d_items = nullptr;
    int64_t n = 0;
};

}  // namespace ie

// A coupling-block store shared by plans (ie_store_create): the canonical far blocks of
// every displacement with |d_i| <= max_disp, in the precisions of prec_mask.
struct ie_store_s {
    double k = 0, eta = 0, a = 0;
    int max_disp = 0;
    unsigned prec_mask = 0;
    int64_t n_blocks = 0;
    std::vector<int32_t> canon;        // [n_blocks][3] sorted |d|
    std::vector<int32_t> index;        // [(max_disp + 1)^3] canonical triple -> block, -1 if near
    float2 *d_Csimt = nullptr;         // FP32 blocks (IE_PREC_FP32)
    uint16_t *d_Cbf16 = nullptr, *d_Cfp16 = nullptr;
    int32_t *d_Cexp16 = nullptr;
    std::vector<void *> allocs;
    size_t bytes = 0;
    double seconds = 0;
    std::atomic<int> refs{1};
};

struct ie_plan_s {
    // problem constants
    double k = 0, eta = 0, a = 0, alpha = 0;
    int G = 0, nbox = 0, self_mode = 0, max_rhs = 1;
    unsigned prec_mask = 0;
    bool identity = false;
    int64_t n = 0;                     // basis unknowns
    // scatterers of a batched plan (one group otherwise): box and unknown ranges
    int ngroups = 1;
    std::vector<int64_t> gbox, goff;   // ngroups + 1 each
    std::vector<double> galpha;        // ngroups
    int32_t *d_box_group = nullptr;    // [nbox]
    double *d_alpha_box = nullptr;     // [nbox] self term of each box's scatterer
    std::vector<int32_t> gnrhs;        // ngroups right-hand sides per scatterer (empty: all)
    std::vector<int32_t> box_group;    // nbox scatterer of each box
    std::vector<int32_t> h_src;        // source box of every far pair (kept only with gnrhs)
    std::vector<int32_t> ijk, nb;
    std::vector<int64_t> off;          // nbox + 1

    // device geometry and mapping
    int32_t *d_nb = nullptr;
    int64_t *d_off = nullptr;
    int32_t *d_ijk = nullptr;
    float2 *d_P = nullptr;             // [n][192] complex64 (null for identity)

    // far zone, grouped by displacement
    int64_t n_far_disp = 0, n_far_pairs = 0;
    std::vector<int32_t> h_disp;       // n_far_disp x 3
    std::vector<int64_t> h_gstart;     // n_far_disp + 1 (pair offsets)
    int64_t *d_gstart = nullptr;       // n_far_disp + 1, device copy of h_gstart
    int32_t *d_disp = nullptr;         // n_far_disp x 3
    int32_t *d_src = nullptr, *d_dst = nullptr;   // [n_far_pairs], sorted by displacement
    float2 *d_Csimt = nullptr;         // [n_far_disp][192 (k)][192 (m)] complex64
    uint16_t *d_Cbf16 = nullptr;       // [n_far_disp][kTcDispElems] bf16 images
    uint16_t *d_Cfp16 = nullptr;       // [n_far_disp][kTcDispElems] fp16 images
    int32_t *d_Cexp16 = nullptr;       // [n_far_disp] power-of-two scale of the fp16 images
    // symmetry-compressed store (symmetry = 1): the block stores above then hold one
    // block per canonical displacement c = sorted |d| (n_blocks of them)
    bool sym = false;
    int64_t n_blocks = 0;              // stored far blocks (n_far_disp without symmetry)
    int32_t *d_gcanon = nullptr;       // [n_far_disp] stored block of each displacement group
    std::vector<int32_t> h_gcanon;     // host copy (symmetric store: groups ordered by block)
    int32_t *d_pgroup = nullptr;       // [n_far_pairs] group of each pair (symmetric store)
    std::vector<int32_t> h_pgroup;
    int32_t *d_gsigma = nullptr;       // [n_far_disp] signed permutation Q (0..47) with Q c = d
    uint16_t *d_symmap = nullptr;      // [48][192] u -> U(u) | 0x100 when negated (G_d[U(u)][U(v)] = +-G_c[u][v])
    int32_t *d_canon_disp = nullptr;   // [n_blocks x 3]
    std::vector<int32_t> h_canon_disp; // host copy
    float2 *d_Xsym = nullptr;          // [48][max_rhs][nbox][192] signed-permuted FP32 translation inputs
    // CVFCNN surrogates (IE_PREC_CVFCNN), one network per stored block
    int cv_hidden = 0;
    int cv_trained = 0;                // 1 once ie_cvfcnn_train has replaced the closed-form weights
    int cv_sweeps = 0;
    double cv_tail = 0;
    float2 *d_cvW = nullptr;           // [n_blocks][kCvBlockElems]
    uint16_t *d_cvimg = nullptr;       // [n_blocks][12 images] fp16 networks for the tensor cores
    int32_t *d_cvexp = nullptr;        // [n_blocks][2] power-of-two scales of the two layers' images

    // near zone: per target box a run of (source box, block offset)
    int64_t n_near_pairs = 0;
    int64_t near_elems = 0;
    int32_t *d_near_start = nullptr;   // nbox + 1
    int32_t *d_near_src = nullptr;     // n_near_pairs
    int64_t *d_near_boff = nullptr;    // n_near_pairs (element offset into d_Nblk)
    float2 *d_Nblk = nullptr;          // blocks, nb_a x nb_b column-major each

    // scratch (sized for max_rhs)
    float2 *d_X = nullptr;             // [max_rhs][nbox][192]
    float2 *d_Yslab = nullptr;         // [kSlabs][max_rhs][nbox][192]
    uint16_t *d_Xtc = nullptr;         // [48 with symmetry][2 hl][max_rhs][nbox][6 chunk][2 reim][32] 16-bit
    int32_t *d_Xexp = nullptr;         // [max_rhs][nbox] power-of-two scale of d_Xtc columns
    float *d_Xinf = nullptr;           // [max_rhs][nbox] max_u |x_u| of each translation input column
    int *d_err = nullptr;              // device error word of bounded waits
    float2 *d_tmp = nullptr;           // [max_rhs][n] scratch of products

    std::map<int, ie::WorkList> simt_work, tc_work;   // keyed by nrhs (tensor core: and its tuning)
    std::map<int, std::pair<int, int>> tc_tuned;      // nrhs -> (tile columns, item order) from ie_plan_tune
    std::vector<void *> allocs;
    size_t bytes = 0;
    ie_store store = nullptr;          // shared coupling-block store the plan reads (not owned)
    double plan_seconds = 0;
    int64_t n_work_simt = 0, n_work_tc = 0;
    int tc_sms = 0;
    // solver objects reused by ie_solve, keyed by (nrhs, restart, max_iters, tol, prec)
    std::vector<std::pair<std::string, ie_solver>> solvers;
    // profiling of the translation kernel
    int profile = 0;
    cudaEvent_t prof_ev[2] = {nullptr, nullptr};
    double translate_ms = 0;
    int64_t translate_launches = 0;
};

namespace ie {

ie_status dalloc(ie_plan p, void **ptr, size_t bytes);
template <class T>
ie_status dalloc_t(ie_plan p, T **ptr, size_t count) {
    return dalloc(p, reinterpret_cast<void **>(ptr), count * sizeof(T));
}

// kernels (launchers), each stream-ordered.  `gate` (device int, may be null): when
// it reads 0 the kernels return at once (used by GMRES after convergence).
ie_status prepare_kernels();
ie_status launch_coupling_simt(const ie_plan p, const int32_t *d_disp, int64_t nd, float2 *out, bool row_major,
                               cudaStream_t st);
// 16-bit split images (and, fp16, the per-block exponents) of nd FP32 blocks [k][m].
ie_status launch_coupling_tc(const float2 *Cs, int64_t nd, uint16_t *out, int32_t *exps, bool fp16, cudaStream_t st);
ie_status launch_near_blocks(ie_plan p, cudaStream_t st);
ie_status launch_aggregate(const ie_plan p, const float2 *c, float2 *X, int nrhs, cudaStream_t st,
                           const int *gate = nullptr);
// symmetry = 1: the 48 signed-permuted FP32 copies of X into p->d_Xsym
ie_status launch_permute_sym(const ie_plan p, const float2 *X, int nrhs, cudaStream_t st, const int *gate = nullptr);
ie_status launch_split_tc(const ie_plan p, const float2 *X, int nrhs, bool fp16, cudaStream_t st,
                          const int *gate = nullptr);
ie_status launch_disaggregate(const ie_plan p, const float2 *Yslab, int nslab, size_t slab_stride, float2 *r,
                              int nrhs, bool accumulate, cudaStream_t st, const int *gate = nullptr);
ie_status launch_sum_slabs(const ie_plan p, const float2 *Yslab, int nslab, size_t slab_stride, float2 *Y, int nrhs,
                           cudaStream_t st);
ie_status launch_zero(void *ptr, size_t bytes, cudaStream_t st, const int *gate = nullptr);
// nslab regions of `count` complex values, `stride` complex values apart, in one launch
ie_status launch_zero_slabs(float2 *base, int nslab, size_t stride, size_t count, cudaStream_t st,
                            const int *gate = nullptr);
ie_status launch_near(const ie_plan p, const float2 *c, float2 *y, int nrhs, cudaStream_t st,
                      const int *gate = nullptr);
ie_status launch_translate_simt(ie_plan p, const float2 *X, float2 *Yslab, int nrhs, cudaStream_t st,
                                const int *gate = nullptr);
ie_status launch_translate_cvfcnn(ie_plan p, const float2 *X, float2 *Yslab, int nrhs, cudaStream_t st,
                                  const int *gate = nullptr);
// fits the surrogates of the ncanon canonical displacements (device, ncanon x 3); with
// gcanon / gsigma / map (device: per stored block its canonical index and signed
// permutation, and the 48 x 192 symmetry map) every stored block gets its canonical
// network turned into its own frame, else the canonical networks are the stored blocks'
ie_status launch_cvfcnn_fit(ie_plan p, const int32_t *canon_disp, int64_t ncanon, const int32_t *gcanon,
                            const int32_t *gsigma, const uint16_t *map, cudaStream_t st);
ie_status launch_translate_tc(ie_plan p, int prec, float2 *Yslab, int nrhs, cudaStream_t st,
                              const int *gate = nullptr);
ie_status launch_plane_wave(const ie_plan p, const double *d_khat, const double *d_pol, int nrhs, float2 *v,
                            cudaStream_t st);

// y = op(c) (see ie_matvec); accumulate adds the far part into y.
ie_status far_product(ie_plan p, int prec, const float2 *c, float2 *y, int nrhs, bool accumulate, cudaStream_t st,
                      const int *gate = nullptr);
ie_status apply(ie_plan p, int which, int prec, const float2 *c, float2 *y, int nrhs, cudaStream_t st,
                const int *gate = nullptr);
// max_cols > 0 (tensor-core lists): no item wider than max_cols columns
ie_status work_list(ie_plan p, bool tc, int nrhs, WorkList **out, int max_cols = 0, bool pack = false);
// The work list the translation of precision `prec` launches with (the same cache entry):
// made ahead of a stream capture, since building one allocates.
ie_status work_list_for(ie_plan p, int prec, int nrhs, WorkList **out);
ie_status launch_coupling_fp32(double k, double eta, double a, const int32_t *d_disp, int64_t nd, float2 *out,
                               bool row_major, cudaStream_t st);
// FP32 blocks of nd displacements (kept in C32 when given, else cut chunk by chunk from a
// staging buffer) and their 16-bit images where the buffers are given
ie_status generate_blocks(double k, double eta, double a, const int32_t *d_disp, int64_t nd, float2 *C32,
                          uint16_t *bf16, uint16_t *fp16, int32_t *exp16, cudaStream_t st);
bool block_prec_only(unsigned mask);
// Process-wide lock around graph capture and instantiation, and around the calls that
// allocate, free or synchronise the whole device (plan, solver and store creation and
// destruction): host threads that serve different plans then never capture a graph while
// another one frees memory or synchronises the device.  Recursive (destruction nests).
std::recursive_mutex &device_mutex();
void store_retain(ie_store s);
void store_release(ie_store s);
int cvfcnn_tc_tile_columns();
void destroy_cached_solvers(ie_plan p);
// launch the translation kernel of `prec` (with the profiling brackets when enabled)
ie_status translate_timed(ie_plan p, int prec, const float2 *X, float2 *Yslab, int nrhs, cudaStream_t st,
                          const int *gate);
int simt_tile_columns();
int tc_tile_columns();
// runs one bounded device wait on an mbarrier nothing signals (IE_ERR_TIMEOUT expected)
ie_status bounded_wait_selftest(double limit_ms, cudaStream_t st);
// synchronises st; IE_ERR_TIMEOUT (and the word cleared) if a translation gave up a wait
ie_status take_device_error(ie_plan p, cudaStream_t st);

size_t slab_stride(const ie_plan p);   // elements between far-field slabs

// canonical c = sorted |d| of a displacement and the signed permutation Q with Q c = d
int canon_of_disp(const int32_t d[3], int32_t c[3]);
// map[Q][u] = U_Q(u) | 0x100 when negated, 48 x 192 (see the symmetric store)
void symmetry_map_host(std::vector<uint16_t> &map);
// every stored block's network from the canonical ones (Wc [ncanon][kCvBlockElems]),
// turned into the block's frame
void launch_cvfcnn_expand(const float2 *Wc, const int32_t *gcanon, const int32_t *gsigma, const uint16_t *map,
                          int64_t nblk, float2 *Wd, cudaStream_t st);
// tensor-core networks: images (after a fit, training or loaded weights) and inference
size_t cvfcnn_image_elems();
ie_status build_cvfcnn_images(ie_plan p, cudaStream_t st);
ie_status launch_translate_cvfcnn_tc(ie_plan p, float2 *Yslab, int nrhs, cudaStream_t st, const int *gate);
// trains the plan's networks (§3, first stage) and stores them in the plan
ie_status launch_cvfcnn_train(ie_plan p, const ie_cvfcnn_train_opts &o, ie_cvfcnn_train_info *info, cudaStream_t st);

}  // namespace ie
