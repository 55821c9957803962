/*
 * ie.h — C ABI of libie, the GB300 (sm_103a) group-by-group far-zone solver.
 *
 * The library computes the matrix-vector product of an integral-equation system
 * Z I = V (eq. 1) split by the one-box-buffer scheme into a stored near part and a
 * far part (eq. 2), and solves the system with restarted GMRES (§5).  The far part
 * runs the paper's three stages on every product:
 *   1. mapping to uniform basis functions, x_b = P_b^T c_b        (Alg. 1, eq. 11)
 *   2. translation, E_t += G_d x_b for every far box pair,
 *      grouped by box displacement d = t - b                       (Alg. 2, eq. 13, eq. 14)
 *   3. inverse mapping, r_t = P_t E_t                              (Alg. 3, eq. 17)
 * with G_d built directly from the free-space dyadic Green's function (eq. 5, eq. 6).
 *
 * Geometry: boxes of edge `box_edge` on a G^3 grid, box (i,j,k) centred at
 * box_edge*((i,j,k) + 1/2 - G/2); each box holds a 4x4x4 cell-centred lattice of
 * x/y/z Hertzian dipoles (192 unknowns), site s = ix + 4 iy + 16 iz, unknown
 * u = 3 s + component.  Two boxes are far when their Chebyshev distance is >= 2.
 *
 * Conventions for every call below:
 *  - Vectors are caller-owned DEVICE buffers of complex64 (interleaved re, im
 *    float32), laid out [rhs][n] where n = sum of nb over boxes, boxes in the
 *    caller's box order, box b's nb_b coefficients contiguous.
 *  - Dipole-space vectors are [rhs][n_boxes][192] complex64.
 *  - All calls are stream-ordered on `stream` (a cudaStream_t passed as void*,
 *    NULL = legacy default stream) and return without waiting, except
 *    ie_plan_create, ie_plan_destroy, ie_plan_tune, ie_plan_check,
 *    ie_diag_bounded_wait, ie_solve, ie_map_basis and ie_cvfcnn_set_weights,
 *    which synchronise it.
 *  - A plan owns all of its device memory.  Nothing throws across the ABI; every
 *    call returns an ie_status, and ie_last_error() gives a message for the
 *    calling thread's last failure.
 *  - Errors common to every entry point (each declaration lists its others):
 *    IE_ERR_INVALID for a null handle or pointer argument, an unknown precision, an
 *    nrhs outside [1, the plan's max_rhs] or another argument outside its stated
 *    range, detected before any device work; IE_ERR_UNSUPPORTED for a precision the
 *    plan was not prepared for or an option it does not hold; IE_ERR_OOM when a device allocation fails; IE_ERR_CUDA when a CUDA
 *    call or launch fails; IE_ERR_TIMEOUT (tensor-core translations, reported by
 *    ie_plan_check and ie_solve) when a bounded device wait gave up.  The destroy and
 *    release calls accept NULL and return IE_OK.
 *  - Calls on one plan must not overlap in time on different streams (the plan's
 *    scratch vectors are shared), nor come from several host threads at once (its
 *    work-list and solver caches are unlocked); distinct plans are independent, and
 *    plans, solvers and stores may be created and destroyed from any host thread.
 */
#ifndef IE_H_
#define IE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ie_plan_s *ie_plan;
typedef struct ie_store_s *ie_store;
typedef struct ie_solver_s *ie_solver;

typedef enum {
    IE_OK = 0,
    IE_ERR_INVALID = 1,        /* bad argument or geometry                          */
    IE_ERR_OOM = 2,            /* device allocation failed                          */
    IE_ERR_CUDA = 3,           /* a CUDA runtime call failed                        */
    IE_ERR_NOT_CONVERGED = 4,  /* solve stopped at max_iters; best iterate written  */
    IE_ERR_TIMEOUT = 5,        /* a bounded device wait gave up                     */
    IE_ERR_UNSUPPORTED = 6     /* precision or option not prepared in this plan     */
} ie_status;

/* Arithmetic of the translation stage (stage 2).
 *  FP32    plain path: FP32 coupling blocks, FP32 FMA, partial sums combined in FP64.
 *  BF16X3  tcgen05 tensor cores, each FP32 operand split into bf16 hi + lo and the
 *          three products hi*hi + hi*lo + lo*hi accumulated in FP32.
 *  FP16X3  as BF16X3 with fp16 halves.
 *  BF16X1  tcgen05, one bf16 product (hi*hi) — the cheapest, least accurate form.
 *  FP16X1  tcgen05, one fp16 product (hi*hi) from the FP16X3 store: three more bits
 *          than BF16X1; with FP16X3 it makes a mixed pair that shares one store.
 *  CVFCNN  the translation surrogate of §3: per stored block a complex network
 *          192 -> H -> 192 (input scaled by its l-infinity norm, one hidden layer
 *          with the Cartesian ReLU max(Re z, 0) + j max(Im z, 0), linear output,
 *          output rescaled), evaluated on the tcgen05 tensor cores: both layers are
 *          fp16 GEMMs with FP32 accumulation, the hidden activations staying in shared
 *          memory between them.  Weights: fitted at plan creation in closed form (the
 *          network whose output is the best rank-H approximation of the block:
 *          truncated SVD by one-sided Jacobi in FP64, once per canonical displacement
 *          sorted |d|, turned into each displacement's frame, with hidden biases that
 *          keep every pre-activation in the ReLU's linear region on the unit
 *          l-infinity ball); ie_cvfcnn_train replaces them by networks trained as in §3
 *          (first stage), ie_cvfcnn_set_weights by any others.
 *  CVFCNN_FP32  the same networks evaluated in FP32 on the SIMT cores. */
typedef enum {
    IE_PREC_FP32 = 1,
    IE_PREC_BF16X3 = 2,
    IE_PREC_FP16X3 = 3,
    IE_PREC_BF16X1 = 4,
    IE_PREC_FP16X1 = 5,
    IE_PREC_CVFCNN = 6,
    IE_PREC_CVFCNN_FP32 = 7
} ie_prec;
#define IE_PRECMASK(p) (1u << (unsigned)(p))

/* Which part of Z a product applies. */
typedef enum {
    IE_FAR = 1,    /* Z^F c (three stages above)                                    */
    IE_NEAR = 2,   /* alpha c + Z^N c (stored near blocks, eq. 2)                   */
    IE_FULL = 3    /* alpha c + Z^N c + Z^F c                                       */
} ie_which;

typedef struct {
    double k;              /* wavenumber (2 pi for wavelength 1)                       */
    double eta;            /* intrinsic impedance                                      */
    double box_edge;       /* a                                                        */
    int lattice;           /* dipoles per box edge; must be 4                          */
    int grid_n;            /* G (box centres, hence plane-wave phases, use it)         */
    int n_boxes;           /* >= 1                                                     */
    const int32_t *box_ijk;/* HOST, n_boxes x 3, unique, any order                     */
    const int32_t *nb;     /* HOST, n_boxes basis counts in [1,192]; NULL iff P NULL   */
    const double *P;       /* HOST, packed complex128 (re,im): box b's nb_b x 192
                              row-major block follows box b-1's. NULL = identity
                              mapping (nb = 192 per box, dipole unknowns directly).   */
    double alpha;          /* self term of the synthetic system                        */
    int self_box_mode;     /* 0: near part includes the box itself minus coincident
                              dipoles; 1: the box itself is left out                   */
    unsigned prec_mask;    /* IE_PRECMASK(...) of every precision the plan must serve  */
    int max_rhs;           /* largest nrhs any later call will pass (>= 1)             */
    /* Batches of independent scatterers (optional; n_groups = 0: one scatterer).
     * Boxes carry a scatterer id, ids non-decreasing in box order (each scatterer's
     * boxes, hence its unknowns, are contiguous); boxes of different scatterers never
     * interact, and two scatterers may occupy the same grid cells.  All scatterers
     * share k, eta, box_edge and grid_n, hence one coupling-block store.           */
    int n_groups;              /* >= 1 when box_group is given                      */
    const int32_t *box_group;  /* HOST, n_boxes ids in [0, n_groups), non-decreasing */
    const double *group_alpha; /* HOST, n_groups self terms (replaces alpha)        */
    /* Symmetry-compressed coupling store (optional; 0 = one block per displacement).
     * The cell-centred lattice is invariant under the 48 signed axis permutations Q,
     * and D(QR) = Q D(R) Q^T, so G_{Qc} = S_Q G_c S_Q^T with S_Q a signed permutation
     * of the 192 unknowns (§2.2: displacements with the same sorted |d| share one
     * matrix up to such a map).  With symmetry = 1 the plan stores G_c for the
     * canonical c = sorted |d| only, keeps 48 signed-permuted copies of the
     * translation input, and applies the output map in the translation epilogue.   */
    int symmetry;
    /* Right-hand sides of each scatterer (optional, batched plans; NULL = every column).
     * HOST, n_groups counts in [1, max_rhs]: in a call with nrhs columns, scatterer g
     * takes part in the translation with its first min(nrhs, group_nrhs[g]) columns
     * only; its other columns get no far-zone contribution (their inputs should be
     * zero, as those of padded right-hand sides are).                              */
    const int32_t *group_nrhs;
    /* Hidden width H of the CVFCNN surrogates (IE_PREC_CVFCNN in prec_mask), 1..64;
     * 0 = 50, the paper's choice.                                                  */
    int cvfcnn_hidden;
} ie_problem;

typedef struct {
    int n_boxes;
    int64_t n;                 /* basis unknowns                                      */
    int64_t n_far_pairs;       /* ordered (basis box, test box) far pairs             */
    int64_t n_far_disp;        /* distinct far displacements (= coupling blocks)      */
    int64_t n_near_pairs;      /* stored near blocks (self blocks included)           */
    int64_t n_work_simt;       /* work items of the FP32 translation                  */
    int64_t n_work_tc;         /* work items of the tensor-core translation           */
    size_t device_bytes;       /* device memory the plan holds                        */
    double plan_seconds;       /* host wall time of ie_plan_create                    */
    double translate_ms;       /* with profiling on: summed device time of the
                                  translation kernel (CUDA events on its stream)      */
    int64_t translate_launches;/* with profiling on: launches timed                   */
    int n_groups;              /* scatterers in the plan (1 without box_group)        */
    int max_rhs;               /* the plan's max_rhs                                  */
    int64_t n_coupling_blocks; /* stored far blocks: n_far_disp, or the canonical
                                  displacements with symmetry = 1                     */
    int cvfcnn_hidden;         /* H of the surrogates (0: none prepared)             */
    int cvfcnn_sweeps;         /* most Jacobi sweeps any canonical block's SVD took
                                  (at most 16: clustered tiny singular values can use
                                  them up; cvfcnn_tail is exact either way)          */
    double cvfcnn_tail;        /* largest relative Frobenius tail of a block's SVD
                                  beyond H: the surrogate's expected relative error
                                  on inputs with independent entries (e^u of §3)     */
} ie_plan_stats;

/* Build a plan: validate the geometry, group far box pairs by displacement, generate
 * every far coupling block G_d (eq. 13) and the near blocks P_a G_{b-a} P_b^T on the
 * device in FP64 arithmetic, stored in the layouts of the requested precisions
 * (the FP32 block store is kept only when IE_PREC_FP32 is requested; otherwise the
 * 16-bit images are cut from a bounded FP32 staging buffer, chunk by chunk).
 * Host inputs are copied; they may be freed on return.  Synchronises `stream`.
 * Errors: IE_ERR_INVALID (lattice != 4, n_boxes < 1, duplicate boxes, nb outside
 * [1,192], P/nb mismatch, max_rhs < 1, empty prec_mask), IE_ERR_OOM, IE_ERR_CUDA. */
ie_status ie_plan_create(const ie_problem *prob, void *stream, ie_plan *out);

/* Device bytes ie_plan_create would allocate for `prob` (for admission control);
 * host-only, no device work.  Errors: as ie_plan_create's validation. */
ie_status ie_plan_footprint(const ie_problem *prob, size_t *bytes);

/* ---- shared coupling-block stores ------------------------------------------------
 *
 * The translation matrices depend on the box edge, k, eta and the displacement only
 * (end of §2: one set serves every scatterer discretised with the same boxes), and
 * with the symmetry of §2.2 on the sorted |d| only.  A store holds the canonical far
 * blocks G_c of every c = (c0 <= c1 <= c2) with c2 <= max_disp and c2 >= 2, in the
 * coupling-block precisions of prec_mask (FP32, BF16X3/X1, FP16X3/X1), generated once;
 * symmetry-compressed plans of any scatterer whose displacements stay within max_disp
 * then attach to it instead of generating their own (ie_plan_create_shared).
 * Ownership: the store is reference counted; ie_store_release drops the creator's
 * reference and every plan attached to it holds one until ie_plan_destroy, so the
 * blocks live while any plan reads them.  Thread safety: creating and destroying
 * plans on one store from several host threads is safe.                           */
typedef struct {
    double k, eta, box_edge;   /* as in ie_problem                                       */
    int lattice;               /* 4                                                      */
    int max_disp;              /* largest |d_i| of a far displacement served, 2..1024    */
    unsigned prec_mask;        /* coupling-block precisions only (no CVFCNN)            */
} ie_store_spec;

/* Device bytes ie_store_create would hold (host only).  Errors: IE_ERR_INVALID. */
ie_status ie_store_footprint(const ie_store_spec *spec, size_t *bytes);

/* Generate the store on `stream` and wait for it.  Errors: IE_ERR_INVALID (spec),
 * IE_ERR_OOM, IE_ERR_CUDA. */
ie_status ie_store_create(const ie_store_spec *spec, void *stream, ie_store *out);

/* Canonical blocks held and device bytes (either pointer may be NULL). */
ie_status ie_store_info(ie_store store, int64_t *n_blocks, size_t *bytes);

/* Drop the caller's reference (the blocks are freed once no plan holds one). */
ie_status ie_store_release(ie_store store);

/* ie_plan_create for a symmetry-compressed problem (symmetry = 1) whose coupling
 * blocks come from `store`: same k, eta, box_edge and lattice (compared exactly),
 * every coupling-block precision of prob->prec_mask held by the store, no CVFCNN,
 * every far |d_i| <= max_disp.  The plan's n_coupling_blocks is the store's count and
 * its device_bytes excludes the store.  Errors: IE_ERR_INVALID (mismatch, reach),
 * IE_ERR_UNSUPPORTED (symmetry 0, CVFCNN), else as ie_plan_create. */
ie_status ie_plan_create_shared(const ie_problem *prob, ie_store store, void *stream, ie_plan *out);

/* Device bytes ie_plan_create_shared would allocate (host only; the store excluded). */
ie_status ie_plan_footprint_shared(const ie_problem *prob, ie_store store, size_t *bytes);

ie_status ie_plan_stats_get(ie_plan plan, ie_plan_stats *out);

/* Profiling of the translation kernel: with enable = 1 (counters reset), every
 * translation launched outside stream capture is bracketed by CUDA events on its
 * stream and its duration added to translate_ms (the call then waits for it). */
ie_status ie_plan_profile(ie_plan plan, int enable);

/* Autotuner of the tensor-core translation (no counterpart in the paper): for calls with
 * this nrhs, times the translation of precision `prec` with tile widths of 96, 80, 64
 * and 48 columns and two work-item orders (largest first; displacement order, which runs
 * the tiles of one group on neighbouring CTAs together) and keeps the fastest for the
 * plan.  Synchronises `stream`; overwrites the plan's scratch.  info (may be NULL): the
 * chosen tile width and order, its time per launch and that of the default (96, 1).
 * Errors: IE_ERR_INVALID, IE_ERR_UNSUPPORTED (FP32 or a precision not in the plan). */
typedef struct {
    int tile_columns;      /* complex columns per work item chosen                       */
    int order;             /* 0: items largest first, 1: displacement order              */
    double ms;             /* its translation time per launch                            */
    double default_ms;     /* the default's (128 columns, order 1)                       */
    int candidates;        /* configurations timed                                       */
} ie_tune_info;
ie_status ie_plan_tune(ie_plan plan, int prec, int nrhs, ie_tune_info *info, void *stream);

/* Status of the plan's earlier asynchronous work: synchronises `stream`; returns
 * IE_ERR_TIMEOUT if a translation launch gave up one of its bounded device waits since
 * the last check (its product is then incomplete; the plan stays usable), IE_OK otherwise.
 * ie_solve checks this itself before it returns. */
ie_status ie_plan_check(ie_plan plan, void *stream);

/* Diagnostic (no counterpart in the paper): one thread waits, with the translation
 * kernels' bounded wait, on an mbarrier that nothing signals, for about limit_ms
 * (0 < limit_ms <= 10000).  Returns IE_ERR_TIMEOUT when the wait gave up and reported
 * it, as designed; any other status means the bound does not work. */
ie_status ie_diag_bounded_wait(double limit_ms, void *stream);

/* Diagnostics of the abort path: sets, process-wide, the give-up limit (SM clock cycles) of
 * the tensor-core translation's pipeline waits for later launches (0 restores the default
 * 2^31, about 1 s).  With a limit far below a wait's normal duration a launch gives up: its
 * roles leave uniformly, the drains (which keep the default limit) wait for the copies and
 * MMAs in flight, TMEM is freed, the plan's error word is set (ie_plan_check then returns
 * IE_ERR_TIMEOUT) and the product is incomplete.  Synchronous.  For tests only. */
ie_status ie_diag_wait_limit(int64_t cycles);

/* Release every device allocation of the plan (synchronises the device first). */
ie_status ie_plan_destroy(ie_plan plan);

/* y = op(c) for nrhs right-hand sides (op from `which`, translation arithmetic from
 * `prec`).  c, y: device complex64 [nrhs][n]; y is overwritten; c and y must not
 * alias.  Errors: IE_ERR_INVALID (null pointers, nrhs outside [1,max_rhs]),
 * IE_ERR_UNSUPPORTED (prec not in the plan's prec_mask), IE_ERR_CUDA. */
ie_status ie_matvec(ie_plan plan, int which, int prec, const void *c, void *y, int nrhs, void *stream);

/* ---- the three far-zone stages and the near product, one call each ---------- */

/* Stage 1 (Alg. 1): X[r][b][u] = sum_i P_b[i][u] c[r][o_b + i].  X: device complex64
 * [nrhs][n_boxes][192]. */
ie_status ie_aggregate(ie_plan plan, const void *c, void *X, int nrhs, void *stream);

/* Stage 2 (Alg. 2): Y[r][t] = sum over far b of G_{t-b} X[r][b], in `prec`.
 * X, Y: device complex64 [nrhs][n_boxes][192]; Y overwritten. */
ie_status ie_translate(ie_plan plan, int prec, const void *X, void *Y, int nrhs, void *stream);

/* Stage 3 (Alg. 3): r[r][o_b + i] = sum_u P_b[i][u] Y[r][b][u] (overwrites r). */
ie_status ie_disaggregate(ie_plan plan, const void *Y, void *r, int nrhs, void *stream);

/* Allocation-free form of ie_translate with prec = IE_PREC_FP32 (the paper has no
 * counterpart; it serves callers that cannot allocate device memory at call time,
 * e.g. code whose device memory belongs to another allocator's pool, or a latency-
 * critical loop where cudaMalloc / cudaFree could block or synchronise the device).
 * Same arithmetic and result as ie_translate; it calls no allocator and copies nothing from host memory (the
 * displacement-group offsets it reads were put on the device with the plan).  Its
 * scratch is a fixed 32 MiB device area inside libie (held by every GPU that loads the
 * library until exit) that must hold 8 x nrhs x n_boxes x 192 complex64 partial sums;
 * larger requests return IE_ERR_INVALID with the sizes in ie_last_error().  The first call on a device looks the area up and sets the kernel
 * up on that device (make it before any stream capture); later calls launch kernels
 * only and may be captured into a CUDA graph and replayed.  Every call reuses the same
 * area, so calls that overlap in time on the GPU (any streams, any plans) race; the
 * partial sums are cleared by each call.  X, Y: device complex64 [nrhs][n_boxes][192].
 * A plan built without IE_PREC_FP32, with symmetry = 1 or with group_nrhs returns
 * IE_ERR_UNSUPPORTED. */
ie_status ie_translate_noalloc(ie_plan plan, const void *X, void *Y, int nrhs, void *stream);

/* Near product (eq. 2, stored Z^N) plus the self term: y = alpha c + Z^N c. */
ie_status ie_near(ie_plan plan, const void *c, void *y, int nrhs, void *stream);

/* Coupling blocks G_d for `nd` displacements d (HOST int32 nd x 3; any d, near or
 * far; d = 0 has its coincident 3x3 diagonal blocks zeroed), written to the device
 * buffer `out` as complex64 [nd][192][192] row-major (row = test unknown).  Uses
 * the plan's k, eta and box edge; the plan's own store is not touched. */
ie_status ie_coupling_blocks(ie_plan plan, const int32_t *d, int nd, void *out, void *stream);

/* Plane-wave excitation tested with the basis functions (§5): v = P e with
 * e[r][b][3s+a] = pol_r[a] exp(-j k khat_r . r_s).  khat, pol: HOST double nrhs x 3
 * (batched plans: n_groups x nrhs x 3, scatterer-major, so each scatterer has its own
 * incidences; a zero polarisation leaves that scatterer's column at zero);
 * nrhs in [1, max_rhs] counts the columns of v, not n_groups x nrhs;
 * v: device complex64 [nrhs][n]. */
ie_status ie_rhs_plane_wave(ie_plan plan, const double *khat, const double *pol, int nrhs, void *v,
                            void *stream);

/* ---- GMRES ------------------------------------------------------------------ */

typedef struct {
    int restart;         /* m of GMRES(m) (default 50)                                  */
    int max_iters;       /* total inner iterations allowed (default 1000)               */
    double tol;          /* stop at ||v - Z c|| <= tol ||v|| per right-hand side        */
    int prec;            /* translation arithmetic inside GMRES (default IE_PREC_FP32)  */
    int refine;          /* 1: outer iterative refinement (see ie_solve)                */
    int refine_prec;     /* arithmetic of the refinement residual (default FP32)        */
    double inner_tol;    /* inner GMRES relative tolerance when refining (default 1e-3) */
    int max_refine;      /* outer steps allowed (default 20)                            */
} ie_solve_opts;

typedef struct {
    int iterations;      /* inner GMRES iterations (max over right-hand sides)          */
    int matvecs;         /* operator applications (all precisions)                      */
    int refinements;     /* outer refinement steps taken                                */
    int converged;       /* 1 when every right-hand side met tol                        */
    double relres;       /* max over right-hand sides of the final relative residual
                            ||v - Z c|| / ||v||, recomputed from c (not the Arnoldi
                            recurrence): without refinement at the end of the last
                            restart cycle with a `prec` product (FP32 difference, FP64
                            norms); with refinement the FP64 residual of the last outer
                            step (`refine_prec` product, FP64 difference and norms)     */
    double seconds;      /* host wall time of the call                                  */
} ie_solve_info;

/* Fill `o` with the defaults above. */
void ie_solve_opts_default(ie_solve_opts *o);

/* Solve Z c = v for nrhs independent right-hand sides with restarted GMRES (§5);
 * in a batched plan every (scatterer, right-hand side) pair is its own GMRES system
 * over its scatterer's unknowns, with its own convergence test:
 * x0 = 0, Arnoldi by classical Gram-Schmidt applied twice with FP64 dot products,
 * Givens rotations and the small least-squares solve in FP64, Krylov vectors in
 * FP32 on the device.  With refine = 1, c is kept in FP64, each outer step forms
 * r = v - Z c with `refine_prec` products and FP64 vector arithmetic, solves
 * Z d = r with GMRES in `prec` to inner_tol and adds d, until ||r|| <= tol ||v||.
 * v, c: device complex64 [nrhs][n]; c overwritten.  Synchronises `stream`.
 * Returns IE_ERR_NOT_CONVERGED (with the best iterate in c and info filled) when
 * the limits are reached first. */
ie_status ie_solve(ie_plan plan, const void *v, void *c, int nrhs, const ie_solve_opts *opts,
                   ie_solve_info *info, void *stream);

/* ---- solver objects: the same GMRES with device-resident state, stepped
 * without host synchronisation (for request loops that interleave many solves). */

/* Allocate the device state of a GMRES(opts->restart) solve of up to nrhs
 * right-hand sides on `plan` (refine must be 0). */
ie_status ie_solver_create(ie_plan plan, int nrhs, const ie_solve_opts *opts, ie_solver *out);

/* Device bytes ie_solver_create would allocate. */
ie_status ie_solver_footprint(ie_plan plan, int nrhs, const ie_solve_opts *opts, size_t *bytes);

/* Enqueue the start of a solve of Z c = v (x0 = 0); v and c must stay valid until
 * the solve is finished.  Nothing waits. */
ie_status ie_solver_start(ie_solver s, const void *v, void *c, void *stream);

/* Enqueue `cycles` restart cycles (each up to `restart` iterations; kernels of a
 * converged right-hand side do nothing) and the solution update.  Nothing waits. */
ie_status ie_solver_advance(ie_solver s, int cycles, void *stream);

/* Non-blocking: *done = 1 once everything enqueued on the solver has finished and
 * every right-hand side converged or hit max_iters; then info is filled.  Start and
 * advance end with an asynchronous copy of the solver's status into pinned host
 * memory, so polling makes no synchronous device call. */
ie_status ie_solver_poll(ie_solver s, int *done, ie_solve_info *info);

/* Non-blocking state for request loops: IE_SOLVER_BUSY while enqueued work runs,
 * IE_SOLVER_IDLE once it has finished with some system still iterating (advance
 * again), IE_SOLVER_DONE once every system converged or hit max_iters (info filled
 * in the last two states). */
enum { IE_SOLVER_BUSY = 0, IE_SOLVER_IDLE = 1, IE_SOLVER_DONE = 2 };
ie_status ie_solver_state(ie_solver s, int *state, ie_solve_info *info);

ie_status ie_solver_destroy(ie_solver s);

/* ---- mapping construction (§2.1): the rows of P_b from subdomain basis functions --
 *
 * A basis function made of point dipoles radiates B_f, its field at N_s sample
 * points r_l on a sphere S about its box centre (eq. 4, eq. 10).  The 192 uniform
 * dipoles radiate A (3 N_s x 192) there.  Eq. 11 takes the least-squares fit
 * C_f = A^+ B_f (eq. 9-10: the uniform dipoles whose field best matches the
 * function's on S), and row f of P_b is C_f^T: x_b = P_b^T c_b is then Alg. 1.
 * The same rows serve the inverse mapping of eq. 15-17 when the test functions
 * are the basis functions: D(R) = D(-R) = D(R)^T makes the tested fields of the
 * virtual dipoles B_f^T, and (A^T)^+ = (A^+)^T, so Alg. 3 reads r_b = P_b y_b.
 *
 * S has radius sample_radius * box_edge; its samples form the spherical Fibonacci
 * lattice: polar angle arccos(1 - (2l+1)/N_s), azimuth 2 pi l / golden ratio,
 * l = 0 .. N_s-1.  A^+ comes from a Householder QR of A in FP64 (A has full column
 * rank for N_s >= 64; its condition number is about 1e7 at N_s = 128), and the
 * fields and products are FP64 throughout.
 *
 * tikhonov = 0 gives eq. 11's plain pseudo-inverse.  Its coefficients oscillate with
 * norms ~100x those of the function's field, and the far product then cancels:
 * FP32 evaluation loses about two more digits.  tikhonov = t > 0 solves instead
 * min ||A C - B||^2 + (t ||A||_F)^2 ||C||^2 (QR of [A; t ||A||_F I]); t = 1e-5 cuts
 * the coefficient norms ~25x at an unchanged field error outside S. */
typedef struct {
    double k, eta, box_edge;   /* as in ie_problem                                     */
    int lattice;               /* dipoles per box edge; must be 4                      */
    int n_samples;             /* N_s, 64 .. 256 (the paper: N_s = 2 N_d = 128)        */
    double sample_radius;      /* radius of S in box edges, > sqrt(3)/2 so that S
                                  encloses the box (the paper: 1.5)                   */
    double tikhonov;           /* >= 0, relative to ||A||_F; 0 = eq. 11 as printed     */
} ie_mapping_spec;

/* Map n_fun basis functions.  All pointers are HOST memory; the call copies them
 * to the device, runs there and copies the results back before returning.
 *   fun_off   n_fun + 1 offsets, fun_off[0] = 0, non-decreasing: function f owns
 *             point dipoles fun_off[f] .. fun_off[f+1]-1 (none: a zero row)
 *   pos       fun_off[n_fun] x 3 doubles, dipole positions relative to the centre
 *             of the function's box; each strictly inside S
 *   mom       fun_off[n_fun] x 3 complex128 (re, im interleaved) dipole moments
 *   P         out: n_fun x 192 complex128, row f = C_f^T (rows in the order given,
 *             so functions listed box by box pack as ie_problem.P)
 *   residual  out, may be NULL: n_fun doubles ||A C_f - B_f|| / ||B_f||, the
 *             field mismatch on S (0 for a function without dipoles)
 * Errors: IE_ERR_INVALID for a bad spec, offsets, a non-finite value or a dipole
 * outside S (nothing runs); IE_ERR_OOM / IE_ERR_CUDA from the device; IE_ERR_INVALID
 * also if A is numerically rank deficient (a zero Householder column). */
ie_status ie_map_basis(const ie_mapping_spec *spec, int64_t n_fun, const int64_t *fun_off,
                       const double *pos, const double *mom, double *P, double *residual,
                       void *stream);

/* ---- Symmetry of the translation matrices (§2.2), host only ------------------------ */

/* Canonical displacement c = sorted |d| (c[0] <= c[1] <= c[2]) of a box displacement d,
 * and the index q (0..47) of a signed axis permutation Q with d = Q c:
 *     q = 8 p + s,   (Q c)_i = (-1)^(bit i of s) c[perm_p(i)],
 *     perm_0..perm_5 = (0,1,2), (0,2,1), (1,0,2), (1,2,0), (2,0,1), (2,1,0);
 * a zero component has its sign bit clear, and when components of |d| are equal one of
 * the permutations that fit is returned.  d, c: HOST, 3 int32 each.  No device call.
 * Errors: IE_ERR_INVALID for a null pointer. */
ie_status ie_sym_canon(const int32_t *d, int32_t *c, int32_t *q);

/* Unknown map of the 48 signed permutations, the table the symmetry-compressed store and
 * the translation epilogues use: map[q * 192 + u] = U_q(u), with 0x100 added when the
 * unknown changes sign, such that for d = Q c (Q of index q)
 *     G_d[U_q(u)][U_q(v)] = sign_q(u) sign_q(v) G_c[u][v]
 * (unknown u = 3 site + component, eq. 13).  map: HOST, 48 x 192 uint16.  No device
 * call.  Errors: IE_ERR_INVALID for a null pointer. */
ie_status ie_sym_map(uint16_t *map);

/* ---- CVFCNN surrogates (§3) ------------------------------------------------------ */

/* Displacements of the stored far blocks, in the plan's block order (the canonical
 * sorted |d| with symmetry = 1, else every far displacement): disp, HOST,
 * n_coupling_blocks x 3. */
ie_status ie_plan_blocks(ie_plan plan, int32_t *disp);

/* Replace the fitted surrogate weights (plan prepared with IE_PREC_CVFCNN or CVFCNN_FP32).  HOST
 * complex64 (re, im interleaved), per stored block in ie_plan_blocks order, H the
 * plan's cvfcnn_hidden:  W1 [blocks][H][192], b1 [blocks][H], W2 [blocks][192][H],
 * b2 [blocks][192].  The network of block c maps x to s (W2 relu(W1 x / s + b1) + b2),
 * relu(z) = max(Re z, 0) + j max(Im z, 0) elementwise, s = max_u |x_u| (0 for x = 0);
 * with symmetry = 1 displacement d = Q c applies it in
 * the frame of c (input through S_Q^T, output through S_Q).  Synchronises stream. */
ie_status ie_cvfcnn_set_weights(ie_plan plan, const float *W1, const float *b1, const float *W2, const float *b2,
                                void *stream);

/* Read the plan's current surrogate weights back (closed-form, trained or set) into HOST
 * buffers of the ie_cvfcnn_set_weights layout, which the caller owns.  Synchronises
 * stream.  Errors: IE_ERR_INVALID (null buffer), IE_ERR_UNSUPPORTED (no surrogates). */
ie_status ie_cvfcnn_get_weights(ie_plan plan, float *W1, float *b1, float *W2, float *b2, void *stream);

/* Training of the networks (§3, first stage; replaces the closed-form weights).  One
 * network per canonical displacement c = sorted |d| of the plan's far groups, width the
 * plan's cvfcnn_hidden, trained from random weights (complex normal, variance 1/192 for
 * W1 and 1/H for W2, zero biases) with Adam (beta 0.9 / 0.999, step size lr on a cosine
 * decay to 2% of it over max_steps) on the mean square error between the network and
 * the DGFA product G_c x (eq. 13) for batches of 32 x minibatches inputs whose real and imaginary
 * parts are uniform in [-1, 1], normalised by their l-infinity norm as the network's
 * input is.  Every eval_every steps e^u of eq. 171 (mean relative l2 error of the
 * outputs) is measured on a fixed test set of 64 such inputs; a network's training ends
 * once e^u < tol (the paper: 1e-3) or after max_steps.  The inputs come from a counter-
 * based generator (splitmix64 of seed, network, step, index), so a training run is
 * reproducible.  The paper's second stage needs RWG-mapped surface data and is not run.
 * Synchronises `stream`.  info (may be NULL) reports the networks trained, how many
 * reached tol, the largest and the mean final e^u, the most steps taken and the time.
 * Errors: IE_ERR_UNSUPPORTED (plan without surrogates), IE_ERR_INVALID, IE_ERR_OOM. */
typedef struct {
    int max_steps;         /* Adam steps per network (default 8000)                        */
    int minibatches;       /* minibatches of 32 inputs per step (default 4: 128 inputs)    */
    int eval_every;        /* steps between e^u checks (default 250; 0: only at the end)   */
    double lr;             /* Adam step size (default 4e-3)                                 */
    double tol;            /* e^u at which a network's training stops (default 1e-3)       */
    uint64_t seed;         /* generator seed                                               */
} ie_cvfcnn_train_opts;
typedef struct {
    int64_t networks;      /* networks trained (canonical displacements)                   */
    int64_t converged;     /* networks whose final e^u < tol                               */
    double eu_max, eu_mean;/* final e^u over the networks                                  */
    int steps_max;         /* most Adam steps any network took                             */
    double seconds;        /* host wall time of the call                                   */
} ie_cvfcnn_train_info;
void ie_cvfcnn_train_opts_default(ie_cvfcnn_train_opts *o);
ie_status ie_cvfcnn_train(ie_plan plan, const ie_cvfcnn_train_opts *opts, ie_cvfcnn_train_info *info,
                          void *stream);

/* ---- diagnostics -------------------------------------------------------------- */
const char *ie_status_str(ie_status s);
const char *ie_last_error(void);   /* thread-local; "" if none */
const char *ie_version(void);

/* Kernels this process has launched through libie so far: direct launches plus the
 * kernel nodes of every replay of a captured GMRES cycle. */
int64_t ie_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* IE_H_ */
