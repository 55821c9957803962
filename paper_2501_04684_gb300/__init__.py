"""Python binding of libie, the GB300 (sm_103a) group-by-group far-zone solver.

Argument marshalling only: every function below forwards to the C ABI declared in
include/ie.h (same names), passing device pointers of caller-owned torch tensors
and the CUDA stream handle.  All arithmetic runs in libie's CUDA kernels; there is
no CPU fallback, and importing the binding fails loudly when libie.so is missing.

Vectors are complex64 CUDA tensors laid out [rhs][n] (basis space) or
[rhs][n_boxes][192] (dipole space).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libie.so")

IE_OK, IE_ERR_INVALID, IE_ERR_OOM, IE_ERR_CUDA, IE_ERR_NOT_CONVERGED, IE_ERR_TIMEOUT, IE_ERR_UNSUPPORTED = range(7)
IE_PREC_FP32, IE_PREC_BF16X3, IE_PREC_FP16X3, IE_PREC_BF16X1, IE_PREC_FP16X1, IE_PREC_CVFCNN = 1, 2, 3, 4, 5, 6
IE_PREC_CVFCNN_FP32 = 7
IE_FAR, IE_NEAR, IE_FULL = 1, 2, 3
PREC_NAMES = {IE_PREC_FP32: "fp32", IE_PREC_BF16X3: "bf16x3", IE_PREC_FP16X3: "fp16x3", IE_PREC_BF16X1: "bf16x1",
              IE_PREC_FP16X1: "fp16x1", IE_PREC_CVFCNN: "cvfcnn", IE_PREC_CVFCNN_FP32: "cvfcnn_fp32"}
NU = 192                      # dipole unknowns per box (4^3 lattice x 3 orientations)

EXPORTED = [
    "ie_plan_create", "ie_plan_footprint", "ie_plan_stats_get", "ie_plan_destroy", "ie_matvec",
    "ie_aggregate", "ie_translate", "ie_disaggregate", "ie_near", "ie_coupling_blocks", "ie_rhs_plane_wave",
    "ie_solve_opts_default", "ie_solve", "ie_solver_create", "ie_solver_footprint", "ie_solver_start",
    "ie_solver_advance", "ie_solver_poll", "ie_solver_destroy", "ie_status_str", "ie_last_error", "ie_version",
    "ie_plan_profile", "ie_kernel_launches", "ie_translate_noalloc", "ie_plan_check", "ie_diag_bounded_wait",
    "ie_plan_tune", "ie_map_basis", "ie_plan_blocks", "ie_cvfcnn_set_weights", "ie_cvfcnn_get_weights",
    "ie_cvfcnn_train",
    "ie_cvfcnn_train_opts_default", "ie_store_footprint", "ie_store_create", "ie_store_info", "ie_store_release",
    "ie_plan_create_shared", "ie_plan_footprint_shared", "ie_solver_state", "ie_diag_wait_limit",
    "ie_sym_canon", "ie_sym_map",
]


def precmask(*precs) -> int:
    m = 0
    for p in precs:
        m |= 1 << p
    return m


class ie_store_spec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("eta", ctypes.c_double), ("box_edge", ctypes.c_double),
                ("lattice", ctypes.c_int), ("max_disp", ctypes.c_int), ("prec_mask", ctypes.c_uint)]


class ie_problem(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("eta", ctypes.c_double), ("box_edge", ctypes.c_double),
                ("lattice", ctypes.c_int), ("grid_n", ctypes.c_int), ("n_boxes", ctypes.c_int),
                ("box_ijk", ctypes.c_void_p), ("nb", ctypes.c_void_p), ("P", ctypes.c_void_p),
                ("alpha", ctypes.c_double), ("self_box_mode", ctypes.c_int), ("prec_mask", ctypes.c_uint),
                ("max_rhs", ctypes.c_int), ("n_groups", ctypes.c_int), ("box_group", ctypes.c_void_p),
                ("group_alpha", ctypes.c_void_p), ("symmetry", ctypes.c_int), ("group_nrhs", ctypes.c_void_p),
                ("cvfcnn_hidden", ctypes.c_int)]


class ie_plan_stats(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int), ("n", ctypes.c_int64), ("n_far_pairs", ctypes.c_int64),
                ("n_far_disp", ctypes.c_int64), ("n_near_pairs", ctypes.c_int64), ("n_work_simt", ctypes.c_int64),
                ("n_work_tc", ctypes.c_int64), ("device_bytes", ctypes.c_size_t), ("plan_seconds", ctypes.c_double),
                ("translate_ms", ctypes.c_double), ("translate_launches", ctypes.c_int64),
                ("n_groups", ctypes.c_int), ("max_rhs", ctypes.c_int), ("n_coupling_blocks", ctypes.c_int64),
                ("cvfcnn_hidden", ctypes.c_int), ("cvfcnn_sweeps", ctypes.c_int), ("cvfcnn_tail", ctypes.c_double)]


class ie_tune_info(ctypes.Structure):
    _fields_ = [("tile_columns", ctypes.c_int), ("order", ctypes.c_int), ("ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("candidates", ctypes.c_int)]


class ie_cvfcnn_train_opts(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int), ("minibatches", ctypes.c_int), ("eval_every", ctypes.c_int),
                ("lr", ctypes.c_double),
                ("tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class ie_cvfcnn_train_info(ctypes.Structure):
    _fields_ = [("networks", ctypes.c_int64), ("converged", ctypes.c_int64), ("eu_max", ctypes.c_double),
                ("eu_mean", ctypes.c_double), ("steps_max", ctypes.c_int), ("seconds", ctypes.c_double)]


class ie_mapping_spec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("eta", ctypes.c_double), ("box_edge", ctypes.c_double),
                ("lattice", ctypes.c_int), ("n_samples", ctypes.c_int), ("sample_radius", ctypes.c_double),
                ("tikhonov", ctypes.c_double)]


class ie_solve_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("tol", ctypes.c_double),
                ("prec", ctypes.c_int), ("refine", ctypes.c_int), ("refine_prec", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int)]


class ie_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int), ("refinements", ctypes.c_int),
                ("converged", ctypes.c_int), ("relres", ctypes.c_double), ("seconds", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libie.so (built in-tree by __graft_entry__.build() / build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libie CUDA library not built ({LIB_PATH} missing); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, u, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    L.ie_plan_create.argtypes = [P(ie_problem), vp, P(vp)]
    L.ie_plan_footprint.argtypes = [P(ie_problem), P(sz)]
    L.ie_store_footprint.argtypes = [P(ie_store_spec), P(sz)]
    L.ie_store_create.argtypes = [P(ie_store_spec), vp, P(vp)]
    L.ie_store_info.argtypes = [vp, P(ctypes.c_int64), P(sz)]
    L.ie_store_release.argtypes = [vp]
    L.ie_plan_create_shared.argtypes = [P(ie_problem), vp, vp, P(vp)]
    L.ie_plan_footprint_shared.argtypes = [P(ie_problem), vp, P(sz)]
    L.ie_plan_stats_get.argtypes = [vp, P(ie_plan_stats)]
    L.ie_plan_destroy.argtypes = [vp]
    L.ie_plan_profile.argtypes = [vp, i]
    L.ie_matvec.argtypes = [vp, i, i, vp, vp, i, vp]
    L.ie_aggregate.argtypes = [vp, vp, vp, i, vp]
    L.ie_translate.argtypes = [vp, i, vp, vp, i, vp]
    L.ie_disaggregate.argtypes = [vp, vp, vp, i, vp]
    L.ie_translate_noalloc.argtypes = [vp, vp, vp, i, vp]
    L.ie_near.argtypes = [vp, vp, vp, i, vp]
    L.ie_coupling_blocks.argtypes = [vp, vp, i, vp, vp]
    L.ie_rhs_plane_wave.argtypes = [vp, vp, vp, i, vp, vp]
    L.ie_solve_opts_default.argtypes = [P(ie_solve_opts)]
    L.ie_solve_opts_default.restype = None
    L.ie_solve.argtypes = [vp, vp, vp, i, P(ie_solve_opts), P(ie_solve_info), vp]
    L.ie_solver_create.argtypes = [vp, i, P(ie_solve_opts), P(vp)]
    L.ie_solver_footprint.argtypes = [vp, i, P(ie_solve_opts), P(sz)]
    L.ie_solver_start.argtypes = [vp, vp, vp, vp]
    L.ie_solver_advance.argtypes = [vp, i, vp]
    L.ie_solver_poll.argtypes = [vp, P(i), P(ie_solve_info)]
    L.ie_solver_state.argtypes = [vp, P(i), P(ie_solve_info)]
    L.ie_diag_wait_limit.argtypes = [ctypes.c_int64]
    L.ie_solver_destroy.argtypes = [vp]
    L.ie_status_str.argtypes = [i]
    L.ie_status_str.restype = ctypes.c_char_p
    L.ie_last_error.restype = ctypes.c_char_p
    L.ie_version.restype = ctypes.c_char_p
    L.ie_kernel_launches.restype = ctypes.c_int64
    L.ie_plan_check.argtypes = [vp, vp]
    L.ie_diag_bounded_wait.argtypes = [ctypes.c_double, vp]
    L.ie_plan_tune.argtypes = [vp, i, i, P(ie_tune_info), vp]
    L.ie_map_basis.argtypes = [P(ie_mapping_spec), ctypes.c_int64, vp, vp, vp, vp, vp, vp]
    L.ie_plan_blocks.argtypes = [vp, vp]
    L.ie_sym_canon.argtypes = [vp, vp, P(ctypes.c_int32)]
    L.ie_sym_map.argtypes = [vp]
    L.ie_cvfcnn_set_weights.argtypes = [vp, vp, vp, vp, vp, vp]
    L.ie_cvfcnn_get_weights.argtypes = [vp, vp, vp, vp, vp, vp]
    L.ie_cvfcnn_train_opts_default.argtypes = [P(ie_cvfcnn_train_opts)]
    L.ie_cvfcnn_train_opts_default.restype = None
    L.ie_cvfcnn_train.argtypes = [vp, P(ie_cvfcnn_train_opts), P(ie_cvfcnn_train_info), vp]
    for name in EXPORTED:          # every declared symbol must resolve
        getattr(L, name)
    _lib = L
    return L


class IEError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        self.status = status
        msg = L.ie_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.ie_status_str(status).decode()} ({msg})")


def _check(status: int, where: str, allow=(IE_OK,)):
    if status not in allow:
        raise IEError(status, where)
    return status


def _ptr(t) -> int:
    """Device (or host numpy) pointer of a tensor / array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _need(t, count: int, what: str):
    """Marshalling check of a device buffer: a CUDA complex64 contiguous tensor of at
    least `count` elements (raw integer pointers are passed through unchecked)."""
    if t is None or isinstance(t, int):
        return
    if isinstance(t, np.ndarray):
        raise TypeError(f"{what}: device buffer expected, got a numpy array")
    import torch
    if not t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous():
        raise TypeError(f"{what}: contiguous CUDA complex64 tensor expected")
    if t.numel() < count:
        raise ValueError(f"{what}: {t.numel()} elements, at least {count} needed")


def _dims(plan) -> tuple[int, int, int]:
    """(n basis unknowns, n_boxes, n_groups) of a plan handle."""
    s = ie_plan_stats()
    _check(lib().ie_plan_stats_get(plan, ctypes.byref(s)), "ie_plan_stats_get")
    return int(s.n), int(s.n_boxes), int(s.n_groups)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return stream


def make_problem(k, eta, box_edge, grid_n, box_ijk, nb, P, alpha, prec_mask, max_rhs=1, self_box_mode=0,
                 lattice=4, box_group=None, group_alpha=None, symmetry=0, group_nrhs=None, cvfcnn_hidden=0):
    """Build an ie_problem struct; keeps the host arrays alive on the returned object.
    box_group / group_alpha: batch of independent scatterers (ids non-decreasing)."""
    ijk = np.ascontiguousarray(box_ijk, dtype=np.int32)
    nb_a = None if nb is None else np.ascontiguousarray(nb, dtype=np.int32)
    P_a = None if P is None else np.ascontiguousarray(np.asarray(P, dtype=np.complex128))
    bg = None if box_group is None else np.ascontiguousarray(box_group, dtype=np.int32)
    ga = None if group_alpha is None else np.ascontiguousarray(group_alpha, dtype=np.float64)
    gr = None if group_nrhs is None else np.ascontiguousarray(group_nrhs, dtype=np.int32)
    pr = ie_problem(k=k, eta=eta, box_edge=box_edge, lattice=lattice, grid_n=grid_n, n_boxes=ijk.shape[0],
                    box_ijk=ijk.ctypes.data, nb=None if nb_a is None else nb_a.ctypes.data,
                    P=None if P_a is None else P_a.ctypes.data, alpha=alpha, self_box_mode=self_box_mode,
                    prec_mask=prec_mask, max_rhs=max_rhs, n_groups=0 if ga is None else len(ga),
                    box_group=None if bg is None else bg.ctypes.data,
                    group_alpha=None if ga is None else ga.ctypes.data, symmetry=int(symmetry),
                    group_nrhs=None if gr is None else gr.ctypes.data, cvfcnn_hidden=int(cvfcnn_hidden))
    pr._keep = (ijk, nb_a, P_a, bg, ga, gr)
    return pr


def problem_from(p, prec_mask: int, max_rhs: int = 1, symmetry: int = 0, cvfcnn_hidden: int = 0):
    """ie_problem from a workloads.Problem-like object."""
    return make_problem(p.k, p.eta, p.a, p.G, p.box_ijk, None if p.P is None else p.nb, p.P, p.alpha, prec_mask,
                        max_rhs, getattr(p, "self_box_mode", 0), p.lattice, symmetry=symmetry,
                        cvfcnn_hidden=cvfcnn_hidden)


def problem_from_batch(b, prec_mask: int, max_rhs: int | None = None, symmetry: int = 0, exact_rhs: bool = False):
    """ie_problem of a batch of scatterers (workloads.Batch-like: members in order,
    box_group ids, one self term per member).  exact_rhs: translate only each member's
    own right-hand sides (b.nrhs), not the padding up to the batch's largest count."""
    m0 = b.members[0]
    return make_problem(m0.k, m0.eta, m0.a, b.G, b.box_ijk, b.nb, b.P, m0.alpha, prec_mask,
                        b.max_rhs if max_rhs is None else max_rhs, getattr(m0, "self_box_mode", 0), m0.lattice,
                        box_group=b.box_group, group_alpha=b.group_alpha, symmetry=symmetry,
                        group_nrhs=np.asarray(b.nrhs, dtype=np.int32) if exact_rhs else None)


# ---------------------------------------------------------------- C ABI, same names
def ie_plan_create(problem: ie_problem, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ie_plan_create(ctypes.byref(problem), _stream(stream), ctypes.byref(h)), "ie_plan_create")
    return h.value


def ie_plan_create_shared(problem: ie_problem, store: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ie_plan_create_shared(ctypes.byref(problem), store, _stream(stream), ctypes.byref(h)),
           "ie_plan_create_shared")
    return h.value


def ie_plan_footprint_shared(problem: ie_problem, store: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().ie_plan_footprint_shared(ctypes.byref(problem), store, ctypes.byref(b)), "ie_plan_footprint_shared")
    return b.value


def store_spec(k: float, eta: float, a: float, max_disp: int, prec_mask: int, lattice: int = 4) -> ie_store_spec:
    return ie_store_spec(k=k, eta=eta, box_edge=a, lattice=lattice, max_disp=int(max_disp), prec_mask=prec_mask)


def ie_store_footprint(spec: ie_store_spec) -> int:
    b = ctypes.c_size_t()
    _check(lib().ie_store_footprint(ctypes.byref(spec), ctypes.byref(b)), "ie_store_footprint")
    return b.value


def ie_store_create(spec: ie_store_spec, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ie_store_create(ctypes.byref(spec), _stream(stream), ctypes.byref(h)), "ie_store_create")
    return h.value


def ie_store_info(store: int) -> dict:
    n, b = ctypes.c_int64(), ctypes.c_size_t()
    _check(lib().ie_store_info(store, ctypes.byref(n), ctypes.byref(b)), "ie_store_info")
    return {"n_blocks": n.value, "bytes": b.value}


def ie_store_release(store: int):
    _check(lib().ie_store_release(store), "ie_store_release")


def max_far_disp(box_ijk) -> int:
    """Largest |d_i| between two boxes of a scatterer: the reach a shared store needs."""
    ijk = np.asarray(box_ijk).reshape(-1, 3)
    return int((ijk.max(axis=0) - ijk.min(axis=0)).max()) if len(ijk) else 0


def ie_plan_footprint(problem: ie_problem) -> int:
    b = ctypes.c_size_t()
    _check(lib().ie_plan_footprint(ctypes.byref(problem), ctypes.byref(b)), "ie_plan_footprint")
    return b.value


def ie_plan_stats_get(plan: int) -> dict:
    s = ie_plan_stats()
    _check(lib().ie_plan_stats_get(plan, ctypes.byref(s)), "ie_plan_stats_get")
    return {f: getattr(s, f) for f, _ in s._fields_}


def ie_plan_profile(plan: int, enable: bool) -> None:
    _check(lib().ie_plan_profile(plan, 1 if enable else 0), "ie_plan_profile")


def ie_plan_destroy(plan: int) -> None:
    _check(lib().ie_plan_destroy(plan), "ie_plan_destroy")


def ie_matvec(plan, which, prec, c, y, nrhs, stream=None):
    n, _, _ = _dims(plan)
    _need(c, nrhs * n, "c")
    _need(y, nrhs * n, "y")
    return _check(lib().ie_matvec(plan, which, prec, _ptr(c), _ptr(y), nrhs, _stream(stream)), "ie_matvec")


def ie_aggregate(plan, c, X, nrhs, stream=None):
    n, nbox, _ = _dims(plan)
    _need(c, nrhs * n, "c")
    _need(X, nrhs * nbox * NU, "X")
    return _check(lib().ie_aggregate(plan, _ptr(c), _ptr(X), nrhs, _stream(stream)), "ie_aggregate")


def ie_translate(plan, prec, X, Y, nrhs, stream=None):
    _, nbox, _ = _dims(plan)
    _need(X, nrhs * nbox * NU, "X")
    _need(Y, nrhs * nbox * NU, "Y")
    return _check(lib().ie_translate(plan, prec, _ptr(X), _ptr(Y), nrhs, _stream(stream)), "ie_translate")


def ie_translate_noalloc(plan, X, Y, nrhs, stream=None):
    _, nbox, _ = _dims(plan)
    _need(X, nrhs * nbox * NU, "X")
    _need(Y, nrhs * nbox * NU, "Y")
    return _check(lib().ie_translate_noalloc(plan, _ptr(X), _ptr(Y), nrhs, _stream(stream)), "ie_translate_noalloc")


def ie_disaggregate(plan, Y, r, nrhs, stream=None):
    n, nbox, _ = _dims(plan)
    _need(Y, nrhs * nbox * NU, "Y")
    _need(r, nrhs * n, "r")
    return _check(lib().ie_disaggregate(plan, _ptr(Y), _ptr(r), nrhs, _stream(stream)), "ie_disaggregate")


def ie_near(plan, c, y, nrhs, stream=None):
    n, _, _ = _dims(plan)
    _need(c, nrhs * n, "c")
    _need(y, nrhs * n, "y")
    return _check(lib().ie_near(plan, _ptr(c), _ptr(y), nrhs, _stream(stream)), "ie_near")


def ie_coupling_blocks(plan, d, out, stream=None):
    d = np.ascontiguousarray(d, dtype=np.int32).reshape(-1, 3)
    _need(out, d.shape[0] * NU * NU, "out")
    return _check(lib().ie_coupling_blocks(plan, d.ctypes.data, d.shape[0], _ptr(out), _stream(stream)),
                  "ie_coupling_blocks")


def ie_map_basis(k, eta, box_edge, fun_off, pos, mom, n_samples=128, sample_radius=1.5, lattice=4,
                 tikhonov=0.0, residual=True, stream=None):
    """Rows of P for point-dipole basis functions (host arrays in, host arrays out).

    fun_off (n_fun+1,) int64; pos (m, 3) float64 relative to each function's box centre;
    mom (m, 3) complex128.  Returns (P (n_fun, 192) complex128, residual (n_fun,) or None).
    """
    fun_off = np.ascontiguousarray(fun_off, dtype=np.int64).reshape(-1)
    n_fun = fun_off.shape[0] - 1
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mom = np.ascontiguousarray(mom, dtype=np.complex128).reshape(-1, 3)
    if n_fun < 0 or pos.shape[0] != mom.shape[0] or pos.shape[0] < fun_off[-1]:
        raise ValueError("fun_off, pos and mom disagree")
    spec = ie_mapping_spec(k=k, eta=eta, box_edge=box_edge, lattice=lattice, n_samples=n_samples,
                           sample_radius=sample_radius, tikhonov=tikhonov)
    P = np.zeros((max(n_fun, 0), NU), dtype=np.complex128)
    res = np.zeros(max(n_fun, 0), dtype=np.float64) if residual else None
    _check(lib().ie_map_basis(ctypes.byref(spec), n_fun, fun_off.ctypes.data, pos.ctypes.data, mom.ctypes.data,
                              P.ctypes.data, None if res is None else res.ctypes.data, _stream(stream)),
           "ie_map_basis")
    return P, res


def ie_plan_blocks(plan) -> np.ndarray:
    """(n_coupling_blocks, 3) displacements of the stored far blocks, in block order."""
    n = int(ie_plan_stats_get(plan)["n_coupling_blocks"])
    out = np.zeros((n, 3), dtype=np.int32)
    _check(lib().ie_plan_blocks(plan, out.ctypes.data), "ie_plan_blocks")
    return out


def ie_sym_canon(d) -> tuple[np.ndarray, int]:
    """(c, q): the canonical displacement sorted |d| and the signed permutation index
    with d = Q c (host only)."""
    dd = np.ascontiguousarray(d, dtype=np.int32).reshape(3)
    c = np.zeros(3, dtype=np.int32)
    q = ctypes.c_int32()
    _check(lib().ie_sym_canon(dd.ctypes.data, c.ctypes.data, ctypes.byref(q)), "ie_sym_canon")
    return c, int(q.value)


def ie_sym_map() -> np.ndarray:
    """(48, 192) uint16: U_q(u), plus 0x100 where the unknown changes sign (host only)."""
    out = np.zeros((48, 192), dtype=np.uint16)
    _check(lib().ie_sym_map(out.ctypes.data), "ie_sym_map")
    return out


def ie_cvfcnn_set_weights(plan, W1, b1, W2, b2, stream=None):
    """Surrogate weights per stored block: W1 (blocks, H, 192), b1 (blocks, H),
    W2 (blocks, 192, H), b2 (blocks, 192), complex (converted to complex64)."""
    arrs = [np.ascontiguousarray(a, dtype=np.complex64) for a in (W1, b1, W2, b2)]
    st = ie_plan_stats_get(plan)
    nblk, H = int(st["n_coupling_blocks"]), int(st["cvfcnn_hidden"])
    shapes = [(nblk, H, NU), (nblk, H), (nblk, NU, H), (nblk, NU)]
    for a, shp, name in zip(arrs, shapes, ("W1", "b1", "W2", "b2")):
        if a.shape != shp:
            raise ValueError(f"{name} has shape {a.shape}, expected {shp}")
    _check(lib().ie_cvfcnn_set_weights(plan, *[a.ctypes.data for a in arrs], _stream(stream)),
           "ie_cvfcnn_set_weights")


def ie_cvfcnn_get_weights(plan, stream=None):
    """The plan's current surrogate weights (W1, b1, W2, b2), complex64, in the shapes
    ie_cvfcnn_set_weights takes."""
    st = ie_plan_stats_get(plan)
    nblk, H = int(st["n_coupling_blocks"]), int(st["cvfcnn_hidden"])
    arrs = [np.zeros(shp, dtype=np.complex64) for shp in [(nblk, H, NU), (nblk, H), (nblk, NU, H), (nblk, NU)]]
    _check(lib().ie_cvfcnn_get_weights(plan, *[a.ctypes.data for a in arrs], _stream(stream)),
           "ie_cvfcnn_get_weights")
    return tuple(arrs)


def ie_rhs_plane_wave(plan, khat, pol, v, stream=None):
    """khat, pol: (nrhs, 3), or (n_groups, nrhs, 3) for a batched plan; v: [nrhs][n]."""
    n, _, groups = _dims(plan)
    khat = np.ascontiguousarray(khat, dtype=np.float64)
    pol = np.ascontiguousarray(pol, dtype=np.float64)
    nrhs = khat.shape[-2] if khat.ndim >= 2 else 1
    if khat.size != groups * nrhs * 3 or pol.shape != khat.shape:
        raise ValueError(f"khat/pol must be ({groups}, nrhs, 3) for this plan, got {khat.shape} / {pol.shape}")
    _need(v, nrhs * n, "v")
    return _check(lib().ie_rhs_plane_wave(plan, khat.ctypes.data, pol.ctypes.data, nrhs, _ptr(v),
                                          _stream(stream)), "ie_rhs_plane_wave")


def solve_opts(**kw) -> ie_solve_opts:
    o = ie_solve_opts()
    lib().ie_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ie_solve(plan, v, c, nrhs, opts: ie_solve_opts | None = None, stream=None):
    """Returns (status, info dict); IE_ERR_NOT_CONVERGED is returned, not raised."""
    info = ie_solve_info()
    o = opts or solve_opts()
    n, _, _ = _dims(plan)
    _need(v, nrhs * n, "v")
    _need(c, nrhs * n, "c")
    st = lib().ie_solve(plan, _ptr(v), _ptr(c), nrhs, ctypes.byref(o), ctypes.byref(info), _stream(stream))
    _check(st, "ie_solve", allow=(IE_OK, IE_ERR_NOT_CONVERGED))
    return st, {f: getattr(info, f) for f, _ in info._fields_}


_solver_sizes: dict = {}     # solver handle -> elements of its v and c


def ie_solver_create(plan, nrhs, opts: ie_solve_opts | None = None) -> int:
    h = ctypes.c_void_p()
    o = opts or solve_opts()
    _check(lib().ie_solver_create(plan, nrhs, ctypes.byref(o), ctypes.byref(h)), "ie_solver_create")
    _solver_sizes[h.value] = nrhs * _dims(plan)[0]
    return h.value


def ie_solver_footprint(plan, nrhs, opts: ie_solve_opts | None = None) -> int:
    b = ctypes.c_size_t()
    o = opts or solve_opts()
    _check(lib().ie_solver_footprint(plan, nrhs, ctypes.byref(o), ctypes.byref(b)), "ie_solver_footprint")
    return b.value


def ie_solver_start(solver, v, c, stream=None):
    _need(v, _solver_sizes.get(solver, 0), "v")
    _need(c, _solver_sizes.get(solver, 0), "c")
    return _check(lib().ie_solver_start(solver, _ptr(v), _ptr(c), _stream(stream)), "ie_solver_start")


def ie_solver_advance(solver, cycles, stream=None):
    return _check(lib().ie_solver_advance(solver, cycles, _stream(stream)), "ie_solver_advance")


def ie_solver_poll(solver):
    done = ctypes.c_int()
    info = ie_solve_info()
    _check(lib().ie_solver_poll(solver, ctypes.byref(done), ctypes.byref(info)), "ie_solver_poll")
    return bool(done.value), {f: getattr(info, f) for f, _ in info._fields_}


def ie_diag_wait_limit(cycles: int):
    """Give-up limit of the tensor-core translation's pipeline waits (0 = default); tests only."""
    _check(lib().ie_diag_wait_limit(int(cycles)), "ie_diag_wait_limit")


IE_SOLVER_BUSY, IE_SOLVER_IDLE, IE_SOLVER_DONE = 0, 1, 2


def ie_solver_state(solver):
    """(state, info): IE_SOLVER_BUSY, IE_SOLVER_IDLE (advance again) or IE_SOLVER_DONE."""
    state = ctypes.c_int()
    info = ie_solve_info()
    _check(lib().ie_solver_state(solver, ctypes.byref(state), ctypes.byref(info)), "ie_solver_state")
    return state.value, {f: getattr(info, f) for f, _ in info._fields_}


def ie_solver_destroy(solver):
    _solver_sizes.pop(solver, None)
    return _check(lib().ie_solver_destroy(solver), "ie_solver_destroy")


def ie_plan_tune(plan, prec, nrhs, stream=None) -> dict:
    """Autotunes the tensor-core translation of `prec` for calls with nrhs columns."""
    info = ie_tune_info()
    _check(lib().ie_plan_tune(plan, prec, nrhs, ctypes.byref(info), _stream(stream)), "ie_plan_tune")
    return {f: getattr(info, f) for f, _ in info._fields_}


def cvfcnn_train_opts(**kw) -> ie_cvfcnn_train_opts:
    """ie_cvfcnn_train_opts with the library's defaults, fields overridden by kw."""
    o = ie_cvfcnn_train_opts()
    lib().ie_cvfcnn_train_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ie_cvfcnn_train(plan, opts: ie_cvfcnn_train_opts | None = None, stream=None) -> dict:
    """Trains the plan's translation networks (first stage of §3); returns the training info."""
    info = ie_cvfcnn_train_info()
    _check(lib().ie_cvfcnn_train(plan, ctypes.byref(opts) if opts is not None else None, ctypes.byref(info),
                                 _stream(stream)), "ie_cvfcnn_train")
    return {f: getattr(info, f) for f, _ in info._fields_}


def ie_plan_check(plan, stream=None):
    """IE_OK, or raises with IE_ERR_TIMEOUT when a translation gave up a bounded wait."""
    return _check(lib().ie_plan_check(plan, _stream(stream)), "ie_plan_check")


def ie_diag_bounded_wait(limit_ms: float = 50.0, stream=None) -> int:
    """Runs the bounded-wait diagnostic; returns its status (IE_ERR_TIMEOUT is the design)."""
    return int(lib().ie_diag_bounded_wait(float(limit_ms), _stream(stream)))


def ie_kernel_launches() -> int:
    return int(lib().ie_kernel_launches())


def ie_version() -> str:
    return lib().ie_version().decode()


class Store:
    """Owning wrapper of an ie_store handle (a shared coupling-block store)."""

    def __init__(self, spec: ie_store_spec, stream=None):
        self.spec = spec
        self.handle = ie_store_create(spec, stream)
        self.info = ie_store_info(self.handle)

    def close(self):
        if self.handle:
            ie_store_release(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper of an ie_plan handle; with `store` the plan attaches to a shared
    coupling-block store (ie_plan_create_shared)."""

    def __init__(self, problem: ie_problem, stream=None, store: Store | None = None):
        self.problem = problem
        if store is not None:
            self.handle = ie_plan_create_shared(problem, store.handle, stream)
        else:
            self.handle = ie_plan_create(problem, stream)
        self.stats = ie_plan_stats_get(self.handle)

    @property
    def n(self) -> int:
        return int(self.stats["n"])

    @property
    def n_boxes(self) -> int:
        return int(self.stats["n_boxes"])

    def close(self):
        if self.handle:
            ie_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
