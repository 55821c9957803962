"""FP64 CPU oracle of the group-by-group far-zone solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call this package; the product
path (the CUDA library and its Python binding) never does, and shares no code
with it.  The oracle takes plain numpy inputs and duck-typed problem objects
(attributes k, eta, a, lattice, G, box_ijk, nb, P, alpha, self_box_mode).

What each function follows (paper sections / equations / algorithms):

  dyad                  D(R), eq. 5 with psi from eq. 6 (C code, FP64)
  site_positions        uniform dipole lattice of each box, §2.1 ("uniform separation")
  aggregate             mapping to uniform basis functions, Alg. 1 (eq. 11 applied: x_b = P_b^T c_b)
  dipole_field          fields at dipole sites, eq. 12 summed over sources as eq. 14,
                        brute force one site pair at a time, far / near split of eq. 2
  disaggregate          inverse mapping, Alg. 3 (r_b = P_b y_b)
  far_matvec            Z^F c of eq. 2 by brute force
  operator              alpha c + Z^N c + Z^F c (the synthetic system Z I = V of eq. 1)
  coupling_block        translation matrix G_w of one displacement, eq. 13
  far_matvec_grouped    Alg. 2 grouped by displacement: E_j += G_w P_i per far pair
  gmres                 restarted GMRES without preconditioning (§5), FP64
  plane_wave_rhs        unit plane-wave excitation (§5) tested with P: v = P e
  fibonacci_sphere      sample points of the field-matching sphere S, §2.1
  mapping_matrix        A of eq. 10: fields of the uniform dipoles at the samples on S
  function_fields       B_k of eq. 10: fields of one point-dipole basis function on S
  map_basis             eq. 11, C_k = A^+ B_k (least squares), rows of P_b
  inverse_map_fields    eq. 15-17 literally: Q = (A^T)^+ E, tested on a basis function
  point_dipole_far      far interactions of the point-dipole basis functions themselves
                        (the original system that the mapping replaces), brute force
  cvfcnn_forward        the translation network of §3 (l-inf input scaling, one hidden
                        layer with the Cartesian ReLU, linear output, rescaling)
  cvfcnn_fit            closed-form weights: the network in its linear regime equal to
                        the truncated SVD of a translation matrix (numpy's SVD)
  cvfcnn_far_matvec     Alg. 2 with the networks in place of eq. 13's matrices

Parity status: every function above is pinned by the CPU tests in
tests/test_oracle_pins.py (closed-form Hertzian dipole field, reciprocity,
translation invariance, counts printed in §2.2, brute force vs grouped, dense
LU vs GMRES, explicit pure-Python construction on a tiny case; for the mapping:
the Fibonacci lattice's closed form, exact reproduction of a uniform dipole,
superposition, the least-squares normal equations, the far field of the
equivalent dipoles against the source's own field, and the inverse mapping
computed literally against the transpose of the forward one).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

FAR, NEAR, ALL = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the C part (gcc, OpenMP) in-tree."""
    src = os.path.join(_HERE, "ie_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.or_dyad.argtypes = [d, d, p, p]
        L.or_site_positions.argtypes = [d, i, i, i64, p, p]
        L.or_dipole_field.argtypes = [d, d, d, i, i, i64, p, p, i, i, i64, p, p]
        L.or_coupling_block.argtypes = [d, d, d, i, p, p]
        L.or_coupling_blocks.argtypes = [d, d, d, i, i64, p, p]
        L.or_plane_wave.argtypes = [d, d, i, i, i64, p, i64, p, p, p]
        L.or_point_dipole_far.argtypes = [d, d, i64, p, p, p, p, p, p, p, p]
        L.or_point_fields.argtypes = [d, d, i64, p, i64, p, p, p]
        L.or_num_threads.restype = i
        _lib = L
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


# ---------------------------------------------------------------- eq. 5, eq. 6
def dyad(k: float, eta: float, R) -> np.ndarray:
    """Free-space dyadic Green's function D(R) (eq. 5, psi of eq. 6), 3x3 complex."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(9, dtype=np.complex128)
    _load().or_dyad(k, eta, _ptr(R), _ptr(out))
    return out.reshape(3, 3)


def nu_of(p) -> int:
    return 3 * p.lattice ** 3


def site_positions(p) -> np.ndarray:
    """(n_boxes, L^3, 3) dipole positions: box centre a(ijk + 1/2 - G/2) + cell-centred offset."""
    ijk = np.ascontiguousarray(p.box_ijk, dtype=np.int32)
    ns = p.lattice ** 3
    pos = np.zeros((ijk.shape[0], ns, 3))
    _load().or_site_positions(p.a, p.lattice, p.G, ijk.shape[0], _ptr(ijk), _ptr(pos))
    return pos


def _offsets(p) -> np.ndarray:
    o = np.zeros(len(p.nb) + 1, dtype=np.int64)
    np.cumsum(np.asarray(p.nb, dtype=np.int64), out=o[1:])
    return o


def _P_block(p, b: int) -> np.ndarray:
    if p.P is None:
        return np.eye(nu_of(p), dtype=np.complex128)
    o = _offsets(p)
    return p.P[o[b]:o[b + 1]]


# ---------------------------------------------------------------- Alg. 1 / Alg. 3
def aggregate(p, c) -> np.ndarray:
    """Alg. 1: per box, x_b = P_b^T c_b.  c: [nrhs][n] -> X: [nrhs][n_boxes][192]."""
    c = _c128(c).reshape(-1, int(np.sum(p.nb)))
    nrhs = c.shape[0]
    o = _offsets(p)
    X = np.zeros((nrhs, len(p.nb), nu_of(p)), dtype=np.complex128)
    for b in range(len(p.nb)):
        X[:, b, :] = c[:, o[b]:o[b + 1]] @ _P_block(p, b)      # (P_b^T c_b)^T
    return X


def disaggregate(p, Y, boxes=None) -> np.ndarray:
    """Alg. 3: per box, r_b = P_b y_b.  Y: [nrhs][len(boxes)][192] -> [nrhs][sum nb over boxes]."""
    Y = _c128(Y)
    boxes = np.arange(len(p.nb)) if boxes is None else np.asarray(boxes)
    parts = [Y[:, i, :] @ _P_block(p, int(b)).T for i, b in enumerate(boxes)]
    return np.concatenate(parts, axis=1)


def basis_rows(p, boxes) -> np.ndarray:
    """Indices into the basis vector of the listed boxes (in the listed order)."""
    o = _offsets(p)
    return np.concatenate([np.arange(o[b], o[b + 1]) for b in boxes])


# ---------------------------------------------------------------- eq. 12-14, brute force
def dipole_field(p, X, mode: int, targets=None) -> np.ndarray:
    """Brute-force field at the dipole sites of the target boxes (eq. 12 summed as eq. 14).

    X: [nrhs][n_boxes][192] dipole moments.  mode FAR / NEAR / ALL (one-box-buffer split).
    Returns [nrhs][n_targets][192].
    """
    X = _c128(X)
    nrhs, nbox, nu = X.shape
    ijk = np.ascontiguousarray(p.box_ijk, dtype=np.int32)
    targets = np.arange(nbox, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    Y = np.zeros((nrhs, len(targets), nu), dtype=np.complex128)
    L = _load()
    for r in range(nrhs):
        xr = np.ascontiguousarray(X[r])
        yr = np.zeros((len(targets), nu), dtype=np.complex128)
        L.or_dipole_field(p.k, p.eta, p.a, p.lattice, p.G, nbox, _ptr(ijk), _ptr(xr), mode,
                          int(getattr(p, "self_box_mode", 0)), len(targets), _ptr(targets), _ptr(yr))
        Y[r] = yr
    return Y


def far_matvec(p, c, targets=None) -> np.ndarray:
    """Z^F c of eq. 2 by brute force: P (sum over far site pairs of D) P^T c.

    Returns the rows of the target boxes ([nrhs][sum nb over targets]).
    """
    X = aggregate(p, c)
    targets = np.arange(len(p.nb)) if targets is None else np.asarray(targets)
    Y = dipole_field(p, X, FAR, targets)
    return disaggregate(p, Y, targets)


def operator(p, c, which: str = "full", targets=None) -> np.ndarray:
    """Z c restricted to the target boxes' rows, brute force.

    which: 'far'  -> Z^F c;  'near' -> alpha c + Z^N c (stored near part and self term);
           'full' -> alpha c + Z^N c + Z^F c.
    """
    c = _c128(c).reshape(-1, int(np.sum(p.nb)))
    targets = np.arange(len(p.nb)) if targets is None else np.asarray(targets)
    X = aggregate(p, c)
    mode = {"far": FAR, "near": NEAR, "full": ALL}[which]
    Y = dipole_field(p, X, mode, targets)
    out = disaggregate(p, Y, targets)
    if which != "far":
        out = out + p.alpha * c[:, basis_rows(p, targets)]
    return out


# ---------------------------------------------------------------- eq. 13, Alg. 2 grouped
def coupling_block(p, d) -> np.ndarray:
    """Translation matrix of box displacement d (test box = basis box + d), eq. 13."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    nu = nu_of(p)
    C = np.zeros((nu, nu), dtype=np.complex128)
    _load().or_coupling_block(p.k, p.eta, p.a, p.lattice, _ptr(d), _ptr(C))
    return C


def coupling_blocks(p, ds) -> np.ndarray:
    ds = np.ascontiguousarray(ds, dtype=np.int32).reshape(-1, 3)
    nu = nu_of(p)
    C = np.zeros((ds.shape[0], nu, nu), dtype=np.complex128)
    _load().or_coupling_blocks(p.k, p.eta, p.a, p.lattice, ds.shape[0], _ptr(ds), _ptr(C))
    return C


def pair_groups(p, mode: int):
    """Ordered box pairs (basis b -> test t) grouped by displacement d = ijk_t - ijk_b.

    mode FAR: Chebyshev distance >= 2 (Alg. 2 test ||w|| >= 2a on the box lattice);
    NEAR: <= 1 (with self_box_mode = 1 the d = 0 group is dropped); ALL: both.
    Returns (ds (ng,3) int32, list of (src slots, dst slots)).
    """
    ijk = np.asarray(p.box_ijk, dtype=np.int64)
    n = ijk.shape[0]
    d = ijk[None, :, :] - ijk[:, None, :]           # d[b, t] = ijk_t - ijk_b
    ch = np.abs(d).max(-1)
    sel = np.zeros((n, n), dtype=bool)
    if mode & FAR:
        sel |= ch >= 2
    if mode & NEAR:
        near = ch <= 1
        if int(getattr(p, "self_box_mode", 0)) == 1:
            near &= ch != 0
        sel |= near
    b_idx, t_idx = np.nonzero(sel)
    dd = d[b_idx, t_idx]
    span = 2 * int(np.abs(dd).max(initial=0)) + 1
    key = ((dd[:, 0] + span) * (2 * span + 1) + (dd[:, 1] + span)) * (2 * span + 1) + (dd[:, 2] + span)
    order = np.argsort(key, kind="stable")
    key, b_idx, t_idx, dd = key[order], b_idx[order], t_idx[order], dd[order]
    starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    ends = np.r_[starts[1:], len(key)]
    ds = dd[starts].astype(np.int32)
    groups = [(b_idx[s:e], t_idx[s:e]) for s, e in zip(starts, ends)]
    return ds, groups


def dipole_field_grouped(p, X, mode: int, chunk: int = 256) -> np.ndarray:
    """Alg. 2 with DGFA, grouped by displacement: for every pair, E_t += G_d P_b.

    Each displacement's translation matrix (eq. 13) multiplies all of that
    displacement's basis-box vectors at once (a library matmul).
    """
    X = _c128(X)
    nrhs, nbox, nu = X.shape
    ds, groups = pair_groups(p, mode)
    Y = np.zeros_like(X)
    for s in range(0, len(ds), chunk):
        Cs = coupling_blocks(p, ds[s:s + chunk])
        for i, (src, dst) in enumerate(groups[s:s + chunk]):
            Y[:, dst, :] += np.einsum("uv,rnv->rnu", Cs[i], X[:, src, :], optimize=True)
    return Y


def far_matvec_grouped(p, c) -> np.ndarray:
    return disaggregate(p, dipole_field_grouped(p, aggregate(p, c), FAR))


def operator_grouped(p, c, which: str = "full") -> np.ndarray:
    c = _c128(c).reshape(-1, int(np.sum(p.nb)))
    mode = {"far": FAR, "near": NEAR, "full": ALL}[which]
    out = disaggregate(p, dipole_field_grouped(p, aggregate(p, c), mode))
    if which != "far":
        out = out + p.alpha * c
    return out


# ---------------------------------------------------------------- excitation (§5)
def plane_wave_fields(p, khat, pol) -> np.ndarray:
    """Plane-wave samples at every dipole: [nrhs][n_boxes][192]."""
    khat = np.ascontiguousarray(khat, dtype=np.float64).reshape(-1, 3)
    pol = np.ascontiguousarray(pol, dtype=np.float64).reshape(-1, 3)
    ijk = np.ascontiguousarray(p.box_ijk, dtype=np.int32)
    e = np.zeros((khat.shape[0], ijk.shape[0], nu_of(p)), dtype=np.complex128)
    _load().or_plane_wave(p.k, p.a, p.lattice, p.G, ijk.shape[0], _ptr(ijk), khat.shape[0],
                          _ptr(khat), _ptr(pol), _ptr(e))
    return e


def plane_wave_rhs(p, khat, pol) -> np.ndarray:
    """Excitation vector tested with the basis functions: v = P e, [nrhs][n]."""
    return disaggregate(p, plane_wave_fields(p, khat, pol))


# ---------------------------------------------------------------- GMRES (§5), FP64
def gmres(matvec, b, restart: int = 50, tol: float = 1e-10, maxiter: int = 1000):
    """Restarted GMRES(m), x0 = 0, no preconditioner, modified Gram-Schmidt twice,
    Givens rotations on the Hessenberg matrix.  Stops when the recurrence residual
    is <= tol * ||b||.  Returns (x, iterations, history of relative residuals)."""
    b = _c128(b)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, [0.0]
    hist = []
    it = 0
    r = b.copy()
    beta = np.linalg.norm(r)
    hist.append(beta / bn)
    while it < maxiter and beta > tol * bn:
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = matvec(V[j])
            for _ in range(2):
                for i in range(j + 1):
                    h = np.vdot(V[i], w)
                    H[i, j] += h
                    w = w - h * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            # rotation [c s; -conj(s) c] with c real that zeroes H[j+1, j]
            a_, b_ = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            elif abs(a_) == 0:
                cs[j], sn[j] = 0.0, np.conj(b_) / abs(b_)
            else:
                cs[j] = abs(a_) / den
                sn[j] = (a_ / abs(a_)) * np.conj(b_) / den
            H[j, j] = cs[j] * a_ + sn[j] * b_
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) <= tol * bn or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / bn
    return x, it, hist


# ---------------------------------------------------------------- small dense forms
def dense_operator(p) -> np.ndarray:
    """Z = alpha I + P D_off P^T as a dense matrix, assembled box pair by box pair
    from the translation matrices (near pairs included, coincident dipoles excluded)."""
    n = int(np.sum(p.nb))
    o = _offsets(p)
    Z = np.zeros((n, n), dtype=np.complex128)
    ds, groups = pair_groups(p, ALL)
    Cs = coupling_blocks(p, ds)
    for i, (src, dst) in enumerate(groups):
        for b, t in zip(src, dst):
            Z[o[t]:o[t + 1], o[b]:o[b + 1]] += _P_block(p, t) @ Cs[i] @ _P_block(p, b).T
    Z += p.alpha * np.eye(n)
    return Z


def operator_norm(p, iters: int = 30, seed: int = 7, matvec=None, log=None):
    """sigma = ||P D_off P^T||_2 by power iteration on K^H K (K complex symmetric,
    so K^H v = conj(K conj(v))).  Returns (sigma, history)."""
    n = int(np.sum(p.nb))
    g = np.random.Generator(np.random.PCG64(seed))
    v = g.standard_normal(n) + 1j * g.standard_normal(n)
    v /= np.linalg.norm(v)

    if matvec is None:
        class _K:
            pass
        q = _K()
        for name in ("k", "eta", "a", "lattice", "G", "box_ijk", "nb", "P", "self_box_mode"):
            setattr(q, name, getattr(p, name))
        q.alpha = 0.0
        K = lambda c: operator_grouped(q, c[None, :], "full")[0]  # noqa: E731
    else:
        K = matvec
    hist = []
    sigma = 0.0
    for it in range(iters):
        t0 = time.time()
        w = K(v)
        sigma = np.linalg.norm(w)
        u = np.conj(K(np.conj(w)))
        v = u / np.linalg.norm(u)
        hist.append(float(sigma))
        if log:
            log(f"power it {it}: sigma {sigma:.6e} ({time.time() - t0:.1f}s)")
    return float(sigma), hist


# ---------------------------------------------------------------- §2.1 mapping, eq. 9-11 / 15-17
GOLDEN_RATIO = 0.5 + 0.5 * 5.0 ** 0.5


def fibonacci_sphere(n: int, radius: float) -> np.ndarray:
    """(n, 3) spherical Fibonacci lattice of §2.1 about the box centre: point l = 0..n-1 at
    polar angle arccos(1 - (2l+1)/n) and azimuth 2 pi l / golden ratio.  (The printed
    formulas give the two angles the other names; the arccos one is the polar angle.)"""
    l = np.arange(n, dtype=np.float64)
    polar = np.arccos(1.0 - (2.0 * l + 1.0) / n)
    azim = 2.0 * np.pi * l / GOLDEN_RATIO
    return radius * np.stack([np.sin(polar) * np.cos(azim), np.sin(polar) * np.sin(azim), np.cos(polar)], 1)


def lattice_offsets(a: float, L: int) -> np.ndarray:
    """(L^3, 3) uniform dipole positions relative to their box centre (site order of site_positions)."""
    pos = np.zeros((1, L ** 3, 3))
    ijk = np.zeros((1, 3), dtype=np.int32)
    _load().or_site_positions(a, L, 1, 1, _ptr(ijk), _ptr(pos))
    return pos[0]


def mapping_matrix(k: float, eta: float, a: float, L: int, n_samples: int, radius_rel: float = 1.5):
    """A of eq. 10, (3 n_samples, 3 L^3): entry (3l + alpha, 3j + beta) is the alpha component
    of the field at sample l on S (radius radius_rel * a) of a unit beta-directed dipole at
    uniform site j.  Returns (A, samples)."""
    S = fibonacci_sphere(n_samples, radius_rel * a)
    sites = lattice_offsets(a, L)
    A = np.zeros((3 * n_samples, 3 * len(sites)), dtype=np.complex128)
    for l, r in enumerate(S):
        for j, q in enumerate(sites):
            A[3 * l:3 * l + 3, 3 * j:3 * j + 3] = dyad(k, eta, r - q)
    return A, S


def point_fields(k: float, eta: float, obs, src, mom) -> np.ndarray:
    """(n_obs, 3) field at obs of point dipoles (src (n, 3), complex moments mom (n, 3)):
    eq. 4 with the integral a sum, brute force in C."""
    obs = np.ascontiguousarray(obs, dtype=np.float64).reshape(-1, 3)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    m = _c128(np.asarray(mom).reshape(-1, 3))
    out = np.zeros((obs.shape[0], 3), dtype=np.complex128)
    _load().or_point_fields(k, eta, obs.shape[0], _ptr(obs), src.shape[0], _ptr(src), _ptr(m), _ptr(out))
    return out


def function_fields(k: float, eta: float, samples, pos, mom) -> np.ndarray:
    """B_k of eq. 10 for a basis function made of point dipoles (positions pos (m, 3)
    relative to the box centre, complex moments mom (m, 3)): its field at the samples,
    stacked (3 n_samples,)."""
    return point_fields(k, eta, samples, pos, mom).reshape(-1)


def map_basis(k, eta, a, L, n_samples, radius_rel, fun_off, pos, mom, tikhonov: float = 0.0):
    """Eq. 11 for every basis function: C_k = A^+ B_k, the least-squares coefficients of
    the uniform dipoles whose field best matches the function's field on S (eq. 9-10).
    Function f owns point dipoles fun_off[f] .. fun_off[f+1]-1.  Returns (P, residual):
    P (n_fun, 3 L^3) with row f = C_f^T, residual[f] = ||A C_f - B_f|| / ||B_f||.
    tikhonov = t > 0 (not in the paper) adds (t ||A||_F)^2 ||C_k||^2 to the squared misfit,
    i.e. the least-squares problem [A; t ||A||_F I] C_k ~ [B_k; 0]."""
    A, S = mapping_matrix(k, eta, a, L, n_samples, radius_rel)
    n_fun = len(fun_off) - 1
    mom = np.asarray(mom, dtype=np.complex128).reshape(-1, 3)
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    B = np.zeros((A.shape[0], n_fun), dtype=np.complex128)
    for f in range(n_fun):
        lo, hi = int(fun_off[f]), int(fun_off[f + 1])
        if hi > lo:
            B[:, f] = function_fields(k, eta, S, pos[lo:hi], mom[lo:hi])
    if tikhonov > 0:
        lam = tikhonov * np.linalg.norm(A)
        nu = A.shape[1]
        C = np.linalg.lstsq(np.vstack([A, lam * np.eye(nu)]), np.vstack([B, np.zeros((nu, n_fun))]), rcond=None)[0]
    else:
        C = np.linalg.lstsq(A, B, rcond=None)[0]
    nb = np.linalg.norm(B, axis=0)
    res = np.where(nb > 0, np.linalg.norm(A @ C - B, axis=0) / np.where(nb > 0, nb, 1.0), 0.0)
    return C.T.copy(), res


def inverse_map_fields(k, eta, a, L, n_samples, radius_rel, E, pos, mom) -> complex:
    """Eq. 15-17 as written, for one test function: the virtual dipoles on S get the
    coefficients Q = (A^T)^+ E that best reproduce the fields E (3 L^3,) at the uniform
    sites (eq. 16-17); their field is then tested on the function (point dipoles pos, mom):
    sum over its dipoles of mom . E_vd(pos) with E_vd from eq. 15."""
    A, S = mapping_matrix(k, eta, a, L, n_samples, radius_rel)
    Q = np.linalg.lstsq(A.T, np.asarray(E, dtype=np.complex128), rcond=None)[0]
    total = 0.0 + 0.0j
    for x, p in zip(np.atleast_2d(pos), np.atleast_2d(np.asarray(mom, dtype=np.complex128))):
        field = np.zeros(3, dtype=np.complex128)
        for l, r in enumerate(S):
            field += dyad(k, eta, x - r) @ Q[3 * l:3 * l + 3]
        total += p @ field
    return total


def point_dipole_far(p, fun_off, pos, mom, c, targets=None) -> np.ndarray:
    """Far part of the original subdomain system for point-dipole basis functions (box b's
    functions are listed in box order, p.nb[b] of them; pos relative to each box centre):
    y_f = sum over dipoles d of f of mom_d . E(r_d), E the field of c_g-weighted dipoles of
    every function g in a box at Chebyshev distance >= 2 (eq. 3-4 with point sources).
    targets: box slots whose functions are computed (the result then holds those rows,
    in basis_rows order); None = all."""
    fun_off = np.ascontiguousarray(fun_off, dtype=np.int64)
    n_fun = len(fun_off) - 1
    fun_box = np.repeat(np.arange(p.n_boxes, dtype=np.int32), np.asarray(p.nb, dtype=np.int64))
    assert len(fun_box) == n_fun
    ijk = np.ascontiguousarray(p.box_ijk, dtype=np.int32)
    centre = p.a * (ijk.astype(np.float64) + 0.5 - p.G / 2.0)
    counts = np.diff(fun_off)
    dip_box = np.repeat(fun_box, counts)
    absolute = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3) + centre[dip_box])
    m = _c128(np.asarray(mom).reshape(-1, 3))
    cc = _c128(np.asarray(c).reshape(-1))
    out = np.zeros(n_fun, dtype=np.complex128)
    want = None
    if targets is not None:
        rows = basis_rows(p, targets)
        want = np.zeros(n_fun, dtype=np.uint8)
        want[rows] = 1
    _load().or_point_dipole_far(p.k, p.eta, n_fun, _ptr(fun_off), _ptr(fun_box), _ptr(ijk), _ptr(absolute),
                                _ptr(m), _ptr(cc), None if want is None else _ptr(want), _ptr(out))
    return out if targets is None else out[basis_rows(p, targets)]


# ---------------------------------------------------------------- §3 translation networks
def cvfcnn_forward(W1, b1, W2, b2, x) -> np.ndarray:
    """The network of §3 on inputs x (..., 192): s = max_u |x_u|, z = W1 (x / s) + b1,
    h = max(Re z, 0) + j max(Im z, 0) (Cartesian ReLU), output s (W2 h + b2); 0 for x = 0."""
    x = _c128(x)
    s = np.abs(x).max(axis=-1, keepdims=True)
    safe = np.where(s > 0, s, 1.0)
    z = (x / safe) @ np.asarray(W1).T + b1
    h = np.maximum(z.real, 0.0) + 1j * np.maximum(z.imag, 0.0)
    o = h @ np.asarray(W2).T + b2
    return np.where(s > 0, s * o, 0.0)


def cvfcnn_fit(C, H: int):
    """Weights of a width-H network whose output on the unit l-inf ball is U_H S_H V_H^H x,
    the truncated SVD of C (the best rank-H approximation): W1 = V_H^H, W2 = U_H S_H,
    b1_h = beta_h (1 + j) with beta_h = sum_u |W1_hu| (so Re and Im of W1 x + b1 stay >= 0
    for |x_u| <= 1 and the ReLU passes them), b2 = -W2 b1."""
    U, S, Vh = np.linalg.svd(_c128(C))
    W1 = Vh[:H].copy()
    W2 = U[:, :H] * S[:H]
    b1 = np.abs(W1).sum(axis=1) * (1.0 + 1.0j)
    b2 = -W2 @ b1
    return W1, b1, W2, b2


def signed_permutation(Q, L: int) -> np.ndarray:
    """S_Q (3 L^3 x 3 L^3) with G_{Qd} = S_Q G_d S_Q^T: site s goes where Q takes its
    centred lattice offset, and its 3 components transform by Q."""
    Q = np.asarray(Q, dtype=np.float64)
    ns = L ** 3
    S = np.zeros((3 * ns, 3 * ns))
    for s in range(ns):
        ii = np.array([s % L, (s // L) % L, s // (L * L)])
        jj = (Q @ (ii + 0.5 - L / 2.0) + L / 2.0 - 0.5).round().astype(int)
        s2 = jj[0] + L * jj[1] + L * L * jj[2]
        S[3 * s2:3 * s2 + 3, 3 * s:3 * s + 3] = Q
    return S


def canonical_frame(d):
    """(c, Q): c = |d| sorted ascending and a signed permutation Q with Q c = d."""
    d = np.asarray(d, dtype=np.int64)
    order = np.argsort(np.abs(d), kind="stable")
    c = np.abs(d)[order]
    Q = np.zeros((3, 3))
    for k, axis in enumerate(order):
        Q[axis, k] = 1.0 if d[axis] >= 0 else -1.0
    return c, Q


def cvfcnn_far_matvec(p, c, H: int = 50, weights=None, targets=None, frames: bool = False) -> np.ndarray:
    """Z^F c with Alg. 2's translation E_t += G_d x_b replaced by the network of d.
    weights None: each canonical c = sorted |d| gets cvfcnn_fit(G_c, H), applied to
    displacement d = Q c in the frame of c: y = S_Q net_c(S_Q^T x).  weights: a dict
    from displacement tuples to (W1, b1, W2, b2), applied directly; with frames=True
    its keys are canonical c and each d = Q c uses net_c in the frame of c as above."""
    X = aggregate(p, c)
    nrhs = X.shape[0]
    ds, groups = pair_groups(p, FAR)
    tset = None if targets is None else set(int(t) for t in targets)
    Y = np.zeros_like(X)
    fitted = {}
    for d, (src, dst) in zip(ds, groups):
        src = np.asarray(src)
        dst = np.asarray(dst)
        if tset is not None:
            keep = np.array([int(t) in tset for t in dst], dtype=bool)
            src, dst = src[keep], dst[keep]
        if len(src) == 0:
            continue
        if weights is not None and not frames:
            net, S = weights[tuple(int(v) for v in d)], None
        elif weights is not None:
            cc, Q = canonical_frame(d)
            net, S = weights[tuple(int(v) for v in cc)], signed_permutation(Q, p.lattice)
        else:
            cc, Q = canonical_frame(d)
            key = tuple(int(v) for v in cc)
            if key not in fitted:
                fitted[key] = cvfcnn_fit(coupling_block(p, np.array(key, dtype=np.int32)), H)
            net, S = fitted[key], signed_permutation(Q, p.lattice)
        for r in range(nrhs):
            xin = X[r, src]
            if S is not None:
                xin = xin @ S                  # rows (S^T x)^T
            out = cvfcnn_forward(*net, xin)
            if S is not None:
                out = out @ S.T                # rows (S o)^T
            np.add.at(Y[r], dst, out)
    if targets is None:
        return disaggregate(p, Y)
    targets = np.asarray(targets)
    return disaggregate(p, Y[:, targets], boxes=targets)
