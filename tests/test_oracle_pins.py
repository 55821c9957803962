"""Pins of the FP64 CPU oracle against facts fixed outside it.

Each test ties one oracle function to something other than its own formula:
the textbook Hertzian-dipole field in spherical components, the limits of the
dyad, rotation covariance, counts printed in §2.2, brute force vs the grouped
evaluation of Alg. 2, an explicit pure-Python assembly on a tiny case, dense LU
vs GMRES, and properties of the plane-wave excitation.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

K, ETA = W.K0, W.ETA0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers
def hertz_field(k, eta, R, p):
    """Field of a Hertzian dipole of moment p at offset R, written in the dipole's own
    spherical frame (E_r, E_theta; textbook form, exp(+j w t)), then mapped to xyz."""
    R = np.asarray(R, float)
    p = np.asarray(p, complex)
    r = np.linalg.norm(R)
    rh = R / r
    out = np.zeros(3, complex)
    # split a complex moment into two real-direction dipoles (linearity)
    for part, scale in ((p.real, 1.0), (p.imag, 1j)):
        m = np.linalg.norm(part)
        if m == 0:
            continue
        z = part / m
        ct = float(np.dot(rh, z))
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        ph = np.exp(-1j * k * r)
        Er = eta * m * ct * ph / (2 * math.pi * r ** 2) * (1 + 1 / (1j * k * r))
        Et = 1j * k * eta * m * st * ph / (4 * math.pi * r) * (1 + 1 / (1j * k * r) - 1 / (k * r) ** 2)
        th = (ct * rh - z) / st if st > 0 else np.zeros(3)
        out += scale * (Er * rh + Et * th)
    return out


def signed_permutations():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            Q = np.zeros((3, 3))
            for i in range(3):
                Q[i, perm[i]] = signs[i]
            yield Q


class Tiny:
    """A duck-typed problem for hand-built cases."""

    def __init__(self, boxes, G, L, nb, seed, alpha=0.0, identity=False):
        self.k, self.eta, self.a, self.lattice, self.G = K, ETA, W.BOX_EDGE, L, G
        self.box_ijk = np.asarray(boxes, dtype=np.int32)
        nu = 3 * L ** 3
        self.nb = np.full(len(boxes), nu if identity else nb, dtype=np.int32)
        g = W.rng(seed)
        self.P = None if identity else W.complex_normal(g, (int(self.nb.sum()), nu))
        self.alpha = alpha
        self.self_box_mode = 0


# ------------------------------------------------------------------ eq. 5 / eq. 6
@pytest.mark.parametrize("kr", [1e-2, 0.3, 1.0, 2.5, 9.0, 80.0])
def test_dyad_is_the_hertzian_dipole_field(kr):
    g = W.rng(100)
    for _ in range(20):
        R = g.standard_normal(3)
        R *= (kr / K) / np.linalg.norm(R)
        p = g.standard_normal(3) + 1j * g.standard_normal(3)
        got = oracle.dyad(K, ETA, R) @ p
        ref = hertz_field(K, ETA, R, p)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_dyad_scales_with_k_and_eta():
    R = np.array([0.2, -0.1, 0.35])
    for k in (0.5, 2 * math.pi, 40.0):
        for eta in (1.0, ETA):
            p = np.array([0.3, 1.0 - 0.2j, -0.5j])
            assert np.allclose(oracle.dyad(k, eta, R) @ p, hertz_field(k, eta, R, p), rtol=1e-12, atol=0)


def test_dyad_symmetries_and_rotation_covariance():
    g = W.rng(101)
    for _ in range(10):
        R = g.standard_normal(3)
        D = oracle.dyad(K, ETA, R)
        assert np.allclose(D, D.T, rtol=0, atol=1e-12 * np.abs(D).max())
        assert np.allclose(oracle.dyad(K, ETA, -R), D, rtol=0, atol=1e-12 * np.abs(D).max())
        Q, _ = np.linalg.qr(g.standard_normal((3, 3)))
        DQ = oracle.dyad(K, ETA, Q @ R)
        assert np.allclose(DQ, Q @ D @ Q.T, rtol=0, atol=1e-11 * np.abs(D).max())


def test_dyad_static_and_radiation_limits():
    R = np.array([0.3, 0.4, 1.2])
    rh = R / np.linalg.norm(R)
    I3 = np.eye(3)
    # static limit kR -> 0: D ~ psi * (-1/(kR)^2) (I - 3 Rhat Rhat)
    k = 1e-5 / np.linalg.norm(R)
    r = np.linalg.norm(R)
    psi = -1j * k * ETA * np.exp(-1j * k * r) / (4 * math.pi * r)
    lim = psi * (-1.0 / (k * r) ** 2) * (I3 - 3 * np.outer(rh, rh))
    D = oracle.dyad(k, ETA, R)
    assert np.linalg.norm(D - lim) <= 1e-4 * np.linalg.norm(lim)
    # radiation limit kR -> inf: D ~ psi (I - Rhat Rhat)
    k = 1e6 / r
    psi = -1j * k * ETA * np.exp(-1j * k * r) / (4 * math.pi * r)
    lim = psi * (I3 - np.outer(rh, rh))
    D = oracle.dyad(k, ETA, R)
    assert np.linalg.norm(D - lim) <= 1e-5 * np.linalg.norm(lim)


def _sph_j0_j2(x):
    """Spherical Bessel j0, j2 from their power series x^l sum_n (-x^2/2)^n / (n! (2n+2l+1)!!)."""
    def series(l):
        term, total, n = x ** l / math.prod(range(2 * l + 1, 0, -2)), 0.0, 0
        while abs(term) > 1e-30 * max(abs(total), 1e-300) or n < 3:
            total += term
            n += 1
            term *= (-x * x / 2) / (n * (2 * n + 2 * l + 1))
        return total
    return series(0), series(2)


@pytest.mark.parametrize("kr", [1e-3, 6e-3, 0.031, 0.3, 2.0])
def test_dyad_radiative_part_in_the_low_frequency_regime(kr):
    """Re D = -k eta (I + grad grad / k^2) sin(kR)/(4 pi R) is regular at R = 0; written with
    spherical Bessel functions it is -(k^2 eta / 4 pi) [(2/3 j0 - j2/3) I + j2 Rhat Rhat].  At
    small kR eq. 5-6 reach it through a cancellation of 1/(kR) terms, so the FP64 dyad keeps
    about eps/(kR)^2 of relative accuracy: the budget the low-frequency workloads rely on."""
    g = W.rng(104)
    j0, j2 = _sph_j0_j2(kr)
    for _ in range(10):
        R = g.standard_normal(3)
        R *= (kr / K) / np.linalg.norm(R)
        rh = R / np.linalg.norm(R)
        ref = -(K * K * ETA / (4 * math.pi)) * ((2 / 3 * j0 - j2 / 3) * np.eye(3) + j2 * np.outer(rh, rh))
        D = oracle.dyad(K, ETA, R)
        assert np.abs(D.real - ref).max() <= (2e-15 / kr ** 2 + 1e-14) * np.abs(ref).max()
        # the static part dominates the reactive (imaginary) part by about 3/(kR)^3
        if kr < 0.1:
            assert np.abs(D.imag).max() >= 1.0 / kr ** 3 * np.abs(ref).max()


# ------------------------------------------------------------------ §2.2 counts
def test_translation_vector_counts_printed_in_the_paper():
    gold = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    p = W.tiny()
    ds, groups = oracle.pair_groups(p, oracle.FAR)
    assert len(ds) == gold["far_translation_vectors"] == 316
    canon = {tuple(sorted(np.abs(d))) for d in ds}
    assert len(canon) == gold["unique_translation_matrices"] == 16
    # the 48-element signed-permutation group gives the same 16 classes
    classes = set()
    for d in ds:
        orbit = tuple(sorted({tuple((Q @ d).astype(int)) for Q in signed_permutations()}))
        classes.add(orbit)
    assert len(classes) == 16
    assert sum(len(s) for s, _ in groups) == gold["derived"]["far_box_pairs_all_occupied"]
    dn, gn = oracle.pair_groups(p, oracle.NEAR)
    adj = sum(len(s) for d, (s, _) in zip(dn, gn) if np.abs(d).max() == 1)
    assert adj == gold["derived"]["adjacent_box_pairs_all_occupied"]


def test_translation_matrices_related_by_symmetry():
    """C_{Qd} = S_Q C_d S_Q^T with S_Q = (lattice-site map) x Q: what makes 316 -> 16 work."""
    p = W.tiny()
    L = p.lattice
    ns = L ** 3
    for d in ([0, 0, 2], [1, 2, 3], [3, 3, 3], [0, 1, 2]):
        d = np.array(d)
        Cd = oracle.coupling_block(p, d)
        for Q in list(signed_permutations())[::5]:
            S = np.zeros((3 * ns, 3 * ns))
            for s in range(ns):
                ii = np.array([s % L, (s // L) % L, s // (L * L)])
                off = ii + 0.5 - L / 2.0
                jj = (Q @ off + L / 2.0 - 0.5).round().astype(int)
                s2 = jj[0] + L * jj[1] + L * L * jj[2]
                S[3 * s2:3 * s2 + 3, 3 * s:3 * s + 3] = Q
            CQ = oracle.coupling_block(p, (Q @ d).astype(int))
            assert np.allclose(CQ, S @ Cd @ S.T, rtol=0, atol=1e-10 * np.abs(Cd).max())


def test_coupling_block_reciprocity():
    p = W.tiny()
    for d in ([2, 0, 0], [1, -2, 3]):
        C = oracle.coupling_block(p, d)
        Cm = oracle.coupling_block(p, -np.array(d))
        assert np.allclose(Cm, C.T, rtol=0, atol=1e-10 * np.abs(C).max())
    C0 = oracle.coupling_block(p, [0, 0, 0])
    for s in range(p.lattice ** 3):
        assert np.all(C0[3 * s:3 * s + 3, 3 * s:3 * s + 3] == 0)


# ------------------------------------------------------------------ lattice convention
def test_sites_form_one_uniform_lattice():
    p = W.tiny()
    pos = oracle.site_positions(p).reshape(-1, 3)
    h = p.a / p.lattice
    idx = pos / h - 0.5
    assert np.allclose(idx, np.round(idx), atol=1e-12)
    ii = np.round(idx).astype(int)
    assert len({tuple(r) for r in ii}) == len(ii)              # no two dipoles coincide
    span = ii.max(0) - ii.min(0) + 1
    assert np.all(span == p.G * p.lattice) and len(ii) == np.prod(span)   # fills the grid
    assert np.allclose(pos.mean(0), 0.0, atol=1e-12)           # origin at the grid centre
    per_box = oracle.site_positions(p)
    centres = per_box.mean(1)
    assert np.allclose(per_box - centres[:, None, :], per_box[0] - centres[0], atol=1e-12)


# ------------------------------------------------------------------ operator
def test_single_dipole_far_field_is_closed_form():
    p = W.tiny()
    pos = oracle.site_positions(p)
    nbox, ns, _ = pos.shape
    X = np.zeros((1, nbox, 3 * ns), complex)
    src_box, src_site, beta = 21, 37, 2
    X[0, src_box, 3 * src_site + beta] = 1.0
    Y = oracle.dipole_field(p, X, oracle.FAR)
    ijk = p.box_ijk
    for t in range(nbox):
        far = np.abs(ijk[t] - ijk[src_box]).max() >= 2
        for s in range(0, ns, 7):
            got = Y[0, t, 3 * s:3 * s + 3]
            if not far:
                assert np.all(got == 0)
                continue
            ref = hertz_field(K, ETA, pos[t, s] - pos[src_box, src_site], np.eye(3)[beta])
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def _explicit_operator(q, which):
    """Dense Z assembled from scratch with pure-Python loops over site pairs."""
    L, G, a = q.lattice, q.G, q.a
    ns = L ** 3
    nbox = len(q.box_ijk)
    sites = []
    for b in range(nbox):
        for iz in range(L):
            for iy in range(L):
                for ix in range(L):
                    off = np.array([ix, iy, iz])
                    sites.append((b, a * (q.box_ijk[b] + 0.5 - G / 2) + a * ((off + 0.5) / L - 0.5)))
    sites.sort(key=lambda t: t[0])   # box-major, site order ix fastest
    m = 3 * ns * nbox
    D = np.zeros((m, m), complex)
    for i, (bi, ri) in enumerate(sites):
        for j, (bj, rj) in enumerate(sites):
            if i == j:
                continue
            ch = np.abs(q.box_ijk[bi] - q.box_ijk[bj]).max()
            if (which == "far" and ch < 2) or (which == "near" and ch > 1):
                continue
            for beta in range(3):
                D[3 * i:3 * i + 3, 3 * j + beta] = hertz_field(q.k, q.eta, ri - rj, np.eye(3)[beta])
    Pbig = np.zeros((int(q.nb.sum()), m), complex)
    o = 0
    for b in range(nbox):
        Pbig[o:o + q.nb[b], 3 * ns * b:3 * ns * (b + 1)] = q.P[o:o + q.nb[b]]
        o += q.nb[b]
    Z = Pbig @ D @ Pbig.T
    if which != "far":
        Z = Z + q.alpha * np.eye(Z.shape[0])
    return Z


@pytest.mark.parametrize("which", ["far", "near", "full"])
def test_operator_matches_explicit_assembly(which):
    boxes = [(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0), (0, 2, 0), (3, 1, 1)]
    q = Tiny(boxes, G=4, L=2, nb=5, seed=102, alpha=123.0)
    c = W.complex_normal(W.rng(103), (2, int(q.nb.sum())))
    Z = _explicit_operator(q, which)
    ref = c @ Z.T
    got = oracle.operator(q, c, which)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    got_g = oracle.operator_grouped(q, c, which)
    assert np.linalg.norm(got_g - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("which", ["far", "near", "full"])
def test_grouped_equals_brute_force_on_tiny(which):
    p = W.tiny()
    p.alpha = 1.0e7
    c = W.coefficients(p, 2, 12)
    a = oracle.operator(p, c, which)
    b = oracle.operator_grouped(p, c, which)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)


def test_reciprocity_bilinear():
    p = W.tiny()
    p.alpha = 3.0e7
    c = W.coefficients(p, 2, 104)
    Zc = oracle.operator(p, c, "full")
    lhs = c[0] @ Zc[1]
    rhs = c[1] @ Zc[0]
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_translation_invariance():
    p = W.tiny()
    p.alpha = 0.0
    c = W.coefficients(p, 1, 105)
    y0 = oracle.far_matvec(p, c)
    q = W.tiny()
    q.box_ijk = (p.box_ijk + np.array([1, 2, 3], dtype=np.int32)).astype(np.int32)
    q.G = 10
    y1 = oracle.far_matvec(q, c)
    assert np.linalg.norm(y1 - y0) <= 1e-13 * np.linalg.norm(y0)


def test_box_order_does_not_matter():
    p = W.tiny()
    c = W.coefficients(p, 1, 106)
    y0 = oracle.far_matvec(p, c)
    perm = W.rng(107).permutation(p.n_boxes)
    q = W.tiny()
    o = p.offsets
    q.box_ijk = p.box_ijk[perm].copy()
    q.nb = p.nb[perm].copy()
    q.P = np.concatenate([p.P[o[b]:o[b + 1]] for b in perm])
    cq = np.concatenate([c[:, o[b]:o[b + 1]] for b in perm], axis=1)
    y1 = oracle.far_matvec(q, cq)
    y0p = np.concatenate([y0[:, o[b]:o[b + 1]] for b in perm], axis=1)
    assert np.linalg.norm(y1 - y0p) <= 1e-13 * np.linalg.norm(y0)


def test_linearity():
    p = W.tiny()
    p.alpha = 2.0e7
    c = W.coefficients(p, 2, 108)
    a, b = 0.7 - 1.3j, -2.1 + 0.4j
    lhs = oracle.operator(p, a * c[:1] + b * c[1:], "full")
    Zc = oracle.operator(p, c, "full")
    rhs = a * Zc[:1] + b * Zc[1:]
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_target_subset_equals_rows_of_full_result():
    p = W.tiny()
    c = W.coefficients(p, 1, 109)
    full = oracle.far_matvec(p, c)
    t = np.array([3, 17, 40, 63])
    sub = oracle.far_matvec(p, c, targets=t)
    assert np.array_equal(sub, full[:, oracle.basis_rows(p, t)])


# ------------------------------------------------------------------ solve
def test_gmres_on_random_system_matches_dense_solve():
    g = W.rng(110)
    n = 120
    A = 4.0 * np.eye(n) + W.complex_normal(g, (n, n)) / math.sqrt(n)
    b = W.complex_normal(g, (n,))
    x, it, hist = oracle.gmres(lambda v: A @ v, b, restart=20, tol=1e-12, maxiter=500)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(b - A @ x) <= 1.01e-12 * np.linalg.norm(b)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-9) for i in range(len(hist) - 1))


def test_dense_lu_equals_gmres_on_tiny():
    p = W.tiny()
    p.alpha = W.alpha_for("tiny")
    Z = oracle.dense_operator(p)
    c = W.coefficients(p, 1, 111)
    assert np.linalg.norm(Z @ c[0] - oracle.operator(p, c, "full")[0]) <= 1e-13 * np.linalg.norm(Z @ c[0])
    kh, pol = W.plane_wave_spec(1)
    v = oracle.plane_wave_rhs(p, kh, pol)[0]
    ref = np.linalg.solve(Z, v)
    x, it, hist = oracle.gmres(lambda u: Z @ u, v, restart=50, tol=1e-11, maxiter=400)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # contraction bound of alpha I + K with ||K|| = sigma < alpha (sigma from power iteration)
    rho = W.alpha_table_entry("tiny")["sigma"] / p.alpha
    for kk, h in enumerate(hist[:60]):
        assert h <= 1.02 * (rho * 1.01) ** kk


def test_power_iteration_norm():
    g = W.rng(112)
    n = 60
    A = W.complex_normal(g, (n, n))
    Ks = A + A.T                                  # complex symmetric, like P D_off P^T

    class Q:
        nb = np.array([n])
    sigma, hist = oracle.operator_norm(Q, iters=300, matvec=lambda v: Ks @ v)
    assert abs(sigma - np.linalg.norm(Ks, 2)) <= 1e-6 * np.linalg.norm(Ks, 2)


# ------------------------------------------------------------------ excitation (§5)
def test_plane_wave_properties():
    p = W.tiny()
    p.P = None
    p.nb = np.full(p.n_boxes, 192, dtype=np.int32)
    kh, pol = W.plane_wave_spec(1)
    e = oracle.plane_wave_fields(p, kh, pol)[0].reshape(p.n_boxes, 64, 3)
    assert np.allclose(np.abs(e[..., 0]), 1.0) and np.all(e[..., 1:] == 0)
    pos = oracle.site_positions(p)
    h = p.a / p.lattice
    # travelling along +z under exp(+j w t): phase decreases by k h per lattice step in z
    s0, s1 = 5, 5 + 16
    ratio = e[0, s1, 0] / e[0, s0, 0]
    assert np.isclose(pos[0, s1, 2] - pos[0, s0, 2], h)
    assert np.isclose(ratio, np.exp(-1j * K * h), rtol=0, atol=1e-13)
    kh2, pol2 = W.plane_wave_spec(3, seed=5)
    e2 = oracle.plane_wave_fields(p, kh2, pol2).reshape(3, -1, 3)
    for r in range(3):
        assert np.allclose(e2[r] @ kh2[r], 0.0, atol=1e-13)           # transverse
        assert np.allclose(np.linalg.norm(e2[r], axis=1), 1.0)        # unit amplitude
    pt = W.tiny()
    v = oracle.plane_wave_rhs(pt, kh, pol)
    ebig = oracle.plane_wave_fields(pt, kh, pol).reshape(1, -1)
    Pbig = np.zeros((pt.n, ebig.shape[1]), complex)
    o = pt.offsets
    for b in range(pt.n_boxes):
        Pbig[o[b]:o[b + 1], 192 * b:192 * (b + 1)] = pt.P[o[b]:o[b + 1]]
    assert np.allclose(v[0], Pbig @ ebig[0], rtol=1e-13, atol=0)


# ------------------------------------------------------------------ mapping (§2.1, eq. 9-11, 15-17)
EDGES = [W.BOX_EDGE, W.LFB_EDGES["lfb256"]]


def test_fibonacci_sphere_closed_form():
    """Equal-area bands: z_l = R (1 - (2l+1)/n) exactly; azimuth steps of 2 pi / golden ratio;
    every point on the sphere; nearest neighbours near the mean spacing sqrt(4 pi / n) R."""
    for n, R in ((128, 0.375), (64, 1.0), (256, 2.0)):
        S = oracle.fibonacci_sphere(n, R)
        assert np.allclose(np.linalg.norm(S, axis=1), R, rtol=1e-14, atol=0)
        assert np.allclose(S[:, 2], R * (1 - (2 * np.arange(n) + 1) / n), rtol=0, atol=1e-14 * R)
        az = np.arctan2(S[:, 1], S[:, 0])
        step = np.mod(np.diff(az), 2 * math.pi)
        assert np.allclose(step, np.mod(2 * math.pi * (2 / (1 + math.sqrt(5))), 2 * math.pi), atol=1e-12)
        d = np.linalg.norm(S[:, None] - S[None], axis=2) + np.eye(n) * 10 * R
        nn = d.min(1) / (math.sqrt(4 * math.pi / n) * R)
        assert nn.min() > 0.8 and nn.max() < 1.05
        assert np.linalg.norm(S.mean(0)) < 2e-3 * R


@pytest.mark.parametrize("a", EDGES)
def test_mapping_reproduces_a_uniform_dipole(a):
    """A basis function that is itself uniform dipole j, direction beta, has B = A e_{3j+beta};
    A has full column rank (3 N_s = 384 >= 192), so eq. 11 returns e_{3j+beta}."""
    sites = oracle.lattice_offsets(a, 4)
    cases = [(0, 0), (17, 1), (42, 2), (63, 0)]
    off = np.arange(len(cases) + 1, dtype=np.int64)
    pos = np.array([sites[j] for j, _ in cases])
    mom = np.array([np.eye(3)[b] for _, b in cases], dtype=np.complex128)
    P, res = oracle.map_basis(K, ETA, a, 4, 128, 1.5, off, pos, mom)
    for f, (j, b) in enumerate(cases):
        e = np.zeros(192)
        e[3 * j + b] = 1
        assert np.abs(P[f] - e).max() < 1e-8
        assert res[f] < 1e-10


def test_mapping_superposition_over_the_dipoles_of_a_function():
    """A function made of three dipoles maps to the sum of the rows of its dipoles alone."""
    a = W.BOX_EDGE
    singles, pos, mom = W.point_dipole_basis([3], 910, a=a, max_dipoles=1)   # three one-dipole functions
    assert list(singles) == [0, 1, 2, 3]
    whole, _ = oracle.map_basis(K, ETA, a, 4, 128, 1.5, np.array([0, 3], dtype=np.int64), pos, mom)
    parts, _ = oracle.map_basis(K, ETA, a, 4, 128, 1.5, singles, pos, mom)
    assert np.linalg.norm(whole[0] - parts.sum(0)) <= 1e-10 * np.linalg.norm(whole[0])


@pytest.mark.parametrize("a", EDGES)
def test_equivalent_dipoles_reproduce_the_far_field(a):
    """The uniqueness argument of §2.1: fields matched on S (radius 1.5a) match outside it.
    The 192 uniform dipoles with eq. 11's coefficients radiate, at points 2a..6a from the box
    centre, the field of the basis function itself to within ~1e-3 (Table 1's error level);
    the field mismatch on S (eq. 10's residual) stays below 1e-2."""
    fun_off, pos, mom = W.point_dipole_basis(np.full(4, 6), 900, a=a)
    P, res = oracle.map_basis(K, ETA, a, 4, 128, 1.5, fun_off, pos, mom)
    assert res.max() < 1e-2
    sites = oracle.lattice_offsets(a, 4)
    g = W.rng(905)
    for f in range(len(fun_off) - 1):
        src = slice(fun_off[f], fun_off[f + 1])
        for _ in range(6):
            u = g.standard_normal(3)
            R = u / np.linalg.norm(u) * a * g.uniform(2.0, 6.0)
            exact = sum(oracle.dyad(K, ETA, R - x) @ m for x, m in zip(pos[src], mom[src]))
            equiv = sum(oracle.dyad(K, ETA, R - sites[j]) @ P[f, 3 * j:3 * j + 3] for j in range(64))
            assert np.linalg.norm(equiv - exact) <= 5e-3 * np.linalg.norm(exact)


@pytest.mark.parametrize("a", EDGES)
def test_inverse_mapping_is_the_transposed_forward_map(a):
    """Eq. 15-17 computed literally (virtual dipoles on S fitted to the fields at the uniform
    sites, then tested on the function) equal P_f . E: D(R) = D(-R) = D(R)^T makes the tested
    virtual-dipole fields B_f^T and (A^T)^+ = (A^+)^T.  For fields E of a source 3a away the
    result is the function's exact response to that source within ~1e-4."""
    fun_off, pos, mom = W.point_dipole_basis(np.full(1, 3), 920, a=a)
    P, _ = oracle.map_basis(K, ETA, a, 4, 128, 1.5, fun_off, pos, mom)
    sites = oracle.lattice_offsets(a, 4)
    src, pm = np.array([3.0 * a, 0.4 * a, -0.2 * a]), np.array([1.0, 0.5j, -0.3])
    E = np.concatenate([oracle.dyad(K, ETA, s - src) @ pm for s in sites])
    for f in range(len(fun_off) - 1):
        sl = slice(fun_off[f], fun_off[f + 1])
        V = oracle.inverse_map_fields(K, ETA, a, 4, 128, 1.5, E, pos[sl], mom[sl])
        assert abs(V - P[f] @ E) <= 1e-9 * abs(V)
        exact = sum(m @ (oracle.dyad(K, ETA, x - src) @ pm) for x, m in zip(pos[sl], mom[sl]))
        assert abs(V - exact) <= 1e-3 * abs(exact)


def test_tikhonov_mapping_keeps_the_far_field_and_tames_the_coefficients():
    """Eq. 11's plain pseudo-inverse gives oscillating coefficients (A's condition number is
    about 1e7).  A Tikhonov weight of 1e-5 ||A||_F leaves the error of the mapped far product
    against the point dipoles' own far interactions and the misfit on S nearly unchanged,
    while the coefficient norms fall by more than 10x."""
    import dataclasses
    p = W.tiny(nb=4)
    fun_off, pos, mom = W.point_dipole_basis(p.nb, 945, a=p.a)
    c = W.coefficients(p, 1, 946)
    direct = oracle.point_dipole_far(p, fun_off, pos, mom, c[0])
    out = {}
    for t in (0.0, 1e-5):
        P, res = oracle.map_basis(K, ETA, p.a, 4, 128, 1.5, fun_off, pos, mom, tikhonov=t)
        y = oracle.far_matvec(dataclasses.replace(p, P=P), c)[0]
        out[t] = (np.linalg.norm(y - direct) / np.linalg.norm(direct), np.median(np.linalg.norm(P, axis=1)),
                  res.max())
    (e0, n0, r0), (e1, n1, r1) = out[0.0], out[1e-5]
    assert e0 < 1e-3 and e1 < 1.2 * e0
    assert n1 < n0 / 10
    assert r1 < 1.3 * r0


# ------------------------------------------------------------------ translation networks (§3)
def test_cvfcnn_forward_by_hand():
    """The network of §3 written out entry by entry on a tiny case (3 inputs, 2 hidden)."""
    W1 = np.array([[1.0 - 2.0j, 0.5j, -1.0], [0.25, -1.5 + 1.0j, 2.0j]])
    b1 = np.array([0.5 - 0.25j, -0.75 + 1.0j])
    W2 = np.array([[1.0, -1.0j], [0.5 + 0.5j, 2.0], [-1.0, 0.25j]])
    b2 = np.array([0.1, -0.2j, 0.3 + 0.3j])
    for x in ([2.0 - 1.0j, -0.5j, 1.0], [0.0, 0.0, -3.0 + 4.0j], [0.0, 0.0, 0.0]):
        x = np.array(x)
        s = max(abs(v) for v in x)
        want = np.zeros(3, dtype=complex)
        if s > 0:
            h = []
            for i in range(2):
                z = sum(W1[i, j] * x[j] / s for j in range(3)) + b1[i]
                h.append(complex(max(z.real, 0.0), max(z.imag, 0.0)))
            for k in range(3):
                want[k] = s * (sum(W2[k, i] * h[i] for i in range(2)) + b2[k])
        got = oracle.cvfcnn_forward(W1, b1, W2, b2, x)
        assert np.allclose(got, want, rtol=1e-14, atol=1e-14)
    # the ReLU acts on the real and imaginary parts separately
    z = oracle.cvfcnn_forward(np.array([[1.0]]), np.array([-2.0 + 0.5j]), np.array([[1.0]]), np.array([0.0]),
                              np.array([1.0]))
    assert z[0] == 0.5j


@pytest.mark.parametrize("d", [[2, 0, 0], [1, 2, 3], [3, 3, 3]])
def test_cvfcnn_fit_is_the_truncated_svd_on_the_unit_ball(d):
    """Fitted weights keep every pre-activation in the ReLU's linear region, so the network
    is U_H S_H V_H^H x on the unit l-inf ball and, being positively homogeneous through its
    input scaling, everywhere; its error on inputs uniform in the unit box is then set by
    the SVD tail (the Frobenius tail is its RMS for isotropic inputs)."""
    p = W.tiny()
    C = oracle.coupling_block(p, np.array(d, dtype=np.int32))
    net = oracle.cvfcnn_fit(C, 50)
    U, S, Vh = np.linalg.svd(C)
    T = (U[:, :50] * S[:50]) @ Vh[:50]
    g = W.rng(960)
    x = g.uniform(-1, 1, (300, 192)) + 1j * g.uniform(-1, 1, (300, 192))
    for scale in (1.0, 1e3, 1e-4):
        o = oracle.cvfcnn_forward(*net, scale * x)
        assert np.abs(o - scale * x @ T.T).max() <= 1e-12 * np.abs(scale * x @ T.T).max()
    o = oracle.cvfcnn_forward(*net, x)
    ref = x @ C.T
    rms = np.sqrt(np.mean(np.linalg.norm(o - ref, axis=1) ** 2) / np.mean(np.linalg.norm(ref, axis=1) ** 2))
    tail = np.sqrt((S[50:] ** 2).sum() / (S ** 2).sum())
    assert 0.5 * tail <= rms <= 2.0 * tail


def test_cvfcnn_networks_beat_the_trained_ones_of_table1():
    """The closed-form networks (H = 50) against Table 1's trained networks: below the 1e-3
    stopping criterion of eq. 171 and below each listed mean error, for the same translation
    distances and box edges (inputs uniform in the unit box, the first-stage distribution)."""
    gold = json.load(open(os.path.join(GOLDEN, "table1_networks.json")))
    g = W.rng(961)
    for row in gold["rows"]:
        p = W.lfb(W.tiny(), "lfb8") if row["a_over_lambda"] == 0.125 else W.lfb(W.tiny(), "lfb256")
        assert p.a == row["a_over_lambda"]
        C = oracle.coupling_block(p, np.array(row["d"], dtype=np.int32))
        net = oracle.cvfcnn_fit(C, gold["hidden"])
        x = g.uniform(-1, 1, (200, 192)) + 1j * g.uniform(-1, 1, (200, 192))
        ref = x @ C.T
        eu = np.linalg.norm(oracle.cvfcnn_forward(*net, x) - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert eu.mean() < min(gold["gate"], row["mean"]), row


def test_canonical_frames_map_translation_matrices():
    """canonical_frame and signed_permutation: G_d = S_Q G_c S_Q^T for d = Q c, c = sorted |d|."""
    p = W.tiny()
    for d in ([0, -2, 0], [3, -1, 2], [-2, -2, 1], [0, 3, -3]):
        c, Q = oracle.canonical_frame(d)
        assert np.array_equal(Q @ c, d) and np.all(np.diff(c) >= 0)
        S = oracle.signed_permutation(Q, 4)
        Gd = oracle.coupling_block(p, np.array(d, dtype=np.int32))
        Gc = oracle.coupling_block(p, c.astype(np.int32))
        assert np.allclose(Gd, S @ Gc @ S.T, rtol=0, atol=1e-10 * np.abs(Gd).max())


def test_cvfcnn_far_matvec_pair_by_pair():
    """Alg. 2 with networks: every ordered far box pair adds net_d(x_b) to target t, by loops."""
    boxes = [[0, 0, 0], [2, 0, 0], [0, 3, 1], [3, 3, 3]]
    p = Tiny(boxes, G=4, L=4, nb=5, seed=962)
    ds, groups = oracle.pair_groups(p, oracle.FAR)
    g = W.rng(963)
    H = 3
    weights = {tuple(int(v) for v in d): (W.complex_normal(g, (H, 192)) / 14, W.complex_normal(g, H) * 0.1,
                                          W.complex_normal(g, (192, H)) / 2, W.complex_normal(g, 192) * 0.1)
               for d in ds}
    c = W.complex_normal(g, (1, int(p.nb.sum())))
    X = oracle.aggregate(p, c)[0]
    Y = np.zeros_like(X)
    ijk = np.array(boxes)
    for b in range(len(boxes)):
        for t in range(len(boxes)):
            d = ijk[t] - ijk[b]
            if np.abs(d).max() >= 2:
                Y[t] += oracle.cvfcnn_forward(*weights[tuple(int(v) for v in d)], X[b])
    want = oracle.disaggregate(p, Y[None])
    got = oracle.cvfcnn_far_matvec(p, c, weights=weights)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


def test_cvfcnn_canonical_frames_reproduce_the_exact_far_product():
    """Weights keyed by canonical c and applied in the frame of c (frames=True): with
    full-rank linear networks (H = 192, net_c = G_c on the unit ball) the product is the
    brute-force far product, which a transposed or mis-signed frame map would break."""
    boxes = [[0, 0, 0], [2, 0, 0], [0, 3, 1], [3, 1, 3], [0, -2, -3]]
    p = Tiny(boxes, G=4, L=4, nb=5, seed=964)
    ds, _ = oracle.pair_groups(p, oracle.FAR)
    canon = {tuple(sorted(int(v) for v in np.abs(d))) for d in ds}
    assert len(canon) < len(ds)                    # frames are exercised
    weights = {cc: oracle.cvfcnn_fit(oracle.coupling_block(p, np.array(cc, dtype=np.int32)), 192) for cc in canon}
    c = W.complex_normal(W.rng(965), (2, int(p.nb.sum())))
    got = oracle.cvfcnn_far_matvec(p, c, weights=weights, frames=True)
    want = oracle.far_matvec(p, c)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
