"""Mapping construction (§2.1, eq. 9-11) on the GPU against the FP64 oracle.

ie_map_basis builds the rows of P for point-dipole basis functions: their fields on the
Fibonacci sphere S, the least-squares fit by the 192 uniform dipoles, and the fit's
mismatch on S.  Each side computes its own rows from the same seeded functions.

Tolerance of the rows: both are least-squares solutions of a system whose matrix A has a
condition number of about 1e7; each side's error is about kappa * eps64 ~ 1e-9 relative
(Householder QR here, LAPACK's SVD-based solver in the oracle), so rows agree within 1e-7
relative, row by row.  The residual on S is first-order insensitive to such errors: 1e-6.
Downstream, a problem whose P the GPU built (Tikhonov weight 1e-5) runs the far product and
the solve against the oracle on the oracle's own P, and the far product approximates the
direct interactions of the point dipoles themselves within the method's error (Table 1's
level).  Rounding in the products grows with ||G| |X|| / ||G X||: 184 here against 63 for
the random-P workloads (computed with the oracle), so their bounds are scaled by 3.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, plan_for, rel_l2

pytestmark = pytest.mark.gpu
ROW_TOL = 1e-7


def _both(fun_off, pos, mom, a, n_samples=128, radius=1.5, tikhonov=0.0):
    P, res = ie.ie_map_basis(W.K0, W.ETA0, a, fun_off, pos, mom, n_samples=n_samples, sample_radius=radius,
                             tikhonov=tikhonov)
    Pr, rr = oracle.map_basis(W.K0, W.ETA0, a, 4, n_samples, radius, fun_off, pos, mom, tikhonov=tikhonov)
    return P, res, Pr, rr


def _row_err(P, Pr):
    nr = np.linalg.norm(Pr, axis=1)
    return np.linalg.norm(P - Pr, axis=1) / np.where(nr > 0, nr, 1.0)


@pytest.mark.parametrize("a,tikhonov", [(W.BOX_EDGE, 0.0), (W.BOX_EDGE, 1e-5), (W.LFB_EDGES["lfb8"], 0.0),
                                         (W.LFB_EDGES["lfb256"], 0.0), (W.LFB_EDGES["lfb256"], 1e-5)])
def test_rows_and_residuals_match_oracle(a, tikhonov):
    # 61 functions (a ragged last CTA of 8), one of them without dipoles
    fun_off, pos, mom = W.point_dipole_basis(np.full(12, 5), 930, a=a)
    fun_off = np.insert(fun_off, 7, fun_off[7])
    P, res, Pr, rr = _both(fun_off, pos, mom, a, tikhonov=tikhonov)
    assert P.shape == Pr.shape == (61, 192)
    assert _row_err(P, Pr).max() <= ROW_TOL
    assert np.all(P[7] == 0) and res[7] == 0
    assert np.allclose(res, rr, rtol=1e-6, atol=1e-12)
    assert rr.max() < 1e-2


@pytest.mark.parametrize("n_samples,radius", [(64, 1.0), (256, 2.0)])
def test_sampling_limits(n_samples, radius):
    """N_s = 64 makes A square: the fit interpolates and both residuals are rounding noise
    (about kappa * eps64); N_s = 256 is the largest sample count."""
    a = W.BOX_EDGE
    fun_off, pos, mom = W.point_dipole_basis(np.full(3, 4), 931, a=a)
    P, res, Pr, rr = _both(fun_off, pos, mom, a, n_samples, radius)
    assert _row_err(P, Pr).max() <= ROW_TOL
    if n_samples == 64:
        assert res.max() < 1e-9 and rr.max() < 1e-9
    else:
        assert np.allclose(res, rr, rtol=1e-6, atol=1e-12)


def test_uniform_dipoles_map_to_unit_rows():
    a = W.BOX_EDGE
    sites = oracle.lattice_offsets(a, 4)
    cases = [(j, b) for j in (0, 5, 21, 42, 63) for b in range(3)]
    fun_off = np.arange(len(cases) + 1, dtype=np.int64)
    pos = np.array([sites[j] for j, _ in cases])
    mom = np.array([np.eye(3)[b] for _, b in cases], dtype=np.complex128)
    P, res = ie.ie_map_basis(W.K0, W.ETA0, a, fun_off, pos, mom)
    for f, (j, b) in enumerate(cases):
        e = np.zeros(192)
        e[3 * j + b] = 1.0
        assert np.abs(P[f] - e).max() < 1e-8
        assert res[f] < 1e-10


def test_many_functions_cross_the_device_chunks():
    """70,000 functions (more than one 65,536-function pass): sampled rows against the oracle."""
    a = W.BOX_EDGE
    fun_off, pos, mom = W.point_dipole_basis(np.full(7000, 10), 932, a=a)
    P, res = ie.ie_map_basis(W.K0, W.ETA0, a, fun_off, pos, mom)
    pick = np.array([0, 1, 65535, 65536, 65537, 69999] + list(W.rng(933).choice(70000, 10, replace=False)))
    sub_off = np.zeros(len(pick) + 1, dtype=np.int64)
    sub_pos, sub_mom = [], []
    for i, f in enumerate(pick):
        sl = slice(fun_off[f], fun_off[f + 1])
        sub_pos.append(pos[sl])
        sub_mom.append(mom[sl])
        sub_off[i + 1] = sub_off[i] + (fun_off[f + 1] - fun_off[f])
    Pr, rr = oracle.map_basis(W.K0, W.ETA0, a, 4, 128, 1.5, sub_off, np.vstack(sub_pos), np.vstack(sub_mom))
    assert _row_err(P[pick], Pr).max() <= ROW_TOL
    assert np.allclose(res[pick], rr, rtol=1e-6, atol=1e-12)


@pytest.fixture(scope="module")
def mapped_tiny():
    """The 4^3 grid with nb = 32 point-dipole functions per box: (GPU problem, oracle problem, basis)."""
    base = W.tiny()
    t = W.MAPPED_TIKHONOV
    fun_off, pos, mom = W.point_dipole_basis(base.nb, W.SEED_MAPPED["tiny"], a=base.a)
    P, _ = ie.ie_map_basis(base.k, base.eta, base.a, fun_off, pos, mom, tikhonov=t)
    Pr, _ = oracle.map_basis(base.k, base.eta, base.a, 4, 128, 1.5, fun_off, pos, mom, tikhonov=t)
    alpha = W.alpha_for("tiny_mapped")
    pg = dataclasses.replace(base, name="tiny_mapped", P=P, alpha=alpha)
    po = dataclasses.replace(base, name="tiny_mapped", P=Pr, alpha=alpha)
    return pg, po, (fun_off, pos, mom)


def test_mapped_far_product_and_the_direct_interactions(mapped_tiny):
    pg, po, (fun_off, pos, mom) = mapped_tiny
    c = W.coefficients(po, 1, 941)
    ref = oracle.far_matvec(po, c)
    direct = oracle.point_dipole_far(po, fun_off, pos, mom, c[0])
    bounds = {ie.IE_PREC_FP32: 3e-6, ie.IE_PREC_FP16X3: 6e-6, ie.IE_PREC_BF16X3: 1.5e-4}
    with plan_for(pg, list(bounds)) as plan:
        for prec, bound in bounds.items():
            y = empty((1, pg.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            got = host(y)
            assert rel_l2(got, ref) <= bound, ie.PREC_NAMES[prec]
            # the method's own error against the original point-dipole system
            assert rel_l2(got[0], direct) <= 1e-3, ie.PREC_NAMES[prec]


def test_mapped_solve_matches_dense_lu(mapped_tiny):
    pg, po, _ = mapped_tiny
    Z = oracle.dense_operator(po)
    kh, pol = W.plane_wave_spec(1)
    v = oracle.plane_wave_rhs(po, kh, pol)
    ref = np.linalg.solve(Z, v[0])
    with plan_for(pg, [ie.IE_PREC_FP32, ie.IE_PREC_FP16X3]) as plan:
        vg = empty((1, pg.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, vg)
        assert rel_l2(host(vg), v) <= 1e-6
        x = empty((1, pg.n))
        st, info = ie.ie_solve(plan.handle, vg, x, 1, ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3))
        assert st == ie.IE_OK, info
        xs = host(x)[0]
    true_res = np.linalg.norm(v[0] - Z @ xs) / np.linalg.norm(v[0])
    assert true_res <= 2e-5
    assert rel_l2(xs, ref) <= 9 * 2e-5


def test_mapped_shell16_against_the_point_dipoles_themselves():
    """Full size: P of the 16^3 shell's 40,448 seeded point-dipole functions built on the GPU;
    the far product (FP32 and FP16X3) on an 8-box sample against the brute-force far
    interactions of the dipoles themselves (the oracle's direct sum, which needs no P):
    within the method's error (1.1e-4 with the oracle's own P, Table 1's level)."""
    base = W.shell16()
    fun_off, pos, mom = W.point_dipole_basis(base.nb, W.SEED_MAPPED["shell16"], a=base.a)
    P, res = ie.ie_map_basis(base.k, base.eta, base.a, fun_off, pos, mom, tikhonov=W.MAPPED_TIKHONOV)
    assert np.median(res) < 1e-3 and res.max() < 5e-2
    pg = dataclasses.replace(base, name="shell16_mapped", P=P, alpha=W.alpha_for("shell16_mapped"))
    c = W.coefficients(pg, 1, 990)
    targets = W.subsample_boxes(pg, 8, W.SEED_SUBSAMPLE["shell16"])
    rows = oracle.basis_rows(pg, targets)
    direct = oracle.point_dipole_far(pg, fun_off, pos, mom, c[0], targets=targets)
    with plan_for(pg, [ie.IE_PREC_FP32, ie.IE_PREC_FP16X3]) as plan:
        for prec in (ie.IE_PREC_FP32, ie.IE_PREC_FP16X3):
            y = empty((1, pg.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            assert rel_l2(host(y)[0, rows], direct) <= 1e-3, ie.PREC_NAMES[prec]
