"""Low-frequency regime: box edge lambda/8 and lambda/256 (§3, §5).

At lambda/256 every interaction is quasi-static.  The reactive (imaginary) part of the
dyad exceeds its radiative (real) part by about 3/(kR)^3, 6e4 at the closest far site
pair, and eq. 5-6 reach the radiative part through a cancellation of 1/(kR) terms.  The
library generates the coupling blocks in FP64 and stores each entry as a float (FP32, or
a 16-bit hi/lo pair under one power-of-two scale per block), so every entry keeps its own
relative precision and the products keep their accuracy, the radiative part included.

Checks against the FP64 oracle: the stored FP32 blocks entry by entry, the far product
of every precision, the radiative part of the far product on its own (a real input on
identity P makes Re y = Re(G) x), the near and full products, dense-LU solves on the
4^3 grid and a sampled solve on the 16^3 shell.
"""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, plan_for, rel_l2

pytestmark = pytest.mark.gpu
BOUND = {ie.IE_PREC_FP32: 1e-6, ie.IE_PREC_BF16X3: 5e-5, ie.IE_PREC_FP16X3: 2e-6, ie.IE_PREC_BF16X1: 1e-2,
         ie.IE_PREC_FP16X1: 2e-3}
ALL = list(BOUND)
TAGS = list(W.LFB_EDGES)


def _name(p):
    return ie.PREC_NAMES[p]


@pytest.fixture(scope="module", params=TAGS)
def tiny(request):
    p = W.lfb(W.tiny(), request.param)
    p.alpha = W.alpha_for(p.name)
    return p


def _fp64_term_scales(p, d):
    """Per entry of C_d, the magnitude of the terms that eq. 5-6 add up for the real and the
    imaginary part: psi = s (-sin x - j cos x) with s = k eta / (4 pi R), x = kR, times
    t = a I - b Rhat Rhat with |Re t| <= |1 - 1/x^2| + |1 - 3/x^2| and |Im t| <= 4/x.  At small
    x these terms (~s/x) cancel to the radiative part (~s x), so an FP64 evaluation carries
    an absolute error of a few eps64 times them: far below an FP32 rounding of the static
    (imaginary) part, but above one of the tiny off-diagonal radiative entries."""
    sites = oracle.lattice_offsets(p.a, 4)
    R = p.a * np.asarray(d, dtype=np.float64)[None, None, :] + sites[:, None, :] - sites[None, :, :]
    r = np.linalg.norm(R, axis=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = p.k * r
        sc = p.k * p.eta / (4 * np.pi * r)
        tre = np.abs(1 - 1 / x ** 2) + np.abs(1 - 3 / x ** 2)
        tim = 4 / x
        s_re = sc * (np.abs(np.sin(x)) * tre + np.abs(np.cos(x)) * tim)
        s_im = sc * (np.abs(np.sin(x)) * tim + np.abs(np.cos(x)) * tre)
    s_re[r == 0] = 0.0
    s_im[r == 0] = 0.0
    expand = lambda m: np.repeat(np.repeat(m, 3, axis=0), 3, axis=1)  # noqa: E731
    return expand(s_re), expand(s_im)


def test_coupling_blocks_within_one_fp32_rounding(tiny):
    """Stored FP32 blocks against the oracle's FP64 ones: one FP32 rounding apart, plus the
    FP64 evaluation error of each side (32 eps64 times the cancelling terms).  A block
    generated in FP32 arithmetic would miss this by a factor of about 1e7."""
    ds = np.array([[2, 0, 0], [3, 3, 3], [-2, 1, 0], [0, -3, 1], [1, -1, 0], [0, 0, 0]], dtype=np.int32)
    with plan_for(tiny) as plan:
        out = empty((len(ds), 192, 192))
        ie.ie_coupling_blocks(plan.handle, ds, out)
        got = host(out)
    eps64 = np.finfo(np.float64).eps
    for i, d in enumerate(ds):
        ref = oracle.coupling_block(tiny, d)
        s_re, s_im = _fp64_term_scales(tiny, d)
        for part, sc in ((np.real, s_re), (np.imag, s_im)):
            ulp = np.spacing(np.abs(part(ref)).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(part(got[i]) - part(ref)) <= ulp + 32 * eps64 * sc + 1e-30), (d, part.__name__)


@pytest.mark.parametrize("prec", ALL, ids=_name)
def test_far_product_every_precision(prec, tiny):
    c = W.coefficients(tiny, 2, 801)
    ref = oracle.far_matvec(tiny, c)
    with plan_for(tiny, ALL, max_rhs=2) as plan:
        y = empty((2, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 2)
        assert rel_l2(host(y), ref) <= BOUND[prec]


@pytest.mark.parametrize("tag", TAGS)
def test_radiative_part_of_the_far_product(tag):
    """Real dipole moments on identity P: Re y = Re(G) x is the radiative part alone."""
    p = W.lfb(W.tiny_identity(), tag)
    c = W.rng(802).standard_normal((1, p.n)).astype(np.complex128)
    ref = oracle.far_matvec(p, c)
    if tag == "lfb256":
        assert np.linalg.norm(ref.real) <= 1e-3 * np.linalg.norm(ref.imag)
    with plan_for(p, ALL) as plan:
        for prec in ALL:
            y = empty((1, p.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            got = host(y)
            assert rel_l2(got.real, ref.real) <= BOUND[prec], _name(prec)
            assert rel_l2(got.imag, ref.imag) <= BOUND[prec], _name(prec)


@pytest.mark.parametrize("which", ["near", "full"])
def test_near_and_full_products(which, tiny):
    c = W.coefficients(tiny, 1, 803)
    ref = oracle.operator(tiny, c, which)
    kind = {"near": ie.IE_NEAR, "full": ie.IE_FULL}[which]
    with plan_for(tiny, [ie.IE_PREC_FP32, ie.IE_PREC_FP16X3]) as plan:
        for prec in (ie.IE_PREC_FP32, ie.IE_PREC_FP16X3):
            y = empty((1, tiny.n))
            ie.ie_matvec(plan.handle, kind, prec, dev(c), y, 1)
            assert rel_l2(host(y), ref) <= BOUND[prec], _name(prec)


@pytest.mark.parametrize("prec,tol", [(ie.IE_PREC_FP32, 1e-6), (ie.IE_PREC_FP16X3, 1e-5)], ids=["fp32", "fp16x3"])
def test_solve_matches_dense_lu(prec, tol, tiny):
    Z = oracle.dense_operator(tiny)
    kh, pol = W.plane_wave_spec(1)
    v = oracle.plane_wave_rhs(tiny, kh, pol)
    ref = np.linalg.solve(Z, v[0])
    with plan_for(tiny, [ie.IE_PREC_FP32, prec]) as plan:
        x = empty((1, tiny.n))
        st, info = ie.ie_solve(plan.handle, dev(v), x, 1, ie.solve_opts(tol=tol, prec=prec))
        assert st == ie.IE_OK and info["converged"] == 1, info
        xs = host(x)[0]
    true_res = np.linalg.norm(v[0] - Z @ xs) / np.linalg.norm(v[0])
    assert true_res <= 2 * tol
    # forward error <= ||r|| / (alpha - sigma) and ||v|| <= (alpha + sigma) ||x||: a factor 9 at alpha = 1.25 sigma
    assert rel_l2(xs, ref) <= 9 * 2 * tol
    assert info["iterations"] <= 62


def test_shell16_lfb256_sampled_products_and_solve():
    p = W.lfb(W.shell16(), "lfb256")
    p.alpha = W.alpha_for(p.name)
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    rows = oracle.basis_rows(p, targets)
    ref = oracle.far_matvec(p, c, targets=targets)
    kh, pol = W.plane_wave_spec(1)
    precs = [ie.IE_PREC_FP32, ie.IE_PREC_BF16X3, ie.IE_PREC_FP16X3]
    with plan_for(p, precs) as plan:
        for prec in precs:
            y = empty((1, p.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, prec, dev(c), y, 1)
            assert rel_l2(host(y)[:, rows], ref) <= BOUND[prec], _name(prec)
        v = empty((1, p.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        x = empty((1, p.n))
        st, info = ie.ie_solve(plan.handle, v, x, 1, ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_FP16X3))
        assert st == ie.IE_OK, info
        xs = host(x)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    Zx = oracle.operator(p, xs, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 1e-5, res
