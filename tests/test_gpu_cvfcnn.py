"""Translation networks of §3 (IE_PREC_CVFCNN) on the GPU against the FP64 oracle.

The library evaluates, per stored block, the network s (W2 relu(W1 x / s + b1) + b2)
with s = ||x||_inf in FP32, inside Alg. 2 in place of G_d x.  Fitted weights put the
network in its linear regime, equal to the truncated SVD of G_c; each side fits its own
(Jacobi SVD on the GPU, LAPACK in the oracle), and the networks' outputs are unique.

Uniqueness: where sigma_H = sigma_H+1 the truncation (hence the network) is not unique.  At
H = 50 that happens on seven of shell16's 473 classes, all with sigma_50 <= 1.1e-8 sigma_1,
so either choice moves the output by less than that; widths whose cutoff splits a large
degenerate pair (H = 1 for axis and diagonal displacements) are not compared.

Tolerances.  Network against network: FP32 sums of 192 and H terms plus the hidden bias,
which is up to sqrt(192) times the hidden signal and cancels in the output bias: about
25 x 6e-8 x sqrt(H) ~ 1e-5 relative, so 3e-5.  Network against the exact translation:
the SVD tail of the blocks (the oracle computes 8.7e-6 on the 4^3 grid), plus the above.
"""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, rel_l2

pytestmark = pytest.mark.gpu
NET_TOL = 3e-5


def _plan(p, precs, symmetry, max_rhs=1, hidden=0):
    return ie.Plan(ie.problem_from(p, ie.precmask(*precs), max_rhs, symmetry=symmetry, cvfcnn_hidden=hidden))


@pytest.fixture(scope="module")
def tiny():
    p = W.tiny()
    p.alpha = W.alpha_for("tiny")
    return p


def _svd_tail(C, H):
    S = np.linalg.svd(C, compute_uv=False)
    return np.sqrt((S[H:] ** 2).sum() / (S ** 2).sum())


def test_fit_statistics_and_block_order(tiny):
    with _plan(tiny, [ie.IE_PREC_CVFCNN], symmetry=1) as plan:
        st = plan.stats
        blocks = ie.ie_plan_blocks(plan.handle)
    ds, _ = oracle.pair_groups(tiny, oracle.FAR)
    canon = sorted({tuple(sorted(np.abs(d))) for d in ds})
    assert sorted(map(tuple, blocks)) == canon and len(blocks) == st["n_coupling_blocks"] == 16
    assert st["cvfcnn_hidden"] == 50 and 2 <= st["cvfcnn_sweeps"] <= 16
    tails = [_svd_tail(oracle.coupling_block(tiny, np.array(c, dtype=np.int32)), 50) for c in canon]
    assert np.isclose(st["cvfcnn_tail"], max(tails), rtol=1e-6, atol=1e-14)


def test_random_weights_match_the_oracle_network(tiny):
    """Weights drawn at random (the ReLU then cuts many pre-activations), one network per
    displacement (full store), loaded through ie_cvfcnn_set_weights."""
    H = 7
    c = W.coefficients(tiny, 2, 970)
    with _plan(tiny, [ie.IE_PREC_CVFCNN], symmetry=0, max_rhs=2, hidden=H) as plan:
        blocks = ie.ie_plan_blocks(plan.handle)
        g = W.rng(971)
        nb = len(blocks)
        W1 = W.complex_normal(g, (nb, H, 192)) / 14
        b1 = W.complex_normal(g, (nb, H)) * 0.3
        W2 = W.complex_normal(g, (nb, 192, H)) / 3
        b2 = W.complex_normal(g, (nb, 192)) * 0.1
        ie.ie_cvfcnn_set_weights(plan.handle, W1, b1, W2, b2)
        y = empty((2, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(c), y, 2)
        got = host(y)
    # the oracle takes the weights as the library stored them (complex64)
    r = lambda a: a.astype(np.complex64).astype(np.complex128)  # noqa: E731
    weights = {tuple(int(v) for v in d): (r(W1[i]), r(b1[i]), r(W2[i]), r(b2[i])) for i, d in enumerate(blocks)}
    ref = oracle.cvfcnn_far_matvec(tiny, c, weights=weights)
    assert rel_l2(got, ref) <= NET_TOL
    # the nonlinearity is active: a good share of hidden pre-activations is cut
    X = oracle.aggregate(tiny, c)[0]
    z = (X[:5] / np.abs(X[:5]).max(axis=1, keepdims=True)) @ W1[0].T + b1[0]
    assert 0.2 < np.mean(z.real < 0) < 0.8


@pytest.mark.parametrize("symmetry", [0, 1])
def test_fitted_far_product(symmetry, tiny):
    c = W.coefficients(tiny, 1, 972)
    ref_net = oracle.cvfcnn_far_matvec(tiny, c, H=50)
    ref = oracle.far_matvec(tiny, c)
    with _plan(tiny, [ie.IE_PREC_FP32, ie.IE_PREC_CVFCNN], symmetry=symmetry) as plan:
        y = empty((1, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(c), y, 1)
        got = host(y)
        tail = plan.stats["cvfcnn_tail"]
    assert rel_l2(got, ref_net) <= NET_TOL
    assert rel_l2(got, ref) <= 2 * rel_l2(ref_net, ref) + NET_TOL
    assert tail < 1e-4


@pytest.mark.parametrize("tag", ["lfb8", "lfb256"])
def test_fitted_far_product_at_the_papers_box_edges(tag):
    """The paper trained its networks for a = lambda/8 and lambda/256 (§3)."""
    p = W.lfb(W.tiny(), tag)
    c = W.coefficients(p, 1, 973)
    ref_net = oracle.cvfcnn_far_matvec(p, c, H=50)
    ref = oracle.far_matvec(p, c)
    with _plan(p, [ie.IE_PREC_CVFCNN], symmetry=1) as plan:
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(c), y, 1)
        got = host(y)
        tail = plan.stats["cvfcnn_tail"]
    assert rel_l2(got, ref_net) <= NET_TOL
    assert rel_l2(got, ref) <= 2 * rel_l2(ref_net, ref) + NET_TOL
    assert tail < 1e-4


def test_surrogate_solve_with_refinement(tiny):
    """GMRES on surrogate products to 1e-3, FP64 residuals of FP16X3 products outside:
    the answer meets 1e-5 against the dense LU of the exact system."""
    Z = oracle.dense_operator(tiny)
    kh, pol = W.plane_wave_spec(1)
    v = oracle.plane_wave_rhs(tiny, kh, pol)
    ref = np.linalg.solve(Z, v[0])
    with _plan(tiny, [ie.IE_PREC_FP16X3, ie.IE_PREC_CVFCNN], symmetry=1) as plan:
        x = empty((1, tiny.n))
        opts = ie.solve_opts(tol=1e-5, prec=ie.IE_PREC_CVFCNN, refine=1, refine_prec=ie.IE_PREC_FP16X3,
                             inner_tol=1e-3)
        st, info = ie.ie_solve(plan.handle, dev(v), x, 1, opts)
        assert st == ie.IE_OK, info
        xs = host(x)[0]
    true_res = np.linalg.norm(v[0] - Z @ xs) / np.linalg.norm(v[0])
    assert true_res <= 2e-5
    assert rel_l2(xs, ref) <= 9 * 2e-5


def test_shell16_sampled(tiny):
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 8, W.SEED_SUBSAMPLE["shell16"])
    rows = oracle.basis_rows(p, targets)
    ref_net = oracle.cvfcnn_far_matvec(p, c, H=50, targets=targets)
    ref = oracle.far_matvec(p, c, targets=targets)
    with _plan(p, [ie.IE_PREC_CVFCNN], symmetry=1) as plan:
        assert plan.stats["n_coupling_blocks"] == 473
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(c), y, 1)
        got = host(y)[:, rows]
    assert rel_l2(got, ref_net) <= NET_TOL
    assert rel_l2(got, ref) <= 2 * rel_l2(ref_net, ref) + NET_TOL


def test_weights_need_a_surrogate_plan(tiny):
    with _plan(tiny, [ie.IE_PREC_FP32], symmetry=0) as plan:
        z = np.zeros(2 * 192, dtype=np.float32)
        ptr = z.ctypes.data
        assert ie.lib().ie_cvfcnn_set_weights(plan.handle, ptr, ptr, ptr, ptr, None) == ie.IE_ERR_UNSUPPORTED
        with pytest.raises(ie.IEError) as e:
            y = empty((1, tiny.n))
            ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(W.coefficients(tiny, 1, 1)), y, 1)
        assert e.value.status == ie.IE_ERR_UNSUPPORTED


@pytest.mark.parametrize("symmetry", [0, 1])
def test_batch_of_scatterers_with_their_own_rhs_counts(symmetry):
    """Four scatterers in one plan, each translating only its own right-hand sides: the
    network kernel runs the FP32 path's work items (runs of pairs with one column count)."""
    b = W.small_batch()
    R = b.max_rhs
    members = [W.coefficients(m, R, 980 + g) for g, m in enumerate(b.members)]
    for g, m in enumerate(b.members):
        members[g][b.nrhs[g]:] = 0.0                      # padding columns stay zero
    refs = [oracle.cvfcnn_far_matvec(m, c[:b.nrhs[g]], H=50) for g, (m, c) in enumerate(zip(b.members, members))]
    pr = ie.problem_from_batch(b, ie.precmask(ie.IE_PREC_CVFCNN), symmetry=symmetry, exact_rhs=True)
    with ie.Plan(pr) as plan:
        y = empty((R, b.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(np.concatenate(members, axis=1)), y, R)
        for g, got in enumerate(b.split(host(y))):
            q = b.nrhs[g]
            assert rel_l2(got[:q], refs[g]) <= NET_TOL, g
            assert not np.any(got[q:]), g


@pytest.mark.parametrize("symmetry", [0, 1])
def test_footprint_covers_the_surrogate_plan(symmetry):
    """ie_plan_footprint (host only) bounds what a plan with the networks holds on the
    device (it also counts the fit's scratch, freed before the plan returns)."""
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    pr = ie.problem_from(p, ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_CVFCNN), symmetry=symmetry)
    fp = ie.ie_plan_footprint(pr)
    with ie.Plan(pr) as plan:
        held = plan.stats["device_bytes"]
    assert held <= fp
    nblk = 473 if symmetry else 16540
    assert held >= nblk * 198656           # the networks themselves


@pytest.mark.parametrize("hidden", [2, 64])
def test_hidden_width_limits(hidden, tiny):
    """A narrow network and the widest the kernel holds (no padding rows).  Width 1 is left
    out on purpose: blocks of axis and diagonal displacements are symmetric under rotations
    about d, so their two largest singular values are equal and a rank-1 network is not
    unique (any vector of that plane is correct); 2 is the narrowest width whose truncation
    is unique on this grid (relative gap 0.2 or more)."""
    c = W.coefficients(tiny, 1, 974)
    ref_net = oracle.cvfcnn_far_matvec(tiny, c, H=hidden)
    with _plan(tiny, [ie.IE_PREC_CVFCNN], symmetry=1, hidden=hidden) as plan:
        assert plan.stats["cvfcnn_hidden"] == hidden
        y = empty((1, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_CVFCNN, dev(c), y, 1)
        got = host(y)
    assert rel_l2(got, ref_net) <= NET_TOL
