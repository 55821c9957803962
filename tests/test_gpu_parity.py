"""GPU parity of the plain FP32 path against the FP64 oracle, through the C ABI.

Tolerance: relative L2 error <= 1e-6 for every product of the plain path (the
accuracy target of the FP32 path); coupling blocks within one FP32 rounding of the
FP64 values.  Full-size workloads are checked on seeded samples of target boxes
that the oracle computes one by one.
"""
import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W
from gpu_util import dev, empty, host, plan_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-6


def ragged_problem(seed=200, G=5, nbmax=64, nrhs=3):
    """Boxes of a 5^3 grid with a random half occupied, random nb in [1, nbmax],
    shuffled box order: ragged tiles, uneven groups, several right-hand sides."""
    g = W.rng(seed)
    ijk = W.full_grid(G)
    keep = g.random(len(ijk)) < 0.5
    ijk = ijk[keep][g.permutation(int(keep.sum()))]
    nb = g.integers(1, nbmax + 1, size=len(ijk)).astype(np.int32)
    nb[0], nb[1] = 1, 192
    p = W.Problem(name="ragged", G=G, box_ijk=ijk.astype(np.int32), nb=nb, P=W.random_P(g, nb), alpha=3.0e7)
    return p, W.coefficients(p, nrhs, seed + 1)


@pytest.fixture(scope="module")
def tiny():
    p = W.tiny()
    p.alpha = W.alpha_for("tiny")
    return p


def test_coupling_blocks_match_oracle(tiny):
    with plan_for(tiny) as plan:
        ds = np.array([[2, 0, 0], [0, -3, 1], [3, 3, 3], [-2, 1, 0], [0, 0, 0], [1, -1, 0], [7, -5, 11]],
                      dtype=np.int32)
        out = empty((len(ds), 192, 192))
        ie.ie_coupling_blocks(plan.handle, ds, out)
        got = host(out)
        for i, d in enumerate(ds):
            ref = oracle.coupling_block(tiny, d)
            ref32 = ref.astype(np.complex64).astype(np.complex128)
            # within one FP32 rounding of the FP64 value, component-wise
            ulp = np.spacing(np.abs(ref.real).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(got[i].real - ref.real) <= ulp + 1e-30)
            ulp = np.spacing(np.abs(ref.imag).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(got[i].imag - ref.imag) <= ulp + 1e-30)
            assert rel_l2(got[i], ref32) < 1e-7


@pytest.mark.parametrize("case", ["tiny", "ragged"])
def test_stages_match_oracle(case, tiny):
    if case == "tiny":
        p, c = tiny, W.coefficients(tiny, 2, 201)
    else:
        p, c = ragged_problem()
    nrhs = c.shape[0]
    with plan_for(p, max_rhs=nrhs) as plan:
        cd = dev(c)
        X = empty((nrhs, p.n_boxes, 192))
        ie.ie_aggregate(plan.handle, cd, X, nrhs)
        Xr = oracle.aggregate(p, c)
        assert rel_l2(host(X), Xr) <= TOL
        # translation on the oracle's own X (stage isolated)
        Y = empty((nrhs, p.n_boxes, 192))
        ie.ie_translate(plan.handle, ie.IE_PREC_FP32, dev(Xr), Y, nrhs)
        Yr = oracle.dipole_field(p, Xr, oracle.FAR)
        assert rel_l2(host(Y), Yr) <= TOL
        r = empty((nrhs, p.n))
        ie.ie_disaggregate(plan.handle, dev(Yr), r, nrhs)
        assert rel_l2(host(r), oracle.disaggregate(p, Yr)) <= TOL
        yn = empty((nrhs, p.n))
        ie.ie_near(plan.handle, cd, yn, nrhs)
        assert rel_l2(host(yn), oracle.operator(p, c, "near")) <= TOL


@pytest.mark.parametrize("which", [ie.IE_FAR, ie.IE_NEAR, ie.IE_FULL])
@pytest.mark.parametrize("case", ["tiny", "ragged"])
def test_matvec_matches_brute_force(which, case, tiny):
    if case == "tiny":
        p, c = tiny, W.coefficients(tiny, 1, 202)
    else:
        p, c = ragged_problem(seed=210)
    nrhs = c.shape[0]
    name = {ie.IE_FAR: "far", ie.IE_NEAR: "near", ie.IE_FULL: "full"}[which]
    with plan_for(p, max_rhs=nrhs) as plan:
        y = empty((nrhs, p.n))
        ie.ie_matvec(plan.handle, which, ie.IE_PREC_FP32, dev(c), y, nrhs)
        assert rel_l2(host(y), oracle.operator(p, c, name)) <= TOL


def test_identity_mapping_dipole_unknowns():
    p = W.tiny()
    p.P = None
    p.nb = np.full(p.n_boxes, 192, dtype=np.int32)
    p.alpha = 1.0e5
    c = W.coefficients(p, 1, 203)
    with plan_for(p) as plan:
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(c), y, 1)
        assert rel_l2(host(y), oracle.operator(p, c, "full")) <= TOL


@pytest.mark.parametrize("boxes", [
    [(0, 0, 0)],                                  # one box: no far zone, self block only
    [(0, 0, 0), (1, 1, 1)],                       # adjacent only: empty far zone
    [(0, 0, 0), (2, 0, 0)],                       # exactly one far pair each way
    [(0, 0, 0), (5, 0, 0), (0, 9, 3)],            # only far pairs (no neighbours)
])
def test_degenerate_geometries(boxes):
    g = W.rng(204)
    ijk = np.array(boxes, dtype=np.int32)
    nb = np.full(len(ijk), 24, dtype=np.int32)
    p = W.Problem(name="deg", G=10, box_ijk=ijk, nb=nb, P=W.random_P(g, nb), alpha=5.0e6)
    c = W.coefficients(p, 2, 205)
    with plan_for(p, max_rhs=2) as plan:
        for which, name in ((ie.IE_FAR, "far"), (ie.IE_FULL, "full")):
            y = empty((2, p.n))
            ie.ie_matvec(plan.handle, which, ie.IE_PREC_FP32, dev(c), y, 2)
            ref = oracle.operator(p, c, name)
            got = host(y)
            if np.linalg.norm(ref) == 0:
                assert np.all(got == 0)
            else:
                assert rel_l2(got, ref) <= TOL


def test_self_box_mode_excludes_the_box_itself():
    p, c = ragged_problem(seed=220, nrhs=1)
    p.self_box_mode = 1
    with plan_for(p) as plan:
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(c), y, 1)
        assert rel_l2(host(y), oracle.operator(p, c, "full")) <= TOL


def test_plane_wave_rhs(tiny):
    kh, pol = W.plane_wave_spec(1)
    kh2, pol2 = W.plane_wave_spec(3, seed=206)
    khat, pols = np.vstack([kh, kh2]), np.vstack([pol, pol2])
    with plan_for(tiny, max_rhs=4) as plan:
        v = empty((4, tiny.n))
        ie.ie_rhs_plane_wave(plan.handle, khat, pols, v)
        assert rel_l2(host(v), oracle.plane_wave_rhs(tiny, khat, pols)) <= TOL


def test_reciprocity_and_translation_invariance_on_gpu(tiny):
    c = W.coefficients(tiny, 2, 207)
    with plan_for(tiny, max_rhs=2) as plan:
        y = empty((2, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(c), y, 2)
        Zc = host(y)
    lhs, rhs = c[0] @ Zc[1], c[1] @ Zc[0]
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    q = W.tiny()
    q.alpha = tiny.alpha
    q.box_ijk = (tiny.box_ijk + np.array([3, 1, 2], dtype=np.int32)).astype(np.int32)
    q.G = 11
    with plan_for(q, max_rhs=2) as plan:
        y = empty((2, q.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(c), y, 2)
        assert rel_l2(host(y), Zc) <= 1e-6


def test_full_size_shell16_far_matvec_sampled():
    p = W.shell16()
    c = W.coefficients(p, 1, W.SEED_C["shell16"])
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    with plan_for(p) as plan:
        st = plan.stats
        assert st["n_far_pairs"] == 1575248 and st["n_far_disp"] == 16540 and st["n_boxes"] == 1264
        y = empty((1, p.n))
        ie.ie_matvec(plan.handle, ie.IE_FAR, ie.IE_PREC_FP32, dev(c), y, 1)
        got = host(y)[:, oracle.basis_rows(p, targets)]
    ref = oracle.far_matvec(p, c, targets=targets)
    assert rel_l2(got, ref) <= TOL


def test_solve_tiny_matches_dense_lu(tiny):
    Z = oracle.dense_operator(tiny)
    kh, pol = W.plane_wave_spec(1)
    v = oracle.plane_wave_rhs(tiny, kh, pol)
    ref = np.linalg.solve(Z, v[0])
    with plan_for(tiny) as plan:
        vd = dev(v)
        cd = empty((1, tiny.n))
        st, info = ie.ie_solve(plan.handle, vd, cd, 1, ie.solve_opts(tol=1e-6, restart=50))
        assert st == ie.IE_OK and info["converged"] == 1
        x = host(cd)[0]
    true_res = np.linalg.norm(v[0] - Z @ x) / np.linalg.norm(v[0])
    assert true_res <= 2e-6
    assert rel_l2(x, ref) <= 1e-5
    assert info["iterations"] <= 62          # (sigma/alpha)^k <= 1e-6 bound at alpha = 1.25 sigma


def test_solve_shell16_plane_wave():
    p = W.shell16()
    p.alpha = W.alpha_for("shell16")
    kh, pol = W.plane_wave_spec(1)
    targets = W.subsample_boxes(p, 12, W.SEED_SUBSAMPLE["shell16"])
    with plan_for(p) as plan:
        v = empty((1, p.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        cd = empty((1, p.n))
        st, info = ie.ie_solve(plan.handle, v, cd, 1, ie.solve_opts(tol=1e-6, restart=50))
        assert st == ie.IE_OK, info
        x = host(cd)
        vh = host(v)
    vref = oracle.plane_wave_rhs(p, kh, pol)
    assert rel_l2(vh, vref) <= TOL
    rows = oracle.basis_rows(p, targets)
    Zx = oracle.operator(p, x, "full", targets=targets)
    res = np.linalg.norm(Zx - vref[:, rows]) / np.linalg.norm(vref[:, rows])
    assert res <= 2e-6, res


def test_multi_rhs_solve_each_matches_alone(tiny):
    kh, pol = W.plane_wave_spec(3, seed=208)
    with plan_for(tiny, max_rhs=3) as plan:
        v = empty((3, tiny.n))
        ie.ie_rhs_plane_wave(plan.handle, kh, pol, v)
        c3 = empty((3, tiny.n))
        st, info = ie.ie_solve(plan.handle, v, c3, 3, ie.solve_opts(tol=1e-6))
        assert st == ie.IE_OK
        both = host(c3)
        for r in range(3):
            c1 = empty((1, tiny.n))
            st, _ = ie.ie_solve(plan.handle, v[r:r + 1].contiguous(), c1, 1, ie.solve_opts(tol=1e-6))
            assert st == ie.IE_OK
            assert rel_l2(host(c1)[0], both[r]) <= 1e-5


def test_bounded_wait_reports_timeout_and_context_survives(tiny):
    """A device wait on a signal that never comes gives up and reports IE_ERR_TIMEOUT;
    the context stays usable (a product afterwards is still correct) and a plan whose
    launches all completed reports IE_OK."""
    import time
    t0 = time.perf_counter()
    assert ie.ie_diag_bounded_wait(50.0) == ie.IE_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    c = W.coefficients(tiny, 1, 210)
    with plan_for(tiny) as plan:
        y = empty((1, tiny.n))
        ie.ie_matvec(plan.handle, ie.IE_FULL, ie.IE_PREC_FP32, dev(c), y, 1)
        assert ie.ie_plan_check(plan.handle) == ie.IE_OK
        assert rel_l2(host(y), oracle.operator(tiny, c, "full")) <= TOL


def test_solve_not_converged_reports_status_and_best_iterate(tiny):
    """Stopping at max_iters returns IE_ERR_NOT_CONVERGED with the iteration count and
    the residual reached, and the iterate written is better than x = 0."""
    kh, pol = W.plane_wave_spec(1)
    v = oracle.plane_wave_rhs(tiny, kh, pol)
    with plan_for(tiny) as plan:
        x = empty((1, tiny.n))
        st, info = ie.ie_solve(plan.handle, dev(v), x, 1, ie.solve_opts(tol=1e-12, max_iters=3, restart=50))
        assert st == ie.IE_ERR_NOT_CONVERGED
        assert info["converged"] == 0 and info["iterations"] == 3 and 0 < info["relres"] < 1, info
        xs = host(x)
    res = np.linalg.norm(oracle.operator(tiny, xs, "full")[0] - v[0]) / np.linalg.norm(v[0])
    assert abs(res - info["relres"]) <= 1e-3 * max(res, 1e-12) + 1e-6 and res < 1


def test_stepped_solver_matches_ie_solve(tiny):
    """The solver object (create / start / advance one cycle at a time / poll) reaches
    the same solution as ie_solve."""
    kh, pol = W.plane_wave_spec(2, seed=211)
    v = dev(oracle.plane_wave_rhs(tiny, kh, pol))
    opts = ie.solve_opts(tol=1e-6, restart=4)              # several restart cycles
    with plan_for(tiny, max_rhs=2) as plan:
        x_ref = empty((2, tiny.n))
        st, info_ref = ie.ie_solve(plan.handle, v, x_ref, 2, opts)
        assert st == ie.IE_OK
        s = ie.ie_solver_create(plan.handle, 2, opts)
        try:
            x = empty((2, tiny.n))
            ie.ie_solver_start(s, v, x)
            cycles = 0
            while True:
                ie.ie_solver_advance(s, 1)
                cycles += 1
                torch_cuda().cuda.synchronize()
                done, info = ie.ie_solver_poll(s)
                if done or cycles > 100:
                    break
            assert done and info["converged"] == 1 and cycles > 1, (cycles, info)
            assert info["iterations"] == info_ref["iterations"]
            assert rel_l2(host(x), host(x_ref)) <= 1e-6
        finally:
            ie.ie_solver_destroy(s)
