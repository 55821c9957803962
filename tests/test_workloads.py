"""The seeded generators shared by both sides: determinism and the recipes' invariants."""
import numpy as np

import workloads as W


def test_point_dipole_basis_recipe():
    nb = np.array([3, 0, 5])
    f, pos, mom = W.point_dipole_basis(nb, 7, a=0.25, max_dipoles=3)
    counts = np.diff(f)
    assert f[0] == 0 and len(f) == nb.sum() + 1
    assert counts.min() >= 1 and counts.max() <= 3
    assert pos.shape == mom.shape == (f[-1], 3)
    assert np.all(np.abs(pos) <= 0.125)                    # inside the box, relative to its centre
    f2, pos2, mom2 = W.point_dipole_basis(nb, 7, a=0.25, max_dipoles=3)
    assert np.array_equal(f, f2) and np.array_equal(pos, pos2) and np.array_equal(mom, mom2)


def test_low_frequency_workloads_keep_geometry_and_seeds():
    base = W.tiny()
    for tag, edge in W.LFB_EDGES.items():
        p = W.lfb(base, tag)
        assert p.name == f"tiny_{tag}" and p.a == edge and p.k == base.k
        assert np.array_equal(p.box_ijk, base.box_ijk) and np.array_equal(p.P, base.P)
        assert np.isfinite(W.alpha_for(p.name))               # frozen by make_alpha.py
    assert W.lfb(W.shell16(), "lfb256").alpha == W.alpha_for("shell16_lfb256")


def test_identity_tiny_and_mapped_alphas():
    p = W.tiny_identity()
    assert p.P is None and np.all(p.nb == W.NU) and p.n == 64 * W.NU
    for name in ("tiny_mapped", "shell16_mapped"):
        assert W.alpha_for(name) > 0


def test_every_bench_variant_has_its_frozen_alpha():
    """bench.py --lfb lfb8|lfb256 and --mapped solve systems whose alpha make_alpha.py froze."""
    for name in ["shell16", "shell32"] + [f"shell16_{t}" for t in W.LFB_EDGES] + ["shell16_mapped"]:
        assert W.alpha_for(name) > 0, name
