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


def _displacement_counts(p):
    """{d: pairs of boxes (b, b + d)} of a scatterer, by the autocorrelation of its box
    occupancy (FFT on a grid twice the size, so no displacement wraps around)."""
    G = p.G
    occ = np.zeros((2 * G,) * 3)
    ijk = np.asarray(p.box_ijk)
    occ[ijk[:, 0], ijk[:, 1], ijk[:, 2]] = 1.0
    f = np.fft.rfftn(occ)
    ac = np.rint(np.fft.irfftn(f * np.conj(f), s=occ.shape, axes=(0, 1, 2))).astype(np.int64)
    out = {}
    r = range(-G + 1, G)
    for dx in r:
        for dy in r:
            for dz in r:
                c = ac[dx % (2 * G), dy % (2 * G), dz % (2 * G)]
                if c:
                    out[(dx, dy, dz)] = int(c)
    return out


def test_shell_workload_counts():
    """The shells' box, far-pair, displacement-group, canonical-block and adjacent-pair
    counts (stated with the workloads and checked on the plans in the GPU tests), from the
    occupancy alone: far = Chebyshev distance >= 2, canonical block = sorted abs(d)."""
    want = {"shell16": (1264, 1575248, 16540, 473, 21184), "shell32": (5000, 24910952, 112160, 2780, None)}
    for name, (boxes, pairs, groups, canon, adjacent) in want.items():
        p = getattr(W, name)()
        counts = _displacement_counts(p)
        far = {d: c for d, c in counts.items() if max(map(abs, d)) >= 2}
        assert len(p.box_ijk) == boxes
        assert sum(far.values()) == pairs and len(far) == groups
        assert len({tuple(sorted(map(abs, d))) for d in far}) == canon
        if adjacent is not None:
            near = sum(c for d, c in counts.items() if 0 < max(map(abs, d)) <= 1)
            assert near == adjacent


def test_frozen_alphas_stay_above_the_longer_sigma_estimates():
    """The longer power iterations recorded beside the frozen alphas (make_alpha.py --check)
    start from the same seed, so they reproduce the frozen histories; alpha stays above
    their sigma, which keeps Z = alpha I + K nonsingular with GMRES contracting by sigma/alpha."""
    import json
    import os
    table = json.load(open(os.path.join(os.path.dirname(W.__file__), "alpha.json")))
    for name in ("shell16", "shell32"):
        e = table[name]
        h, hc = e["history"], e["history_check"]
        assert len(hc) > len(h) and np.allclose(hc[:len(h)], h, rtol=1e-9, atol=0)
        assert np.all(np.diff(hc) > 0) and e["sigma_check"] == hc[-1]
        assert e["alpha"] == W.alpha_for(name) and e["alpha"] / e["sigma_check"] > 1.15
