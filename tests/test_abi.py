"""CPU checks of the C ABI: the library loads, exports every symbol include/ie.h
declares, and rejects bad problems in its host-side validation (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2501_04684_gb300 as ie
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2501_04684_gb300 import build
    return build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ie_[a-z_]+)\s*\(", src)) - {"ie_problem"})


def test_header_and_binding_agree():
    assert declared_functions() == sorted(ie.EXPORTED)


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in declared_functions() if f not in syms]
    assert not missing, missing
    L = ie.lib()
    for f in declared_functions():
        assert hasattr(L, f)
    assert "sm_103a" in ie.ie_version()


def test_status_strings(built):
    L = ie.lib()
    for s in range(7):
        assert L.ie_status_str(s).decode().startswith("IE_")


def _tiny_problem(**over):
    p = W.tiny()
    kw = dict(k=p.k, eta=p.eta, box_edge=p.a, grid_n=p.G, box_ijk=p.box_ijk, nb=p.nb, P=p.P, alpha=1.0,
              prec_mask=ie.precmask(ie.IE_PREC_FP32), max_rhs=1)
    kw.update(over)
    return ie.make_problem(**kw)


def test_footprint_is_host_only_and_counts_pairs(built):
    b = ie.ie_plan_footprint(_tiny_problem())
    # 316 coupling blocks of 192 x 192 complex64 at least
    assert b > 316 * 192 * 192 * 8
    b2 = ie.ie_plan_footprint(_tiny_problem(prec_mask=ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_BF16X3)))
    assert b2 > b + 316 * 147456 * 2 - 1


@pytest.mark.parametrize("bad", [
    dict(lattice=3),
    dict(max_rhs=0),
    dict(prec_mask=0),
    dict(nb=np.full(64, 193, dtype=np.int32)),
    dict(box_ijk=np.zeros((64, 3), dtype=np.int32)),          # duplicates
    dict(nb=None),                                           # P given without nb
    dict(box_group=np.r_[np.ones(32), np.zeros(32)], group_alpha=[1.0, 1.0]),   # ids decreasing
    dict(box_group=np.full(64, 2), group_alpha=[1.0, 1.0]),                     # id out of range
    dict(box_group=np.zeros(64)),                                               # no self terms
    dict(group_nrhs=[1]),                                                       # counts without groups
    dict(box_group=np.zeros(64), group_alpha=[1.0], group_nrhs=[2]),            # count above max_rhs
    dict(box_group=np.zeros(64), group_alpha=[1.0], group_nrhs=[0]),            # count below 1
    dict(prec_mask=ie.precmask(ie.IE_PREC_CVFCNN), cvfcnn_hidden=65),           # hidden width above 64
    dict(prec_mask=ie.precmask(ie.IE_PREC_CVFCNN), cvfcnn_hidden=-1),
    dict(prec_mask=ie.precmask(ie.IE_PREC_CVFCNN_FP32), cvfcnn_hidden=65),
    dict(prec_mask=1 << 8),                                                     # unknown precision
])
def test_validation_rejects(built, bad):
    pr = _tiny_problem(**bad)
    with pytest.raises(ie.IEError) as e:
        ie.ie_plan_footprint(pr)
    assert e.value.status == ie.IE_ERR_INVALID
    h = ctypes.c_void_p()
    assert ie.lib().ie_plan_create(ctypes.byref(pr), None, ctypes.byref(h)) == ie.IE_ERR_INVALID
    assert h.value is None


def test_batch_of_two_copies_is_valid(built):
    """Two scatterers may occupy the same cells; duplicates inside one stay invalid."""
    p = W.tiny()
    two = dict(box_ijk=np.concatenate([p.box_ijk, p.box_ijk]), nb=np.concatenate([p.nb, p.nb]),
               P=np.concatenate([p.P, p.P]), box_group=np.repeat([0, 1], 64), group_alpha=[1.0, 2.0])
    b1 = ie.ie_plan_footprint(_tiny_problem())
    b2 = ie.ie_plan_footprint(_tiny_problem(**two))
    assert b2 > b1
    bad = dict(two, box_group=np.zeros(128))
    bad["group_alpha"] = [1.0]
    with pytest.raises(ie.IEError):
        ie.ie_plan_footprint(_tiny_problem(**bad))


def test_symmetry_footprint_and_validation(built):
    """The symmetry-compressed store keeps one block per sorted |d|: a much smaller
    footprint on a shell; symmetry must be 0 or 1."""
    p = W.shell16()
    full = ie.ie_plan_footprint(ie.problem_from(p, ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_FP16X3)))
    comp = ie.ie_plan_footprint(ie.problem_from(p, ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_FP16X3), symmetry=1))
    assert comp < full / 3
    with pytest.raises(ie.IEError) as e:
        ie.ie_plan_footprint(_tiny_problem(symmetry=2))
    assert e.value.status == ie.IE_ERR_INVALID


def test_diagnostic_and_tuner_argument_checks(built):
    """Argument errors are reported before any device work (no GPU needed)."""
    L = ie.lib()
    assert L.ie_diag_bounded_wait(0.0, None) == ie.IE_ERR_INVALID
    assert L.ie_diag_bounded_wait(1e6, None) == ie.IE_ERR_INVALID
    assert L.ie_diag_wait_limit(-1) == ie.IE_ERR_INVALID
    info = ie.ie_tune_info()
    assert L.ie_plan_tune(None, ie.IE_PREC_FP16X3, 1, ctypes.byref(info), None) == ie.IE_ERR_INVALID
    assert L.ie_plan_check(None, None) == ie.IE_ERR_INVALID


MAP_BAD = [
    dict(lattice=3), dict(n_samples=63), dict(n_samples=257), dict(sample_radius=0.8),
    dict(sample_radius=float("nan")), dict(box_edge=0.0), dict(k=-1.0), dict(tikhonov=-1e-5),
    dict(pos_scale=1.6),          # a dipole outside S (radius 1.5 a)
    dict(off0=1), dict(decreasing=True), dict(nan_mom=True),
]


@pytest.mark.parametrize("bad", MAP_BAD, ids=lambda b: ",".join(b))
def test_map_basis_validation_rejects(built, bad):
    """ie_map_basis checks its spec, offsets and dipoles on the host before any device work."""
    a = W.BOX_EDGE
    fun_off, pos, mom = W.point_dipole_basis([2], 3, a=a)
    fun_off, pos, mom = fun_off.copy(), pos.copy(), mom.copy()
    args = dict(k=W.K0, eta=W.ETA0, box_edge=a, lattice=4, n_samples=128, sample_radius=1.5, tikhonov=0.0)
    args.update({k: v for k, v in bad.items() if k in args})
    if "pos_scale" in bad:
        pos[0] = np.array([1.0, 0.0, 0.0]) * bad["pos_scale"] * a
    if "off0" in bad:
        fun_off[0] = 1
    if "decreasing" in bad:
        fun_off[1] = fun_off[2] + 1
        pos, mom = np.vstack([pos, pos]), np.vstack([mom, mom])
    if "nan_mom" in bad:
        mom[0, 1] = complex(np.nan, 0.0)
    with pytest.raises(ie.IEError) as e:
        ie.ie_map_basis(args["k"], args["eta"], args["box_edge"], fun_off, pos, mom, n_samples=args["n_samples"],
                        sample_radius=args["sample_radius"], lattice=args["lattice"], tikhonov=args["tikhonov"],
                        stream=0)
    assert e.value.status == ie.IE_ERR_INVALID


def test_map_basis_of_no_functions_is_a_no_op(built):
    P, res = ie.ie_map_basis(W.K0, W.ETA0, W.BOX_EDGE, np.zeros(1, dtype=np.int64), np.zeros((0, 3)),
                             np.zeros((0, 3), dtype=np.complex128), stream=0)
    assert P.shape == (0, 192) and res.shape == (0,)


def test_store_footprint_host_only(built):
    """ie_store_footprint (no device work): every canonical far triple up to the reach, in the
    requested coupling-block precisions; invalid specs are refused."""
    p = W.tiny()
    D = 15
    nblk = (D + 1) * (D + 2) * (D + 3) // 6 - 4
    b16 = ie.ie_store_footprint(ie.store_spec(p.k, p.eta, p.a, D, ie.precmask(ie.IE_PREC_FP16X3)))
    b32 = ie.ie_store_footprint(ie.store_spec(p.k, p.eta, p.a, D, ie.precmask(ie.IE_PREC_FP32, ie.IE_PREC_FP16X3)))
    # 16-bit hi + lo images 294,912 B per block (plus a staging buffer when FP32 is not kept),
    # FP32 blocks 294,912 B more
    assert b16 >= nblk * 294912 and b32 >= nblk * (294912 + 192 * 192 * 8)
    for bad in (dict(max_disp=1), dict(max_disp=2000), dict(prec_mask=ie.precmask(ie.IE_PREC_CVFCNN)),
                dict(prec_mask=0), dict(lattice=3)):
        kw = dict(k=p.k, eta=p.eta, a=p.a, max_disp=D, prec_mask=ie.precmask(ie.IE_PREC_FP32)) | bad
        lattice = kw.pop("lattice", 4)
        with pytest.raises(ie.IEError) as e:
            ie.ie_store_footprint(ie.store_spec(kw["k"], kw["eta"], kw["a"], kw["max_disp"], kw["prec_mask"],
                                                lattice=lattice))
        assert e.value.status == ie.IE_ERR_INVALID


def test_binding_refuses_host_buffers():
    """The binding hands the library device buffers only: a numpy array or a CPU tensor is
    refused before any library call (there is no CPU path)."""
    import torch
    with pytest.raises(TypeError):
        ie._need(np.zeros(4, dtype=np.complex64), 4, "x")
    with pytest.raises(TypeError):
        ie._need(torch.zeros(4, dtype=torch.complex64), 4, "x")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libie.so every call raises: nothing falls back to another implementation."""
    monkeypatch.setattr(ie, "_lib", None)
    monkeypatch.setattr(ie, "LIB_PATH", str(tmp_path / "libie.so"))
    with pytest.raises(ImportError):
        ie.lib()
    with pytest.raises(ImportError):
        ie.ie_sym_map()
