"""Seeded synthetic inputs for the group-by-group far-zone solver.

This module is shared by the CUDA library's tests/bench and by the CPU oracle's
tests.  It draws random numbers and lays out occupancy patterns; it holds none
of the method's arithmetic (no Green's function, no mapping, no translation).

Units: wavelength 1 (k = 2*pi), box edge a = 0.25, 4x4x4 dipole lattice per box
(192 unknowns per box), as in the paper's 4x4x4 uniform-dipole choice (§3).

Recipes (one per workload; all inputs synthetic, the paper's meshes are not
available, so sphere-like shells of boxes stand in for its PEC-sphere surface
discretisation, §5):

  tiny     4x4x4 grid, every box occupied, nb = 32 basis functions per box,
           P_b and c complex N(0,1) (seeds 11, 12).
  shell16  16^3 grid, boxes whose centre lies within 1 box of a sphere of
           radius 7 boxes about the grid centre (1,264 boxes), nb = 32
           (seeds 21, 22).
  shell32  32^3 grid, shell of radius 14 (5,000 boxes), nb = 32 (seeds 31, 33).
  batch    64 scatterers on 32^3: sphere / cube / ellipsoid shells of radius
           3..14, nb 16..64 per box, 1..8 plane waves each (seed 41).
  serve    Poisson arrivals; sphere shells with box counts log-uniform in
           [200, 20000] on the smallest grid in {16, 32, 64} that holds them,
           1..4 plane waves each (seed 51).
  *_lfb8, *_lfb256
           the same geometry and seeds with box edge a = lambda/8 or lambda/256
           (the paper's low-frequency regime, §3 and §5).  The closest far site
           pairs then have kR = 0.98 or 0.031; at lambda/256 a shell16 object is
           1/16 wavelength across, so every interaction is quasi-static and the
           1/(kR)^2 terms of the dyad dominate.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

K0 = 2.0 * math.pi          # free-space wavenumber, wavelength = 1
ETA0 = 376.730313668        # free-space impedance (ohm)
BOX_EDGE = 0.25             # a = lambda/4
LATTICE = 4                 # 4x4x4 dipoles per box
NU = 3 * LATTICE ** 3       # 192 unknowns per box

_HERE = os.path.dirname(os.path.abspath(__file__))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def complex_normal(g: np.random.Generator, shape) -> np.ndarray:
    """Re and Im each i.i.d. N(0,1), complex128."""
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im).astype(np.complex128)


def _grid_centres(G: int) -> tuple[np.ndarray, np.ndarray]:
    ii = np.stack(np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij"), -1)
    ijk = ii.reshape(-1, 3).astype(np.int32)
    c = ijk + 0.5 - G / 2.0           # box centre in units of a, grid centre at 0
    return ijk, c


def full_grid(G: int) -> np.ndarray:
    ijk, _ = _grid_centres(G)
    return ijk


def sphere_shell(G: int, R: float, width: float = 1.0) -> np.ndarray:
    """Boxes whose centre is within `width` boxes of a sphere of radius R boxes."""
    ijk, c = _grid_centres(G)
    r = np.sqrt((c * c).sum(1))
    return ijk[np.abs(r - R) <= width]


def cube_shell(G: int, R: float, width: float = 1.0) -> np.ndarray:
    """Boxes whose centre is within `width` boxes of a cube surface (Chebyshev radius R)."""
    ijk, c = _grid_centres(G)
    r = np.abs(c).max(1)
    return ijk[np.abs(r - R) <= width]


def ellipsoid_shell(G: int, semi: tuple[float, float, float], width: float = 1.0) -> np.ndarray:
    """Boxes within about `width` boxes of an ellipsoid with the given semi-axes (boxes).

    Distance to the surface is approximated to first order by (rho-1)/|grad rho|.
    """
    ijk, c = _grid_centres(G)
    s = np.asarray(semi, dtype=np.float64)
    rho = np.sqrt(((c / s) ** 2).sum(1))
    rho = np.maximum(rho, 1e-12)
    grad = np.sqrt(((c / s ** 2) ** 2).sum(1)) / rho
    dist = (rho - 1.0) / np.maximum(grad, 1e-12)
    return ijk[np.abs(dist) <= width]


@dataclass
class Problem:
    """One scatterer: geometry, mapping matrices and constants.

    P is packed box-major: box b's nb_b x 192 block (row-major) starts at
    row offset sum(nb[:b]).
    """
    name: str
    G: int
    box_ijk: np.ndarray                   # (n_boxes, 3) int32
    nb: np.ndarray                        # (n_boxes,) int32
    P: np.ndarray | None                  # (sum(nb), 192) complex128, None = identity
    alpha: float
    k: float = K0
    eta: float = ETA0
    a: float = BOX_EDGE
    lattice: int = LATTICE
    self_box_mode: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_boxes(self) -> int:
        return int(self.box_ijk.shape[0])

    @property
    def n(self) -> int:
        return int(self.nb.sum())

    @property
    def offsets(self) -> np.ndarray:
        o = np.zeros(self.n_boxes + 1, dtype=np.int64)
        np.cumsum(self.nb, out=o[1:])
        return o


def _alpha_table() -> dict:
    path = os.path.join(_HERE, "alpha.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def alpha_table_entry(name: str) -> dict:
    """Everything make_alpha.py recorded for a workload (alpha, sigma, iterations)."""
    return dict(_alpha_table()[name])


def alpha_for(name: str, default: float | None = None) -> float:
    """Frozen self-term alpha of a workload (written by make_alpha.py with the oracle)."""
    t = _alpha_table()
    if name in t:
        return float(t[name]["alpha"])
    if default is None:
        raise KeyError(f"no frozen alpha for workload {name!r}; run workloads/make_alpha.py")
    return default


def random_P(g: np.random.Generator, nb: np.ndarray) -> np.ndarray:
    return complex_normal(g, (int(nb.sum()), NU))


def make_problem(name: str, G: int, box_ijk: np.ndarray, nb_per_box, seed_P: int,
                 alpha: float | None = None, identity: bool = False) -> Problem:
    box_ijk = np.ascontiguousarray(box_ijk, dtype=np.int32)
    n_boxes = box_ijk.shape[0]
    if identity:
        nb = np.full(n_boxes, NU, dtype=np.int32)
        P = None
    else:
        nb = np.broadcast_to(np.asarray(nb_per_box, dtype=np.int32), (n_boxes,)).copy()
        P = random_P(rng(seed_P), nb)
    if alpha is None:
        alpha = alpha_for(name, default=float("nan"))
    return Problem(name=name, G=G, box_ijk=box_ijk, nb=nb, P=P, alpha=float(alpha))


def tiny(nb: int = 32) -> Problem:
    """4x4x4 grid, every box occupied, nb basis functions per box (seed 11)."""
    return make_problem("tiny", 4, full_grid(4), nb, seed_P=11)


def shell16(nb: int = 32, identity: bool = False) -> Problem:
    """16^3 grid, shell of radius 7 boxes (1,264 boxes) (seed 21)."""
    name = "shell16_identity" if identity else "shell16"
    return make_problem(name, 16, sphere_shell(16, 7.0), nb, seed_P=21, identity=identity)


def tiny_identity() -> Problem:
    """4x4x4 grid, every box occupied, identity P (nb = 192: c is the dipole vector)."""
    return make_problem("tiny_identity", 4, full_grid(4), NU, seed_P=11, identity=True)


def shell32(nb: int = 32) -> Problem:
    """32^3 grid, shell of radius 14 boxes (5,000 boxes) (seed 31)."""
    return make_problem("shell32", 32, sphere_shell(32, 14.0), nb, seed_P=31)


LFB_EDGES = {"lfb8": 1.0 / 8.0, "lfb256": 1.0 / 256.0}


def lfb(p: Problem, tag: str) -> Problem:
    """The workload `p` with its box edge shrunk to LFB_EDGES[tag] wavelengths.

    Geometry, P and seeds are unchanged; the name gains the tag and the frozen alpha
    (if any) is the one make_alpha.py recorded under that name.
    """
    name = f"{p.name}_{tag}"
    return Problem(name=name, G=p.G, box_ijk=p.box_ijk, nb=p.nb, P=p.P,
                   alpha=alpha_for(name, default=float("nan")), k=p.k, eta=p.eta,
                   a=LFB_EDGES[tag], lattice=p.lattice, self_box_mode=p.self_box_mode)


def point_dipole_basis(nb, seed: int, a: float = BOX_EDGE, max_dipoles: int = 3):
    """Seeded subdomain basis functions made of point dipoles, the input of the mapping
    construction (§2.1): box b owns nb[b] functions, each of 1..max_dipoles dipoles at
    positions uniform in the box (relative to its centre) with complex N(0,1) moments.

    Returns (fun_off (n_fun+1,) int64, pos (m, 3) float64, mom (m, 3) complex128), the
    functions in box order, so that mapped rows pack as P does.
    """
    g = rng(seed)
    nb = np.asarray(nb, dtype=np.int64)
    n_fun = int(nb.sum())
    counts = g.integers(1, max_dipoles + 1, size=n_fun)
    fun_off = np.zeros(n_fun + 1, dtype=np.int64)
    np.cumsum(counts, out=fun_off[1:])
    m = int(fun_off[-1])
    pos = g.uniform(-0.5 * a, 0.5 * a, size=(m, 3))
    mom = complex_normal(g, (m, 3))
    return fun_off, pos, mom


def coefficients(p: Problem, nrhs: int, seed: int) -> np.ndarray:
    """Basis coefficients c, layout [rhs][n], complex128 N(0,1)."""
    return complex_normal(rng(seed), (nrhs, p.n))


SEED_C = {"tiny": 12, "shell16": 22, "shell16_identity": 22, "shell32": 32}
SEED_SUBSAMPLE = {"shell32": 33, "shell16": 23, "tiny": 13}
SEED_MAPPED = {"tiny": 940, "shell16": 942}     # point-dipole basis functions of the mapped workloads
MAPPED_TIKHONOV = 1e-5                          # Tikhonov weight of their mapping, relative to ||A||_F


def subsample_boxes(p: Problem, count: int, seed: int) -> np.ndarray:
    """Seeded sample of target box slots (sorted, without replacement)."""
    count = min(count, p.n_boxes)
    return np.sort(rng(seed).choice(p.n_boxes, size=count, replace=False)).astype(np.int64)


def plane_wave_spec(nrhs: int, seed: int | None = None):
    """Incidence directions and polarisations of nrhs plane waves.

    seed None: the paper's excitation (x-polarised, propagating along +z, §5).
    Otherwise: k-hat uniform on the unit sphere, polarisation theta-hat.
    Returned as (khat (nrhs,3), pol (nrhs,3)) float64.  The field samples are
    computed by each side from these directions.
    """
    if seed is None:
        khat = np.tile(np.array([0.0, 0.0, 1.0]), (nrhs, 1))
        pol = np.tile(np.array([1.0, 0.0, 0.0]), (nrhs, 1))
        return khat, pol
    g = rng(seed)
    u = g.uniform(-1.0, 1.0, nrhs)             # cos(theta)
    phi = g.uniform(0.0, 2 * math.pi, nrhs)
    st = np.sqrt(1.0 - u * u)
    khat = np.stack([st * np.cos(phi), st * np.sin(phi), u], 1)
    pol = np.stack([u * np.cos(phi), u * np.sin(phi), -st], 1)   # theta-hat
    return khat, pol


def batch_scatterers(count: int = 64, G: int = 32, seed: int = 41,
                     rmin: int = 3, rmax: int = 14, nbmin: int = 16, nbmax: int = 64,
                     rhs_max: int = 8):
    """Batching workload: `count` scatterers with uneven occupancy and RHS counts.

    Returns a list of dicts with keys: kind, radius, box_ijk, nb, P, nrhs, khat, pol.
    """
    g = rng(seed)
    out = []
    for s in range(count):
        kind = ["sphere", "cube", "ellipsoid"][int(g.integers(0, 3))]
        R = int(g.integers(rmin, rmax + 1))
        if kind == "sphere":
            boxes = sphere_shell(G, R)
        elif kind == "cube":
            boxes = cube_shell(G, R)
        else:
            semi = (R, R * g.uniform(0.5, 1.0), R * g.uniform(0.5, 1.0))
            boxes = ellipsoid_shell(G, semi)
        nb = g.integers(nbmin, nbmax + 1, size=boxes.shape[0]).astype(np.int32)
        P = complex_normal(g, (int(nb.sum()), NU))
        nrhs = int(g.integers(1, rhs_max + 1))
        u = g.uniform(-1.0, 1.0, nrhs)
        phi = g.uniform(0.0, 2 * math.pi, nrhs)
        st = np.sqrt(1.0 - u * u)
        khat = np.stack([st * np.cos(phi), st * np.sin(phi), u], 1)
        pol = np.stack([u * np.cos(phi), u * np.sin(phi), -st], 1)
        out.append(dict(kind=kind, radius=R, G=G, box_ijk=boxes.astype(np.int32), nb=nb, P=P,
                        nrhs=nrhs, khat=khat, pol=pol))
    return out


def serve_requests(count: int = 256, seed: int = 51, rate_hz: float = 10.0,
                   nmin: int = 200, nmax: int = 20000, rhs_max: int = 4, nb: int = 32):
    """Serving workload: Poisson arrivals of scattering solves.

    Box counts log-uniform in [nmin, nmax]; each becomes a sphere shell of radius
    sqrt(n / (8 pi)) on the smallest grid G in {16, 32, 64} with G >= 2R + 4.
    Returns a list of dicts: t_arrival (s), G, radius, box_ijk, nb, seed_P, nrhs, khat, pol.
    P is drawn lazily from seed_P (see random_P) so the list stays small.
    """
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += g.exponential(1.0 / rate_hz)
        n = math.exp(g.uniform(math.log(nmin), math.log(nmax)))
        R = math.sqrt(n / (8 * math.pi))
        G = next(Gc for Gc in (16, 32, 64) if Gc >= 2 * R + 4)
        boxes = sphere_shell(G, R)
        nrhs = int(g.integers(1, rhs_max + 1))
        u = g.uniform(-1.0, 1.0, nrhs)
        phi = g.uniform(0.0, 2 * math.pi, nrhs)
        st = np.sqrt(1.0 - u * u)
        khat = np.stack([st * np.cos(phi), st * np.sin(phi), u], 1)
        pol = np.stack([u * np.cos(phi), u * np.sin(phi), -st], 1)
        out.append(dict(t_arrival=t, G=G, radius=R, box_ijk=boxes.astype(np.int32),
                        nb=np.full(boxes.shape[0], nb, dtype=np.int32),
                        seed_P=int(seed * 1000 + i), nrhs=nrhs, khat=khat, pol=pol))
    return out


# ---------------------------------------------------------------- batches of scatterers
@dataclass
class Batch:
    """Independent scatterers on one grid.  Each member is a Problem (what the oracle
    sees, one at a time); their concatenation in member order (boxes, basis unknowns)
    is what one batched plan takes.  Member g has nrhs[g] plane waves khat[g], pol[g]."""
    name: str
    G: int
    members: list
    nrhs: list
    khat: list
    pol: list

    @property
    def n_groups(self) -> int:
        return len(self.members)

    @property
    def box_ijk(self) -> np.ndarray:
        return np.concatenate([m.box_ijk for m in self.members]).astype(np.int32)

    @property
    def nb(self) -> np.ndarray:
        return np.concatenate([m.nb for m in self.members]).astype(np.int32)

    @property
    def P(self) -> np.ndarray:
        return np.concatenate([m.P for m in self.members])

    @property
    def box_group(self) -> np.ndarray:
        return np.concatenate([np.full(m.n_boxes, g, dtype=np.int32) for g, m in enumerate(self.members)])

    @property
    def group_alpha(self) -> np.ndarray:
        return np.array([m.alpha for m in self.members], dtype=np.float64)

    @property
    def unknown_offsets(self) -> np.ndarray:
        o = np.zeros(self.n_groups + 1, dtype=np.int64)
        np.cumsum([m.n for m in self.members], out=o[1:])
        return o

    @property
    def n(self) -> int:
        return int(self.unknown_offsets[-1])

    @property
    def max_rhs(self) -> int:
        return max(self.nrhs)

    def padded_waves(self, R: int | None = None):
        """(khat, pol) as (n_groups, R, 3); columns beyond a member's own waves get a
        zero polarisation (a zero right-hand side)."""
        R = self.max_rhs if R is None else R
        kh = np.zeros((self.n_groups, R, 3))
        kh[:, :, 2] = 1.0
        po = np.zeros((self.n_groups, R, 3))
        for g in range(self.n_groups):
            q = self.nrhs[g]
            kh[g, :q] = self.khat[g]
            po[g, :q] = self.pol[g]
        return kh, po

    def split(self, packed: np.ndarray) -> list:
        """Member slices of a packed [rhs][n] array."""
        o = self.unknown_offsets
        return [packed[..., o[g]:o[g + 1]] for g in range(self.n_groups)]


def batch_alpha(nb: np.ndarray) -> float:
    """Self term of a batched scatterer: the shell16 value rescaled by the square of
    the usual random-matrix estimate sqrt(nb) + sqrt(192) of ||P_b||_2 at the
    member's largest nb (the members are too large for the oracle's power iteration)."""
    ref = alpha_for("shell16")
    s = (math.sqrt(float(np.max(nb))) + math.sqrt(NU)) / (math.sqrt(32.0) + math.sqrt(NU))
    return float(ref * s * s)


def as_batch(items: list, name: str) -> Batch:
    """Batch from the dicts of batch_scatterers()."""
    members = []
    for i, it in enumerate(items):
        nb = np.asarray(it["nb"], dtype=np.int32)
        members.append(Problem(name=f"{name}[{i}]", G=it["G"], box_ijk=np.asarray(it["box_ijk"], dtype=np.int32),
                               nb=nb, P=it["P"], alpha=batch_alpha(nb)))
    return Batch(name=name, G=items[0]["G"], members=members, nrhs=[it["nrhs"] for it in items],
                 khat=[it["khat"] for it in items], pol=[it["pol"] for it in items])


def batch64() -> Batch:
    """64 scatterers on a 32^3 grid: sphere, cube and ellipsoid shells of radius 3..14,
    nb 16..64 per box, 1..8 plane waves each (seed 41)."""
    return as_batch(batch_scatterers(), "batch64")


def small_batch(count: int = 4, seed: int = 45) -> Batch:
    """A few small scatterers on an 8^3 grid (radius 1..2, nb 16..64, 1..3 waves)."""
    return as_batch(batch_scatterers(count=count, G=8, seed=seed, rmin=1, rmax=2, rhs_max=3), "small_batch")
