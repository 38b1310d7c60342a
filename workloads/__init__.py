"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds none of the method's arithmetic.  It only draws and
describes inputs:

* geometries (atoms, species, nuclear charges) and basis rules
  (radial functions per species: angular momentum l and a Gaussian exponent);
* grid and batching parameters;
* the input potential v(r) = sum_A -Z_A erf(|r - R_A|)/|r - R_A| evaluated at
  whatever points a caller passes (an operator F = v of Eqs. 29-30);
* random block-sparse matrices (density matrix P, adjoint seeds G) drawn per
  atom-pair block with a counter-based generator (numpy Philox keyed by
  seed, kind and the atom pair), so that any side that knows the block pattern
  gets identical values without sharing code or files.

Units: Bohr, Hartree.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# --------------------------------------------------------------------------
# workload description
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Species:
    name: str
    Z: float
    l: List[int]          # angular momentum of each radial function
    alpha: List[float]    # Gaussian exponent of each radial function

    @property
    def n_fn(self) -> int:
        return sum(2 * l + 1 for l in self.l)


@dataclasses.dataclass
class Workload:
    name: str
    xyz: np.ndarray               # (n_atoms, 3) Bohr
    species_of_atom: np.ndarray   # (n_atoms,) int32 index into species
    species: List[Species]
    # radial tabulation
    r_c: float = 6.0
    r_on: float = 5.0
    r_min: float = 1e-4
    n_log: int = 200
    # integration grid (per atom) and batching
    n_rad: int = 30
    R: float = 1.0
    n_theta: int = 8
    n_phi: int = 16
    r_nb: float = 12.0
    batch_max: int = 128
    # periodic cell: lattice vectors as rows (Bohr) and the image shell
    # T in [-n_shell, n_shell]^3; None for a molecule
    lattice: Optional[np.ndarray] = None
    n_shell: int = 0
    # batched independent molecules: atom ranges [n_molecules + 1]; None for one system
    mol_atom_ptr: Optional[np.ndarray] = None
    # partition of unity: "becke" (Becke 1988) or "stratmann" (Stratmann et al. 1996)
    partition: str = "becke"

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def Z_of_atom(self) -> np.ndarray:
        return np.array([self.species[s].Z for s in self.species_of_atom], dtype=np.float64)

    @property
    def nf_of_atom(self) -> np.ndarray:
        return np.array([self.species[s].n_fn for s in self.species_of_atom], dtype=np.int64)

    @property
    def n_basis(self) -> int:
        return int(self.nf_of_atom.sum())

    # flat species-major radial arrays (the layout both sides consume)
    @property
    def n_rad_per_species(self) -> np.ndarray:
        return np.array([len(s.l) for s in self.species], dtype=np.int32)

    @property
    def rad_l(self) -> np.ndarray:
        return np.array([l for s in self.species for l in s.l], dtype=np.int32)

    @property
    def rad_alpha(self) -> np.ndarray:
        return np.array([a for s in self.species for a in s.alpha], dtype=np.float64)

    @property
    def n_raw_points(self) -> int:
        return self.n_atoms * self.n_rad * self.n_theta * self.n_phi

    @property
    def n_molecules(self) -> int:
        return 1 if self.mol_atom_ptr is None else len(self.mol_atom_ptr) - 1

    def molecule(self, m: int) -> "Workload":
        """Molecule m of a batched workload as a workload of its own."""
        a0, a1 = int(self.mol_atom_ptr[m]), int(self.mol_atom_ptr[m + 1])
        return dataclasses.replace(self, name=f"{self.name}-mol{m}", xyz=self.xyz[a0:a1].copy(),
                                   species_of_atom=self.species_of_atom[a0:a1].copy(), mol_atom_ptr=None)

    def translated(self, shift) -> "Workload":
        return dataclasses.replace(self, xyz=self.xyz + np.asarray(shift, dtype=np.float64)[None, :])


def _draw_alphas(rng: np.random.Generator, n: int) -> List[float]:
    """Exponents log-uniform in [0.1, 10]."""
    return [float(10.0 ** rng.uniform(-1.0, 1.0)) for _ in range(n)]


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

LIGHT_MIX_L = {"O": [0, 0, 0, 1, 1, 2], "H": [0, 0, 1]}        # 3s2p1d = 14, 2s1p = 5
HEAVY_L = [0, 0, 1, 1, 2, 3]                                     # 2s2p1d1f = 20
LIGHT_L = [0, 0, 1]                                              # 2s1p = 5


def water(seed: int = 1001, n_rad: int = 30, n_theta: int = 8, n_phi: int = 16,
          batch_max: int = 128) -> Workload:
    """Three atoms: Z=8 at the origin, Z=1 at (+-1.43, 1.11, 0) Bohr.
    O carries 3s2p1d (14 functions), H 2s1p (5), 24 in total; exponents
    log-uniform in [0.1, 10] drawn species by species from `seed`;
    30 radial shells x (8 x 16) angular points per atom; batches <= 128."""
    rng = np.random.default_rng(seed)
    sp = [Species("O", 8.0, LIGHT_MIX_L["O"], _draw_alphas(rng, 6)),
          Species("H", 1.0, LIGHT_MIX_L["H"], _draw_alphas(rng, 3))]
    xyz = np.array([[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]])
    return Workload("water-3atom", xyz, np.array([0, 1, 1], dtype=np.int32), sp,
                    n_rad=n_rad, n_theta=n_theta, n_phi=n_phi, batch_max=batch_max)


def _place(rng: np.random.Generator, n: int, box: float, min_sep: float) -> np.ndarray:
    pts: List[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 1_000_000:
            raise RuntimeError("could not place atoms with the requested separation")
        c = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(c - p) >= min_sep for p in pts):
            pts.append(c)
    return np.array(pts)


def heavy_light_cluster(n_atoms: int = 64, box: float = 24.0, min_sep: float = 4.0,
                        seed: int = 1002, n_rad: int = 60, n_theta: int = 14, n_phi: int = 28,
                        batch_max: int = 300, name: Optional[str] = None) -> Workload:
    """Random cluster in a cube: half heavy (Z=82 or 53, 2s2p1d1f = 20 functions),
    half light (Z=6 or 1, 2s1p = 5 functions), the four species in equal
    numbers, assigned by a seeded permutation; positions uniform in the cube
    with rejection below `min_sep`; exponents log-uniform in [0.1, 10]."""
    rng = np.random.default_rng(seed)
    sp = [Species("Pb", 82.0, HEAVY_L, _draw_alphas(rng, len(HEAVY_L))),
          Species("I", 53.0, HEAVY_L, _draw_alphas(rng, len(HEAVY_L))),
          Species("C", 6.0, LIGHT_L, _draw_alphas(rng, len(LIGHT_L))),
          Species("H", 1.0, LIGHT_L, _draw_alphas(rng, len(LIGHT_L)))]
    kinds = np.array([k % 4 for k in range(n_atoms)], dtype=np.int32)
    kinds = rng.permutation(kinds).astype(np.int32)
    xyz = _place(rng, n_atoms, box, min_sep)
    return Workload(name or f"cluster-{n_atoms}atom", xyz, kinds, sp, n_rad=n_rad,
                    n_theta=n_theta, n_phi=n_phi, batch_max=batch_max)


def cluster64() -> Workload:
    """64 atoms in a 24 Bohr cube (the throughput workload): ~800 functions,
    60 radial x (14 x 28) = 392 angular points per atom, batches <= 300."""
    return heavy_light_cluster(64, 24.0, 4.0, seed=1002, name="cluster-64atom")


def cluster512() -> Workload:
    """The 512-atom adjoint configuration: the 64-atom rules in a 64 Bohr cube
    (minimum separation 4, ~6,400 functions), 100 x (14 x 28) points per atom
    (20.07M raw), batches <= 128, seed 1004."""
    return heavy_light_cluster(512, 64.0, 4.0, seed=1004, n_rad=100, n_theta=14, n_phi=28, batch_max=128,
                               name="cluster-512atom")


def small_cluster(n_atoms: int = 8, seed: int = 7, n_rad: int = 24, n_theta: int = 8,
                  n_phi: int = 16, batch_max: int = 200) -> Workload:
    """A reduced heavy/light cluster that the oracle finishes in seconds but
    that still spans several batches, n_b above 64 and a ragged tail."""
    box = 4.0 * n_atoms ** (1.0 / 3.0) + 2.0
    return heavy_light_cluster(n_atoms, box, 3.0, seed=seed, n_rad=n_rad, n_theta=n_theta,
                               n_phi=n_phi, batch_max=batch_max, name=f"small-{n_atoms}atom")


def single_atom(l_list=(0, 1, 2, 3), alphas=None, Z: float = 8.0, n_rad: int = 60,
                n_theta: int = 8, n_phi: int = 16, batch_max: int = 128) -> Workload:
    """One atom at the origin (closed-form pins and edge cases)."""
    l_list = list(l_list)
    if alphas is None:
        alphas = [1.5 + 0.5 * k for k in range(len(l_list))]
    sp = [Species("X", Z, l_list, list(alphas))]
    return Workload("single-atom", np.zeros((1, 3)), np.array([0], dtype=np.int32), sp,
                    n_rad=n_rad, n_theta=n_theta, n_phi=n_phi, batch_max=batch_max)


# --------------------------------------------------------------------------
# per-column operator inputs (eigenvalue and defining potential per radial)
# --------------------------------------------------------------------------

def column_operator(wl: Workload, seed: int = 1201):
    """(eps [n_rad_tot], knots [n_rad_tot][n_log]): per radial function a seeded
    eigenvalue in [-3, -0.1] Hartree and a free-atom-like potential
    V(r) = -Z erf(a r)/r (a in [0.8, 1.5], -2 Z a / sqrt(pi) at r = 0) given at the
    radial knots r_k = r_min (r_c/r_min)^(k/(n_log-1))."""
    rng = np.random.default_rng(seed)
    n_tot = int(sum(len(sp.l) for sp in wl.species))
    eps = rng.uniform(-3.0, -0.1, n_tot)
    a = rng.uniform(0.8, 1.5, n_tot)
    Z = np.array([sp.Z for sp in wl.species for _ in sp.l], dtype=np.float64)
    r = wl.r_min * (wl.r_c / wl.r_min) ** (np.arange(wl.n_log) / (wl.n_log - 1))
    knots = np.empty((n_tot, wl.n_log))
    for k in range(n_tot):
        x = a[k] * r
        knots[k] = -Z[k] * a[k] * np.where(x > 1e-8, _erf(x) / np.maximum(x, 1e-300), 2.0 / math.sqrt(math.pi))
    return eps, knots


# --------------------------------------------------------------------------
# small-component radial functions (synthetic stand-ins for the free-atom Dirac
# solutions, which are inputs of the integration)
# --------------------------------------------------------------------------

C_LIGHT = 137.035999084  # speed of light in Hartree atomic units


def _taper(r, r_on, r_c):
    """(c(r), c'(r)) of the quintic taper 1 - (10 s^3 - 15 s^4 + 6 s^5),
    s = (r - r_on)/(r_c - r_on), that the large-component radials carry."""
    s = np.clip((r - r_on) / (r_c - r_on), 0.0, 1.0)
    c = 1.0 - s ** 3 * (10.0 - 15.0 * s + 6.0 * s * s)
    dc = -30.0 * s * s * (1.0 - s) ** 2 / (r_c - r_on)
    return c, dc


def small_radial(r, l: int, alpha: float, kappa: int, V, r_on: float, r_c: float, c: float = C_LIGHT):
    """Q(r) = c / (2c^2 - V) (P' + kappa P/r) for P(r) = r^(l+1) exp(-alpha r^2) c(r)
    at radii r > 0 (V: the potential at r, or a constant)."""
    r = np.asarray(r, dtype=np.float64)
    cut, dcut = _taper(r, r_on, r_c)
    e = np.exp(-alpha * r * r)
    P = r ** (l + 1) * e * cut
    dP = ((l + 1) * r ** l - 2.0 * alpha * r ** (l + 2)) * e * cut + r ** (l + 1) * e * dcut
    return c / (2.0 * c * c - V) * (dP + kappa * P / r)


def small_component(wl: Workload, knots_V: np.ndarray, c: float = C_LIGHT):
    """The small-component basis of a workload: per large-component radial
    P(r) = r^(l+1) exp(-alpha r^2) c(r) and each kappa of its shell, in the
    order of its spinor functions (kappa = l for l >= 1, small-component
    l~ = l-1; then kappa = -l-1, l~ = l+1),
    Q(r) = c / (2c^2 - V(r)) (P'(r) + kappa P(r)/r) (the atomic-ZORA balance of
    Eq. 8b; V the radial's potential, given at the knots).  Returns
    (workload with the l~ per radial, Q at the knots [n_rad_S][n_log], index of
    the parent large-component radial [n_rad_S], kappa [n_rad_S])."""
    r = wl.r_min * (wl.r_c / wl.r_min) ** (np.arange(wl.n_log) / (wl.n_log - 1))
    r[-1] = wl.r_c
    species, Q, parent, kappas = [], [], [], []
    k = 0
    for sp in wl.species:
        l_s, a_s = [], []
        for l, alpha in zip(sp.l, sp.alpha):
            for kappa in ([l, -l - 1] if l >= 1 else [-1]):
                Q.append(small_radial(r, l, alpha, kappa, knots_V[k], wl.r_on, wl.r_c, c))
                l_s.append(l + 1 if kappa < 0 else l - 1)
                a_s.append(alpha)
                parent.append(k)
                kappas.append(kappa)
            k += 1
        species.append(Species(sp.name + "~", sp.Z, l_s, a_s))
    wl_s = dataclasses.replace(wl, name=wl.name + "-small", species=species)
    return wl_s, np.array(Q), np.array(parent, dtype=np.int64), np.array(kappas, dtype=np.int64)


# --------------------------------------------------------------------------
# input potential
# --------------------------------------------------------------------------

def molecule_batch(n_mol: int = 2000, seed: int = 1003, n_min: int = 3, n_max: int = 40, n_rad: int = 40,
                   n_theta: int = 10, n_phi: int = 20, batch_max: int = 128) -> Workload:
    """Many independent molecules integrated together: sizes N uniform in
    n_min..n_max, atoms O (probability 1/3, 3s2p1d) or H (2s1p) with the basis
    of the water workload, placed uniformly in a cube of side 3 N^(1/3) + 2
    Bohr with a minimum separation of 1.8 Bohr (drawn in order from `seed`).
    Every molecule keeps its own coordinates; they are independent through
    mol_atom_ptr, not through distance.  40 x (10 x 20) points per atom."""
    base = water()
    rng = np.random.default_rng(seed)
    xyz, kinds, ptr = [], [], [0]
    for _ in range(n_mol):
        n = int(rng.integers(n_min, n_max + 1))
        box = 3.0 * n ** (1.0 / 3.0) + 2.0
        xyz.append(_place(rng, n, box, 1.8))
        kinds.append((rng.uniform(size=n) >= 1.0 / 3.0).astype(np.int32))  # 0 = O, 1 = H
        ptr.append(ptr[-1] + n)
    return Workload(f"molecules-{n_mol}", np.vstack(xyz), np.concatenate(kinds), base.species, n_rad=n_rad,
                    n_theta=n_theta, n_phi=n_phi, batch_max=batch_max,
                    mol_atom_ptr=np.array(ptr, dtype=np.int32))


def periodic_cell(seed: int = 1005, cell=(9.0, 10.0, 11.0), n_atoms: int = 3, n_rad: int = 16,
                  n_theta: int = 6, n_phi: int = 12, r_nb: float = 8.0, n_shell: int = 2,
                  batch_max: int = 64) -> Workload:
    """A small orthorhombic periodic cell (the periodic-slab configuration in
    miniature): one heavier atom (2s2p1d) and light ones (2s1p) placed
    uniformly with a minimum image separation of 3 Bohr.  r_nb = 8 keeps the
    Becke neighbour sets small; n_shell = 2 covers every image within
    r_nb + r_c of the cell."""
    rng = np.random.default_rng(seed)
    L = np.diag(np.asarray(cell, dtype=np.float64))
    heavy = Species("Pb", 82.0, [0, 0, 1, 1, 2], _draw_alphas(rng, 5))
    light = Species("H", 1.0, [0, 0, 1], _draw_alphas(rng, 3))
    pts = []
    while len(pts) < n_atoms:
        p = rng.uniform(0.0, 1.0, 3) @ L
        ok = True
        for q in pts:
            d = p - q
            d = d - np.round(d / np.asarray(cell)) * np.asarray(cell)  # minimum image
            if np.linalg.norm(d) < 3.0:
                ok = False
        if ok:
            pts.append(p)
    kinds = np.array([0] + [1] * (n_atoms - 1), dtype=np.int32)
    return Workload("periodic-cell", np.array(pts), kinds, [heavy, light], n_rad=n_rad, n_theta=n_theta,
                    n_phi=n_phi, r_nb=r_nb, batch_max=batch_max, lattice=L, n_shell=n_shell)


HEAVY64_L = [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4                # 4 radials per l, l = 0..3: 64


def _place_periodic(rng, L, count, z_range, sep, placed, placed_sep):
    """`count` positions uniform in x, y over the orthorhombic cell L and in
    z over z_range (taken modulo the cell), rejected when closer than `sep` to
    a position placed by this call or `placed_sep[k]` to placed[k] (minimum
    image in all three directions); a hash of 4 Bohr cells finds the
    neighbours."""
    cell = 4.0
    nc = np.maximum((L // cell).astype(int), 1)
    size = L / nc
    buckets = {}

    def key(c):
        return tuple((np.floor(c / size).astype(int)) % nc)

    for q, sq in zip(placed, placed_sep):
        buckets.setdefault(key(q), []).append((q, sq))
    reach = int(math.ceil(max([sep] + list(placed_sep)) / size.min()))
    offs = [np.array(o) - reach for o in np.ndindex(2 * reach + 1, 2 * reach + 1, 2 * reach + 1)]
    out, tries = [], 0
    while len(out) < count:
        tries += 1
        if tries > 200 * count + 100000:
            raise RuntimeError("could not place atoms with the requested separation")
        c = np.array([rng.uniform(0.0, L[0]), rng.uniform(0.0, L[1]), rng.uniform(*z_range) % L[2]])
        k = np.array(key(c))
        ok = True
        for o in offs:
            for q, sq in buckets.get(tuple((k + o) % nc), ()):
                dv = c - q
                dv -= L * np.round(dv / L)
                if dv @ dv < sq * sq:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            out.append(c)
            buckets.setdefault(tuple(k), []).append((c, sep))
    return np.array(out).reshape(-1, 3)


def slab(seed: int = 2005, n_atoms: int = 3383, cell=(100.0, 100.0, 25.0), heavy_frac: float = 0.3,
         heavy_half: float = 8.0, n_rad: int = 40, n_theta: int = 12, n_phi: int = 25, batch_max: int = 300,
         name: Optional[str] = None) -> Workload:
    """The periodic-slab configuration (the shape of the paper's largest
    layered perovskite cell): an orthorhombic cell of n_atoms, a fraction
    heavy_frac heavy (one third Pb Z=82, two thirds I Z=53, four radial
    functions per l = 0..3: 64 functions) in the layer |z - c/2| < heavy_half
    at least 4 Bohr apart, the rest light (H 2s1p = 5 functions, C and N
    3s2p1d = 14, drawn in the proportions 1728 : 1152 : 144) in the rest of
    the cell at least 1.8 Bohr from any atom (minimum image); exponents
    log-uniform in [0.1, 10] per species; 40 x (12 x 25) points per atom,
    batches <= 300, r_nb = 12 and the image shell T in {-1, 0, 1}^3 (every
    cell edge is at least 2 r_nb)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(cell, dtype=np.float64)
    sp = [Species("Pb", 82.0, HEAVY64_L, _draw_alphas(rng, len(HEAVY64_L))),
          Species("I", 53.0, HEAVY64_L, _draw_alphas(rng, len(HEAVY64_L))),
          Species("H", 1.0, LIGHT_MIX_L["H"], _draw_alphas(rng, 3)),
          Species("C", 6.0, LIGHT_MIX_L["O"], _draw_alphas(rng, 6)),
          Species("N", 7.0, LIGHT_MIX_L["O"], _draw_alphas(rng, 6))]
    n_heavy = int(round(heavy_frac * n_atoms))
    n_light = n_atoms - n_heavy
    zc = 0.5 * L[2]
    heavy = _place_periodic(rng, L, n_heavy, (zc - heavy_half, zc + heavy_half), 4.0, [], [])
    light = _place_periodic(rng, L, n_light, (zc + heavy_half, zc - heavy_half + L[2]), 1.8,
                            list(heavy), [1.8] * n_heavy)
    hk = (rng.uniform(size=n_heavy) >= 1.0 / 3.0).astype(np.int32)           # 0 Pb, 1 I
    u = rng.uniform(size=n_light) * (1728 + 1152 + 144)
    lk = np.where(u < 1728, 2, np.where(u < 1728 + 1152, 3, 4)).astype(np.int32)
    return Workload(name or f"slab-{n_atoms}atom", np.vstack([heavy, light]), np.concatenate([hk, lk]), sp,
                    n_rad=n_rad, n_theta=n_theta, n_phi=n_phi, r_nb=12.0, batch_max=batch_max,
                    lattice=np.diag(L), n_shell=1)


def small_slab(n_atoms: int = 304, seed: int = 2006, n_rad: int = 20, n_theta: int = 8, n_phi: int = 16,
               batch_max: int = 300) -> Workload:
    """The slab's density and layering in a 30 x 30 x 25 Bohr cell (304
    atoms for the same atoms per volume): batches of up to about 800
    functions on a grid the oracle samples in seconds."""
    return slab(seed=seed, n_atoms=n_atoms, cell=(30.0, 30.0, 25.0), n_rad=n_rad, n_theta=n_theta, n_phi=n_phi,
                batch_max=batch_max, name=f"small-slab-{n_atoms}atom")


def _erf(x: np.ndarray) -> np.ndarray:
    try:
        from scipy.special import erf
        return erf(x)
    except ImportError:  # pragma: no cover
        return np.vectorize(math.erf)(x)


def _images(wl: Workload, reach: float) -> np.ndarray:
    """Lattice translations T.L of a periodic workload (rows), T in [-k, k]^3
    with k chosen so that every image within `reach` of the cell's atoms is
    present (the lattice vectors of the workloads here are orthogonal)."""
    L = np.asarray(wl.lattice, dtype=np.float64).reshape(3, 3)
    k = [int(math.ceil(reach / np.linalg.norm(L[d]))) + 1 for d in range(3)]
    T = np.array([(a, b, c) for a in range(-k[0], k[0] + 1) for b in range(-k[1], k[1] + 1)
                  for c in range(-k[2], k[2] + 1)], dtype=np.float64)
    return T @ L


def _near_box(P, centres, reach):
    """Indices of the centres within `reach` of the bounding box of points P
    (a periodic term vanishes exactly beyond 2 r_c, so the others add zeros)."""
    lo, hi = P.min(0), P.max(0)
    gap = np.maximum(0.0, np.maximum(lo[None, :] - centres, centres - hi[None, :]))
    return np.nonzero((gap * gap).sum(-1) < reach * reach)[0]


def _smoothstep_cut(d: np.ndarray, r_on: float, r_off: float) -> np.ndarray:
    s = np.clip((d - r_on) / (r_off - r_on), 0.0, 1.0)
    return 1.0 - s * s * s * (10.0 - 15.0 * s + 6.0 * s * s)


def potential(points: np.ndarray, wl: Workload, chunk: int = 65536, device=None) -> np.ndarray:
    """v(r) = sum_A -Z_A erf(d_A)/d_A, d_A = |r - R_A|, with
    erf(d)/d -> 2/sqrt(pi) (1 - d^2/3 + d^4/10) for d < 1e-4.
    Periodic workloads sum over the images within 2 r_c, each term times a
    quintic smoothstep that goes from 1 at 2 r_c - 1 to 0 at 2 r_c (the bare
    lattice sum of -Z/r diverges); each chunk of points sums over the images
    within 2 r_c of its bounding box only.  device (a torch device) evaluates
    the same expression in FP64 with torch there, for inputs of many million
    points."""
    points = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    Z = wl.Z_of_atom
    centres, Zc = wl.xyz, Z
    periodic = wl.lattice is not None
    if periodic:
        sh = _images(wl, 2.0 * wl.r_c + wl.r_nb)
        centres = (wl.xyz[None, :, :] + sh[:, None, :]).reshape(-1, 3)
        Zc = np.tile(Z, len(sh))
    if device is not None:
        return _potential_torch(points, centres, Zc, wl, periodic, device)
    out = np.empty(points.shape[0], dtype=np.float64)
    c = 2.0 / math.sqrt(math.pi)
    if periodic:
        chunk = min(chunk, 4096)  # consecutive points: tight boxes, few images each
    for s in range(0, points.shape[0], chunk):
        P = points[s:s + chunk]
        cs, zs = centres, Zc
        if periodic:
            near = _near_box(P, centres, 2.0 * wl.r_c)
            cs, zs = centres[near], Zc[near]
        d = np.sqrt(((P[:, None, :] - cs[None, :, :]) ** 2).sum(-1))
        small = d < 1e-4
        ds = np.where(small, 1.0, d)
        f = np.where(small, c * (1.0 - d * d / 3.0 + d ** 4 / 10.0), _erf(ds) / ds)
        if periodic:
            f = f * _smoothstep_cut(d, 2.0 * wl.r_c - 1.0, 2.0 * wl.r_c)
        out[s:s + chunk] = -(f * zs[None, :]).sum(-1)
    return out


def _potential_torch(points, centres, Zc, wl, periodic, device) -> np.ndarray:
    import torch
    out = np.empty(points.shape[0], dtype=np.float64)
    c = 2.0 / math.sqrt(math.pi)
    if periodic:  # chunks of consecutive points, each with the images near its bounding box
        step = 16384
    else:
        C = torch.tensor(centres, dtype=torch.float64, device=device)
        Zt = torch.tensor(Zc, dtype=torch.float64, device=device)
        step = max(1, (1 << 26) // max(len(Zc), 1))
    for s in range(0, points.shape[0], step):
        if periodic:
            near = _near_box(points[s:s + step], centres, 2.0 * wl.r_c)
            C = torch.tensor(centres[near], dtype=torch.float64, device=device)
            Zt = torch.tensor(Zc[near], dtype=torch.float64, device=device)
        P = torch.tensor(points[s:s + step], dtype=torch.float64, device=device)
        d = torch.sqrt(((P[:, None, :] - C[None, :, :]) ** 2).sum(-1))
        small = d < 1e-4
        ds = torch.where(small, torch.ones_like(d), d)
        f = torch.where(small, c * (1.0 - d * d / 3.0 + d ** 4 / 10.0), torch.special.erf(ds) / ds)
        if periodic:
            r_on, r_off = 2.0 * wl.r_c - 1.0, 2.0 * wl.r_c
            t = torch.clamp((d - r_on) / (r_off - r_on), 0.0, 1.0)
            f = f * (1.0 - t * t * t * (10.0 - 15.0 * t + 6.0 * t * t))
        out[s:s + step] = (-(f * Zt[None, :]).sum(-1)).cpu().numpy()
    return out


def molecule_potential(points: np.ndarray, point_atom: np.ndarray, wl: Workload, device=None) -> np.ndarray:
    """v of a batched workload: each point feels only its own molecule (the
    molecule of the atom that generated it, point_atom)."""
    points = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    mol = np.searchsorted(wl.mol_atom_ptr, np.asarray(point_atom), side="right") - 1
    order = np.argsort(mol, kind="stable")
    bounds = np.searchsorted(mol[order], np.arange(wl.n_molecules + 1))
    out = np.empty(points.shape[0], dtype=np.float64)
    for m in range(wl.n_molecules):
        sel = order[bounds[m]:bounds[m + 1]]
        if len(sel):
            out[sel] = potential(points[sel], wl.molecule(m), device=device)
    return out


# --------------------------------------------------------------------------
# random block-sparse matrices on a CSR block pattern
# --------------------------------------------------------------------------

KINDS = {"P": 1, "GV": 2, "GW0": 3, "GSOx": 4, "GSOy": 5, "GSOz": 6}


def _block_rng(seed: int, kind: str, A: int, B: int, T=(0, 0, 0)) -> np.random.Generator:
    key = [(int(seed) << 8) | KINDS[kind], (int(A) << 32) | int(B)]
    if tuple(T) == (0, 0, 0):
        return np.random.Generator(np.random.Philox(key=key))
    ctr = [((int(T[0]) + 512) << 20) | ((int(T[1]) + 512) << 10) | (int(T[2]) + 512), 0, 0, 1]
    return np.random.Generator(np.random.Philox(key=key, counter=ctr))


def block_values(seed: int, kind: str, A: int, B: int, nfA: int, nfB: int, antisym: bool,
                 T=(0, 0, 0)) -> np.ndarray:
    """Block (A, B, T) of a random matrix that is symmetric (antisym=False) or
    antisymmetric (antisym=True) as a whole, pairing block (A, B, T) with
    (B, A, -T): the pair is drawn once, keyed by the lexicographically smaller
    of the two, and transposed (and negated) for the other.  A block that is
    its own partner (A = B, T = 0) is symmetrised (antisymmetrised)."""
    T = tuple(int(t) for t in T)
    mT = tuple(-t for t in T)
    if (A, T) == (B, mT):
        R = _block_rng(seed, kind, A, A, T).standard_normal((nfA, nfA))
        return 0.5 * (R - R.T) if antisym else 0.5 * (R + R.T)
    if (A, B, T) < (B, A, mT):
        return _block_rng(seed, kind, A, B, T).standard_normal((nfA, nfB))
    R = _block_rng(seed, kind, B, A, mT).standard_normal((nfB, nfA))
    return -R.T if antisym else R.T.copy()


def fill_pattern(blk_ptr: np.ndarray, blk_col: np.ndarray, blk_off: np.ndarray,
                 nf_of_atom: np.ndarray, seed: int, kind: str, antisym: bool = False,
                 blk_T: Optional[np.ndarray] = None) -> np.ndarray:
    """Values of a random matrix on a CSR block pattern (rows = atoms,
    blocks dense row-major nf_A x nf_B at blk_off; blk_T the lattice shift of
    each block, [n_blocks][3], None for a molecule)."""
    n_atoms = len(blk_ptr) - 1
    out = np.zeros(int(blk_off[int(blk_ptr[-1])]), dtype=np.float64)
    Ts = None if blk_T is None else np.asarray(blk_T).reshape(-1, 3)
    for A in range(n_atoms):
        for q in range(int(blk_ptr[A]), int(blk_ptr[A + 1])):
            B = int(blk_col[q])
            T = (0, 0, 0) if Ts is None else tuple(int(t) for t in Ts[q])
            blk = block_values(seed, kind, A, B, int(nf_of_atom[A]), int(nf_of_atom[B]), antisym, T)
            out[int(blk_off[q]):int(blk_off[q]) + blk.size] = blk.ravel()
    return out


ADJOINT_KINDS = [("GV", False), ("GW0", False), ("GSOx", True), ("GSOy", True), ("GSOz", True)]
