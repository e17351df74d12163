"""Seeded synthetic inputs shaped like the paper's docking workloads.

The paper (Section II-A) docks ligands of 21/43/108 atoms with 2/15/31
rotatable bonds against a receptor represented by interaction grids; none of
those input files exist here, so this module draws stand-ins of the same kind:

* a ligand as a random tree of atoms (bond length 1.5 A, atom types, partial
  charges summing to zero, a chosen set of rotatable bonds);
* a receptor as atoms scattered uniformly in a spherical shell around an
  empty pocket, and the grid box (dimensions, origin, spacing) around it;
* genotypes (translation, orientation quaternion, torsion angles).

This module holds no part of the docking method's arithmetic (no energy,
interpolation, pose or search code).  It only produces arrays; both the CUDA
library and the CPU oracle take them as plain inputs.  Every draw uses
``numpy.random.default_rng(seed)`` so that a seed fixes the whole input.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Atom type codes shared by every interface of this project.
TYPE_NAMES = ("C", "A", "N", "NA", "OA", "SA", "HD")
TYPE_CODE = {name: i for i, name in enumerate(TYPE_NAMES)}

BOND_LENGTH = 1.5        # A, every synthetic bond
MIN_13 = 2.2             # A, least distance of atoms 2 or 3 bonds apart
MIN_15 = 3.6             # A, least distance of atoms 4 or more bonds apart
PLACE_TRIES = 400        # random directions tried per new atom
MAX_VALENCE = 4
GRID_SPACING = 0.375     # A
POCKET_CENTER = (12.5, -3.25, 7.0)   # deliberately off the origin


@dataclass
class Ligand:
    xyz: np.ndarray          # [N,3] float64, A
    types: np.ndarray        # [N] int32 type codes
    charges: np.ndarray      # [N] float64, sums to ~0
    bonds: np.ndarray        # [B,2] int32, atom index pairs
    rotatable: np.ndarray    # [B] int32, 1 = rotatable bond

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_torsions(self) -> int:
        return int(self.rotatable.sum())

    @property
    def n_genes(self) -> int:
        return 7 + self.n_torsions

    def nbytes(self) -> int:
        return int(self.xyz.nbytes + self.types.nbytes + self.charges.nbytes
                   + self.bonds.nbytes + self.rotatable.nbytes)


@dataclass
class Receptor:
    xyz: np.ndarray          # [R,3] float64
    types: np.ndarray        # [R] int32
    charges: np.ndarray      # [R] float64


@dataclass
class GridBox:
    dims: tuple              # (nx, ny, nz) grid points per axis
    origin: tuple            # A, coordinates of point (0,0,0)
    spacing: float = GRID_SPACING
    map_types: tuple = field(default_factory=tuple)   # ligand type code per type map

    @property
    def n_maps(self) -> int:
        return len(self.map_types) + 2     # type maps, then electrostatic, then desolvation

    def box_lo(self):
        return np.asarray(self.origin, dtype=np.float64)

    def box_hi(self):
        return self.box_lo() + (np.asarray(self.dims, dtype=np.float64) - 1.0) * self.spacing


def _unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def _place_one_by_one(rng, origin, others, need):
    """Draw directions one at a time until the new atom keeps every required
    distance (slack >= 0), at most PLACE_TRIES times; keep the least crowded
    (first of the largest slack)."""
    best, best_slack = None, -np.inf
    for _ in range(PLACE_TRIES):
        p = origin + BOND_LENGTH * _unit(rng)
        slack = float(np.min(np.linalg.norm(others - p, axis=1) - need))
        if slack > best_slack:
            best, best_slack = p, slack
        if slack >= 0.0:
            break
    return best


def _place(rng, origin, others, need):
    """_place_one_by_one, with the tries screened all at once: the candidate
    directions are drawn as one block from a copy of the generator's state,
    the try the one-by-one loop would stop at is found from all slacks, and
    the generator is then advanced by exactly the draws that loop makes.
    Where rounding could decide the outcome (a slack within 1e-9 of zero, or
    of the best slack), the one-by-one loop itself runs instead.  Same
    directions, same atom, same generator state afterwards."""
    state = rng.bit_generator.state
    v = rng.standard_normal((PLACE_TRIES, 3))
    p = origin + BOND_LENGTH * (v / np.sqrt(np.einsum("ij,ij->i", v, v))[:, None])

    def slacks(rows):
        d = np.sqrt(((p[rows, None, :] - others[None, :, :]) ** 2).sum(axis=2))
        return (d - need).min(axis=1)

    slack = slacks(slice(0, 16))          # most atoms fit within the first few tries
    if not (slack >= 0.0).any():
        slack = np.concatenate([slack, slacks(slice(16, PLACE_TRIES))])
    ok = np.nonzero(slack >= 0.0)[0]
    i = int(ok[0]) if ok.size else int(np.argmax(slack))
    top = slack[i]
    close = np.abs(slack[: i + 1]) < 1e-9 if ok.size else np.abs(slack) < 1e-9
    if ok.size == 0:
        close |= np.abs(slack - top) < 1e-9
        close[i] = False
    rng.bit_generator.state = state
    if close.any():
        return _place_one_by_one(rng, origin, others, need)
    rng.standard_normal(((i + 1) if ok.size else PLACE_TRIES, 3))
    w = v[i]
    return origin + BOND_LENGTH * (w / np.linalg.norm(w))


def make_ligand(n_atoms: int, n_torsions: int, type_names=TYPE_NAMES, seed: int = 0) -> Ligand:
    """Random tree ligand: atom k bonds to a uniformly chosen earlier atom of
    valence < 4, 1.5 A away in a random direction.  The direction is redrawn
    (up to PLACE_TRIES times, keeping the least crowded one) while the new
    atom lands within MIN_13 of an atom 2 or 3 bonds away or within MIN_15 of
    one 4 or more bonds away, so that the reference conformation has no
    steric clash of the kind the intramolecular term penalises.
    ``n_torsions`` rotatable bonds are drawn among bonds whose two ends both
    have degree >= 2; when fewer exist, all of them are used (read the
    effective count from ``Ligand.n_torsions``)."""
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rng = np.random.default_rng(seed)
    xyz = np.zeros((n_atoms, 3))
    deg = np.zeros(n_atoms, dtype=np.int64)
    hops = np.zeros((n_atoms, n_atoms), dtype=np.int64)  # bonds between atoms
    bonds = []
    for k in range(1, n_atoms):
        cand = np.nonzero(deg[:k] < MAX_VALENCE)[0]
        parent = int(cand[rng.integers(len(cand))])
        hk = hops[parent, :k] + 1
        need = np.where(hk <= 1, 0.0, np.where(hk <= 3, MIN_13, MIN_15))
        xyz[k] = _place(rng, xyz[parent], xyz[:k], need)
        hops[k, :k] = hk
        hops[:k, k] = hk
        bonds.append((parent, k))
        deg[parent] += 1
        deg[k] += 1
    bonds = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
    rot = np.zeros(len(bonds), dtype=np.int32)
    inner = [b for b in range(len(bonds)) if deg[bonds[b, 0]] >= 2 and deg[bonds[b, 1]] >= 2]
    if inner and n_torsions > 0:
        pick = rng.choice(len(inner), size=min(n_torsions, len(inner)), replace=False)
        rot[np.asarray(inner)[pick]] = 1
    codes = np.asarray([TYPE_CODE[t] for t in type_names], dtype=np.int32)
    types = codes[rng.integers(len(codes), size=n_atoms)].astype(np.int32)
    q = rng.uniform(-0.4, 0.4, size=n_atoms)
    q = q - q.mean()
    # Centre the drawn coordinates somewhere away from the origin so that
    # frame bugs cannot hide behind a zero centroid.
    xyz = xyz + np.asarray([1.25, -0.5, 2.0])
    return Ligand(xyz=xyz, types=types, charges=q, bonds=bonds, rotatable=rot)


def make_receptor(n_atoms: int, inner: float = 10.0, outer: float = 30.0,
                  center=POCKET_CENTER, type_names=TYPE_NAMES, seed: int = 1) -> Receptor:
    """Receptor atoms uniform in the volume of the shell inner <= r <= outer
    around ``center`` (the empty pocket is the ball of radius ``inner``)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=n_atoms)
    r = np.cbrt(inner ** 3 + u * (outer ** 3 - inner ** 3))
    d = rng.standard_normal((n_atoms, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    xyz = np.asarray(center, dtype=np.float64) + r[:, None] * d
    codes = np.asarray([TYPE_CODE[t] for t in type_names], dtype=np.int32)
    types = codes[rng.integers(len(codes), size=n_atoms)].astype(np.int32)
    q = rng.uniform(-0.4, 0.4, size=n_atoms)
    q = q - q.mean()
    return Receptor(xyz=xyz, types=types, charges=q)


def make_box(n: int, center=POCKET_CENTER, type_names=TYPE_NAMES, spacing=GRID_SPACING) -> GridBox:
    """Cubic grid of n^3 points centred on ``center``."""
    c = np.asarray(center, dtype=np.float64)
    origin = c - 0.5 * (n - 1) * spacing
    return GridBox(dims=(n, n, n), origin=tuple(float(v) for v in origin), spacing=spacing,
                   map_types=tuple(TYPE_CODE[t] for t in type_names))


def make_genotypes(n: int, n_torsions: int, box: GridBox, seed: int = 0) -> np.ndarray:
    """[n, 7+T] float32 genotypes: translation uniform in the grid box,
    orientation a uniformly random unit quaternion (w, x, y, z), torsions
    uniform in [-pi, pi)."""
    rng = np.random.default_rng(seed)
    g = np.zeros((n, 7 + n_torsions), dtype=np.float64)
    g[:, 0:3] = rng.uniform(box.box_lo(), box.box_hi(), size=(n, 3))
    qv = rng.standard_normal((n, 4))
    g[:, 3:7] = qv / np.linalg.norm(qv, axis=1, keepdims=True)
    g[:, 7:] = rng.uniform(-np.pi, np.pi, size=(n, n_torsions))
    return g.astype(np.float32)


# ---------------------------------------------------------------------------
# The workloads of the benchmark configurations, by what they are.

@dataclass
class Workload:
    name: str
    ligand: Ligand
    receptor: Receptor
    box: GridBox
    nruns: int
    max_evals: int
    pop_size: int
    ls_iters: int
    ls_rate_pct: int
    seed: int


def small_ligand_workload() -> Workload:
    """16 atoms / 4 torsions, types {C,A,N,OA,HD}, 40^3 grid, 7 maps,
    800 receptor atoms; 10 runs x 100k evaluations, ADADELTA 100 iterations."""
    types = ("C", "A", "N", "OA", "HD")
    return Workload("small-ligand 16 atoms/4 torsions, 40^3x7 maps, 10 runs x 100k evals",
                    make_ligand(16, 4, types, seed=0), make_receptor(800, type_names=types, seed=1),
                    make_box(40, type_names=types), nruns=10, max_evals=100_000, pop_size=150,
                    ls_iters=100, ls_rate_pct=6, seed=0)


def drug_ligand_workload() -> Workload:
    """40 atoms / 10 torsions, 7 types, 64^3 grid, 9 maps, 3000 receptor
    atoms; 50 runs x 2.5M evaluations, ADADELTA 300 iterations."""
    return Workload("drug-size ligand 40 atoms/10 torsions, 64^3x9 maps, 50 runs x 2.5M evals",
                    make_ligand(40, 10, TYPE_NAMES, seed=0), make_receptor(3000, seed=1),
                    make_box(64), nruns=50, max_evals=2_500_000, pop_size=150,
                    ls_iters=300, ls_rate_pct=6, seed=0)
