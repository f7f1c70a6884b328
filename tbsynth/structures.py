"""Seeded atomic structures in a periodic orthorhombic box (lengths in Angstrom).

* ``diamond``: conventional cubic diamond cells, every coordinate jittered by an
  i.i.d. normal displacement.  Stands in for the crystalline part of the
  sp2-sp3 carbon solid of the paper's strong-scaling run (Section 2, Fig. 1(a)).
* ``amorphous_carbon``: random sequential addition at a given mass density with
  a hard minimum distance.  Stands in for the amorphous sp2-sp3 nano-composite
  carbon of the same run.

Atoms are finally put in Morton (Z-curve) order of a cell grid so that atoms
that are close in space are close in index; this is what any order-N code does
with its atom list and it keeps the neighbour blocks of a BSR row close in
memory.  No arithmetic of the mArnoldi method lives here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CARBON = 0
HYDROGEN = 1

A_DIAMOND = 3.567          # conventional cubic lattice constant of diamond, Angstrom
CARBON_MASS_U = 12.011
ATOMIC_MASS_G = 1.66053906660e-24


@dataclass
class Structure:
    positions: np.ndarray      # (N, 3) float64, wrapped into [0, box)
    species: np.ndarray        # (N,) uint8, CARBON or HYDROGEN
    box: np.ndarray            # (3,) float64 periodic box lengths

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def _morton3(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray) -> np.ndarray:
    """Interleave the bits of three non-negative integer arrays (21 bits each)."""
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v
    return spread(ix) | (spread(iy) << np.uint64(1)) | (spread(iz) << np.uint64(2))


def spatial_sort(s: Structure, cell: float = 2.6) -> Structure:
    """Return the structure with atoms in Morton order of a grid of ~``cell`` cells."""
    n = np.maximum(1, np.floor(s.box / cell)).astype(np.int64)
    c = np.floor(s.positions / s.box * n).astype(np.int64)
    c = np.minimum(np.maximum(c, 0), n - 1)
    key = _morton3(c[:, 0], c[:, 1], c[:, 2])
    order = np.argsort(key, kind="stable")
    return Structure(s.positions[order].copy(), s.species[order].copy(), s.box.copy())


def diamond(ncell: int = 2, a: float = A_DIAMOND, jitter: float = 0.05, seed: int = 0,
            sort: bool = True) -> Structure:
    """ncell^3 conventional diamond cells (8 atoms each), jittered N(0, jitter^2) per coordinate."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    basis = np.concatenate([fcc, fcc + 0.25])
    g = np.arange(ncell)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)) * a
    box = np.full(3, ncell * a)
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    pos = np.mod(pos, box)
    s = Structure(pos, np.zeros(pos.shape[0], np.uint8), box)
    return spatial_sort(s) if sort else s


def number_density(density_gcc: float, mass_u: float = CARBON_MASS_U) -> float:
    """Atoms per cubic Angstrom for a mass density in g/cm^3."""
    return density_gcc / (mass_u * ATOMIC_MASS_G) * 1e-24


def amorphous_carbon(n_atoms: int, density_gcc: float = 3.0, d_min: float = 1.3,
                     seed: int = 0, sort: bool = True) -> Structure:
    """Random sequential addition of ``n_atoms`` carbon atoms in a periodic cube.

    Candidates are drawn uniformly in the box and accepted when no accepted atom
    lies closer than ``d_min`` (minimum-image distance).  A cell grid of edge
    >= d_min keeps each test local.
    """
    L = (n_atoms / number_density(density_gcc)) ** (1.0 / 3.0)
    nc = max(1, int(L // d_min))
    cs = L / nc
    rng = np.random.default_rng(seed)
    cells: dict[tuple[int, int, int], list[int]] = {}
    xs: list[float] = []
    ys: list[float] = []
    zs: list[float] = []
    d2min = d_min * d_min
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    batch = rng.random((4096, 3)) * L
    bi = 0
    tries = 0
    while len(xs) < n_atoms:
        if bi == batch.shape[0]:
            batch = rng.random((4096, 3)) * L
            bi = 0
        x, y, z = batch[bi]
        bi += 1
        tries += 1
        if tries > 200 * n_atoms + 10000:
            raise RuntimeError("random packing did not converge; density too high for d_min")
        cx, cy, cz = int(x / cs) % nc, int(y / cs) % nc, int(z / cs) % nc
        ok = True
        for a, b, c in offs:
            lst = cells.get(((cx + a) % nc, (cy + b) % nc, (cz + c) % nc))
            if not lst:
                continue
            for k in lst:
                dx = xs[k] - x
                dy = ys[k] - y
                dz = zs[k] - z
                dx -= L * round(dx / L)
                dy -= L * round(dy / L)
                dz -= L * round(dz / L)
                if dx * dx + dy * dy + dz * dz < d2min:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            cells.setdefault((cx, cy, cz), []).append(len(xs))
            xs.append(x)
            ys.append(y)
            zs.append(z)
    pos = np.stack([np.array(xs), np.array(ys), np.array(zs)], axis=1)
    s = Structure(pos, np.zeros(n_atoms, np.uint8), np.full(3, L))
    return spatial_sort(s) if sort else s


def min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    return d - box * np.round(d / box)


def min_pair_distance(s: Structure) -> float:
    """Smallest minimum-image distance between two atoms (used by tests)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(s.positions, boxsize=s.box)
    d, _ = tree.query(s.positions, k=2)
    return float(d[:, 1].min())


def unit_cell_volume(s: Structure) -> float:
    return float(math.prod(s.box))
