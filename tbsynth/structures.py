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

    Candidates are drawn uniformly in the box (batches of 4096 from the seeded
    generator) and taken in order; a candidate is accepted when no accepted atom
    lies closer than ``d_min`` (minimum-image distance).  Each batch is tested
    at once against the atoms accepted before it (a cell grid of edge >= d_min
    keeps the test local), and then in order against the batch's own earlier
    acceptances, which gives the same atoms as testing one candidate at a time.
    """
    from scipy.spatial import cKDTree

    L = (n_atoms / number_density(density_gcc)) ** (1.0 / 3.0)
    nc = max(1, int(L // d_min))
    cs = L / nc
    rng = np.random.default_rng(seed)
    d2min = d_min * d_min
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.int64)
    K = 2                                             # atom slots per cell, grown when one fills
    slots = np.full((nc * nc * nc, K), -1, dtype=np.int64)
    counts = np.zeros(nc * nc * nc, dtype=np.int64)
    pos = np.empty((n_atoms, 3))
    n = 0
    tries = 0
    limit = 200 * n_atoms + 10000

    def d2_to(P, x):
        # minimum-image squared distance from the points P to x, rounded as in
        # a one-candidate-at-a-time test: d -= L round(d / L), (dx^2 + dy^2) + dz^2
        d = P - x
        d = d - L * np.round(d / L)
        return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]

    while n < n_atoms:
        batch = rng.random((4096, 3)) * L
        cidx = (batch / cs).astype(np.int64) % nc                    # (B, 3)
        cell = (cidx[:, 0] * nc + cidx[:, 1]) * nc + cidx[:, 2]
        # against the atoms accepted before this batch
        nb = (cidx[:, None, :] + offs[None, :, :]) % nc               # (B, 27, 3)
        ncell = (nb[..., 0] * nc + nb[..., 1]) * nc + nb[..., 2]
        ids = slots[ncell]                                            # (B, 27, K)
        valid = ids >= 0
        d2 = d2_to(pos[np.where(valid, ids, 0)], batch[:, None, None, :])
        free = ~np.any(valid & (d2 < d2min), axis=(1, 2))
        # pairs of this batch's candidates that may conflict (exact test below):
        # only a candidate with an earlier partner needs the in-order test
        tree = cKDTree(np.minimum(batch, np.nextafter(L, 0.0)), boxsize=L)
        earlier: dict[int, list[int]] = {}
        for i, j in tree.query_pairs(d_min * (1.0 + 1e-9) + 1e-12):
            a, b = (i, j) if i < j else (j, i)
            earlier.setdefault(b, []).append(a)
        accepted = free.copy()
        for i in sorted(earlier):
            if accepted[i]:
                for k in earlier[i]:
                    if accepted[k] and d2_to(batch[k], batch[i]) < d2min:
                        accepted[i] = False
                        break
        # candidates are consumed in order until n_atoms are accepted
        order = np.flatnonzero(accepted)
        take = order[:n_atoms - n]
        used = int(take[-1]) + 1 if take.size == n_atoms - n else batch.shape[0]
        if tries + used > limit:
            # the one-at-a-time test stops at candidate number limit + 1
            if np.count_nonzero(accepted[:max(0, limit - tries)]) < n_atoms - n:
                raise RuntimeError("random packing did not converge; density too high for d_min")
        tries += used
        # the new atoms into the cell grid (slots within a cell in any order)
        c_new = cell[take]
        o = np.argsort(c_new, kind="stable")
        srt = c_new[o]
        starts = np.r_[0, np.flatnonzero(srt[1:] != srt[:-1]) + 1] if srt.size else np.zeros(0, np.int64)
        rank = np.empty(c_new.size, dtype=np.int64)   # earlier new atoms in the same cell
        rank[o] = np.arange(srt.size) - np.repeat(starts, np.diff(np.r_[starts, srt.size]))
        need = int((counts[c_new] + rank).max(initial=-1)) + 1
        if need > slots.shape[1]:
            slots = np.concatenate([slots, np.full((slots.shape[0], need - slots.shape[1]), -1, np.int64)], axis=1)
        slots[c_new, counts[c_new] + rank] = np.arange(n, n + take.size)
        np.add.at(counts, c_new, 1)
        pos[n:n + take.size] = batch[take]
        n += take.size
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
