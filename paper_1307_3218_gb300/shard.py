"""Columns split over ranks (one GPU each) with one shared Fermi level.

The columns of the multiple Arnoldi method are independent (arXiv:1307.3218,
Section 2: one Krylov subspace per basis index j), and only the Fermi level
couples them: N(mu) is a sum over all columns.  A run over several GPUs
therefore gives every rank the columns of a spatial domain of atoms (all
orbitals of an atom on one rank, so a regional solve's four columns share a
region) and finds mu by a bisection whose electron count is summed over the
ranks: one scalar all-reduce per step, no exchange of vectors.  The bisection
follows the library's own rule: bracket [min eps - 40 kT, max eps + 40 kT]
over all ranks, stop at |N - N_e| <= 1e-12 N_e or after 200 halvings.

Host logic only; every level count runs in the library on the rank's GPU
(``marnoldi_fermi_at``).  The reductions are callables, so the same code runs
over torch.distributed (NCCL between GPUs, gloo on CPUs) or in one process.
"""

from __future__ import annotations

from typing import Callable

import numpy as np

BISECT_RTOL = 1e-12
BISECT_MAXIT = 200
BRACKET_KT = 40.0


def _morton3(q: np.ndarray) -> np.ndarray:
    """Interleave the bits of three 10-bit integer coordinates (z-order key)."""
    key = np.zeros(q.shape[0], dtype=np.int64)
    for bit in range(10):
        for axis in range(3):
            key |= ((q[:, axis] >> bit) & 1).astype(np.int64) << (3 * bit + axis)
    return key


def domain_columns(positions: np.ndarray, box: np.ndarray, orbital_mask: np.ndarray | None,
                   world: int, rank: int) -> np.ndarray:
    """The real orbital columns of rank `rank` out of `world` spatial domains.

    Atoms are ordered along a z-order curve of their wrapped fractional
    coordinates (ties by atom index) and cut into `world` contiguous pieces of
    about equal real-column counts.  Returns the rank's columns 4 I + a,
    ascending.  Every atom's columns land on exactly one rank.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(box, dtype=np.float64).reshape(3)
    n = pos.shape[0]
    mask = (np.ones((n, 4), dtype=bool) if orbital_mask is None
            else np.asarray(orbital_mask).reshape(n, 4).astype(bool))
    frac = np.mod(pos / L, 1.0)
    q = np.minimum((frac * 1024).astype(np.int64), 1023)
    order = np.lexsort((np.arange(n), _morton3(q)))
    per_atom = mask[order].sum(axis=1)
    start = np.concatenate([[0], np.cumsum(per_atom)[:-1]])
    total = int(per_atom.sum())
    owner = np.minimum((start * world) // max(total, 1), world - 1)
    atoms = np.sort(order[owner == rank])
    cols = (4 * atoms[:, None] + np.arange(4)[None, :])[mask[atoms]]
    return np.sort(cols.reshape(-1)).astype(np.int64)


def fermi_bisect(count: Callable[[float], tuple[float, float]], lo: float, hi: float,
                 electron_count: float, allreduce_sum: Callable[[np.ndarray], np.ndarray]):
    """Bisection for mu with the electron count summed over the ranks.

    count(mu) returns this rank's (N, E); allreduce_sum adds a float64 array
    over the ranks.  Every rank runs the same halvings and returns the same
    (mu, N, E, iterations), N and E being the global sums at mu.
    """
    def total(mu):
        return allreduce_sum(np.asarray(count(mu), dtype=np.float64))

    n_lo = total(lo)[0]
    n_hi = total(hi)[0]
    if not (n_lo <= electron_count <= n_hi):
        raise ValueError(f"electron count {electron_count:.6g} outside [N(lo) = {n_lo:.6g}, "
                         f"N(hi) = {n_hi:.6g}]")
    mu, NE, it = lo, np.zeros(2), 0
    for it in range(1, BISECT_MAXIT + 1):
        mu = 0.5 * (lo + hi)
        NE = total(mu)
        if abs(NE[0] - electron_count) <= BISECT_RTOL * electron_count:
            break
        if NE[0] < electron_count:
            lo = mu
        else:
            hi = mu
    return mu, float(NE[0]), float(NE[1]), it


def level_bracket(eps_min: float, eps_max: float, kT: float,
                  allreduce_min: Callable[[float], float],
                  allreduce_max: Callable[[float], float]) -> tuple[float, float]:
    """The bisection bracket over all ranks' levels."""
    return (allreduce_min(eps_min) - BRACKET_KT * kT, allreduce_max(eps_max) + BRACKET_KT * kT)


def solve_sharded(ctx, columns: np.ndarray, nu: int, electron_count: float, kT: float,
                  allreduce_sum, allreduce_min, allreduce_max, region_atoms: int = 0):
    """Solve this rank's columns and adopt the Fermi level shared by all ranks.

    Runs the hot path on the rank's GPU for its columns, then the shared
    bisection with every count evaluated by the library; afterwards the
    context's density, energy and Green's-function calls use the shared mu.
    Returns (mu, N, E) with N and E summed over the ranks.
    """
    from . import marnoldi as m

    m.marnoldi_solve(ctx, columns, nu, region_atoms, electron_count, kT, mu_fixed=0.0)
    lo, hi = level_bracket(*m.marnoldi_level_range(ctx), kT, allreduce_min, allreduce_max)
    mu, N, E, _ = fermi_bisect(lambda x: m.marnoldi_fermi_at(ctx, x, kT), lo, hi, electron_count,
                               allreduce_sum)
    m.marnoldi_fermi_at(ctx, mu, kT)
    return mu, N, E


def torch_reducers(device=None):
    """(sum, min, max) reducers over torch.distributed's default group."""
    import torch
    import torch.distributed as dist

    def red(x, op):
        t = torch.as_tensor(np.asarray(x, dtype=np.float64), device=device).clone()
        dist.all_reduce(t, op=op)
        return t.cpu().numpy()

    return (lambda a: red(a, dist.ReduceOp.SUM),
            lambda v: float(red([v], dist.ReduceOp.MIN)[0]),
            lambda v: float(red([v], dist.ReduceOp.MAX)[0]))
