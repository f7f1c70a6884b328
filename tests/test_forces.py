"""Atomic forces F_K = -Tr(rho dH/dR_K) + Tr(rho^E dS/dR_K) (Section 2: the Green's
function gives the total energy and the force).

CPU pins of the oracle: the derivative blocks against rebuilt matrices of
displaced structures; in the dense limit (nu = the full Krylov dimension) the
force equals minus the central difference of the Mermin free energy
A = E_band - kT S_el at fixed N_e, computed from a dense generalized
eigensolve of the displaced structures (a plausible sign, factor or index
error in the force formula fails it); the forces sum to zero; on a perfect
diamond lattice every force vanishes by symmetry, also at nu < M.  GPU:
marnoldi_forces against the oracle (FP64 and mixed).
"""

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from tbsynth import build_tb, build_tb_derivatives, config_c1, diamond, tiny_system
from tbsynth.structures import Structure, min_image

KT = 0.1


def _displaced(t, K, x, h):
    s = t.structure
    pos = s.positions.copy()
    pos[K, x] += h
    return build_tb(Structure(pos, s.species.copy(), s.box.copy()), check_spd=False)


def _safe_atom(t, margin=1e-3):
    """An atom none of whose pairs lies within `margin` of the 2.6 A cutoff."""
    s = t.structure
    n = t.n_block_rows
    d = np.linalg.norm(min_image(s.positions[None, :, :] - s.positions[:, None, :], s.box), axis=2)
    for K in range(n):
        r = np.delete(d[K], K)
        if np.all(np.abs(r - 2.6) > margin) and np.any(r < 2.6):
            return K
    raise RuntimeError("no atom clear of the cutoff")


def _free_energy(t, kT):
    Hd, Sd = t.dense()
    real = t.orbital_mask.astype(bool)
    eps = sla.eigh(Hd[np.ix_(real, real)], Sd[np.ix_(real, real)], eigvals_only=True)
    mu, _, _, _ = oracle.bisect(eps, np.ones_like(eps), t.n_electrons, kT)
    x = (eps - mu) / kT
    f = np.where(x >= 0, np.exp(-np.abs(x)) / (1 + np.exp(-np.abs(x))), 1 / (1 + np.exp(-np.abs(x))))
    ent = np.zeros_like(f)
    ok = (f > 0) & (f < 1)
    ent[ok] = f[ok] * np.log(f[ok]) + (1 - f[ok]) * np.log(1 - f[ok])
    return np.sum(2 * f * eps) + kT * np.sum(2 * ent)


def test_derivative_blocks_match_displaced_matrices():
    t = tiny_system(10, seed=4)
    dH, dS = build_tb_derivatives(t)
    K = _safe_atom(t)
    rows = np.repeat(np.arange(t.n_block_rows), np.diff(t.row_ptr))
    h = 1e-6
    for x in range(3):
        tp, tm = _displaced(t, K, x, h), _displaced(t, K, x, -h)
        assert np.array_equal(tp.col_idx, t.col_idx) and np.array_equal(tm.col_idx, t.col_idx)
        fdH = (tp.H - tm.H) / (2 * h)
        fdS = (tp.S - tm.S) / (2 * h)
        sign = np.where(t.col_idx == K, 1.0, 0.0) - np.where(rows == K, 1.0, 0.0)   # d/dR_K of d = R_J - R_I
        assert np.abs(fdH - sign[:, None, None] * dH[x]).max() < 1e-6
        assert np.abs(fdS - sign[:, None, None] * dS[x]).max() < 1e-7


def test_dense_limit_force_is_minus_free_energy_gradient():
    t = tiny_system(10, seed=4)
    dH, dS = build_tb_derivatives(t)
    M_real = int(t.orbital_mask.sum())
    ref = oracle.solve(t, nu=M_real, kT=KT)
    F = oracle.forces(t, ref.rho, ref.rhoE, dH, dS)
    K = _safe_atom(t)
    h = 1e-4
    for x in range(3):
        fd = -(_free_energy(_displaced(t, K, x, h), KT) - _free_energy(_displaced(t, K, x, -h), KT)) / (2 * h)
        assert abs(F[K, x] - fd) <= 2e-6 + 1e-7 * abs(fd), (x, F[K, x], fd)
    assert np.abs(F).max() > 0.1   # a real test: the forces are not all ~0


def test_forces_sum_to_zero():
    t = config_c1()
    dH, dS = build_tb_derivatives(t)
    ref = oracle.solve(t, nu=12, kT=KT)
    F = oracle.forces(t, ref.rho, ref.rhoE, dH, dS)
    assert np.abs(F.sum(axis=0)).max() <= 1e-10 * np.abs(F).max()
    assert np.abs(F).max() > 0.1


def test_perfect_diamond_has_no_forces():
    # nu = 12 stays below the dimension of the symmetric subspace that the
    # Krylov space of a single orbital of the perfect lattice can reach; past it
    # the process continues on rounding noise, which breaks the symmetry
    t = build_tb(diamond(2, jitter=0.0, seed=0))
    dH, dS = build_tb_derivatives(t)
    ref = oracle.solve(t, nu=12, kT=KT)
    F = oracle.forces(t, ref.rho, ref.rhoE, dH, dS)
    assert np.abs(F).max() <= 1e-9


# ---------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_3218_gb300 as mm
    from paper_1307_3218_gb300 import build as b
    mm.load(b.build())
    return mm


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_gpu_forces_match_oracle(m, prec):
    t = config_c1()
    dH, dS = build_tb_derivatives(t)
    ref = oracle.solve(t, nu=30, kT=KT)
    Fo = oracle.forces(t, ref.rho, ref.rhoE, dH, dS)
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, 30, 0, t.n_electrons, KT)
    Fg = m.marnoldi_forces(ctx, dH, dS)
    m.marnoldi_destroy(ctx)
    # FP64: 1e-9 of the largest force; mixed: 1e-3 eV/A (rho within 1e-5 and
    # rho^E within 1e-4 eV, times derivative entries of a few eV/A summed over
    # a block row, bound the difference at about that size)
    tol = 1e-9 * np.abs(Fo).max() if prec == 0 else 1e-3
    assert np.abs(Fg - Fo).max() <= tol
    assert np.abs(Fg.sum(axis=0)).max() <= (1e-10 if prec == 0 else 1e-6) * np.abs(Fo).max() * t.n_block_rows


@pytest.mark.gpu
def test_gpu_forces_regional_and_errors(m):
    t = tiny_system(40, seed=5)
    dH, dS = build_tb_derivatives(t)
    ref = oracle.solve(t, nu=16, kT=KT, region_atoms=24)
    Fo = oracle.forces(t, ref.rho, ref.rhoE, dH, dS)
    ctx = m.setup_system(t, 0)
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_forces(ctx, dH, dS)          # before a solve
    m.marnoldi_solve(ctx, None, 16, 24, t.n_electrons, KT)
    Fg = m.marnoldi_forces(ctx, dH, dS)
    assert np.abs(Fg - Fo).max() <= 1e-9 * np.abs(Fo).max()
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_forces(ctx, dH[:, :-1], dS)   # wrong size
    m.marnoldi_destroy(ctx)


FORCE_MUTATIONS = {
    "overlap_term_sign": ("np.add.at(F[:, x], rows, trH - trS)", "np.add.at(F[:, x], rows, trH + trS)"),
    "no_overlap_term": ("trS = np.einsum(\"kab,kab->k\", rEbar, dS[x])", "trS = 0.0 * trH"),
    "first_index_sign": ("np.add.at(F[:, x], rows, trH - trS)", "np.add.at(F[:, x], rows, -trH + trS)"),
    "transposed_derivative": ("trH = np.einsum(\"kab,kab->k\", rbar, dH[x])",
                              "trH = np.einsum(\"kab,kba->k\", rbar, dH[x])"),
    "energy_density_as_density": ("rEbar = 0.5 * (rE + rE[kt].transpose(0, 2, 1))",
                                  "rEbar = 0.5 * (r + r[kt].transpose(0, 2, 1))"),
}


@pytest.mark.parametrize("name", sorted(FORCE_MUTATIONS))
def test_force_mutation_is_caught(name, monkeypatch):
    """A planted slip in a copy of the oracle's force formula fails a pin."""
    import inspect
    old, new = FORCE_MUTATIONS[name]
    src = inspect.getsource(oracle.forces)
    assert src.count(old) == 1
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    monkeypatch.setattr(oracle, "forces", ns["forces"])
    failed = False
    for pin in (test_dense_limit_force_is_minus_free_energy_gradient, test_forces_sum_to_zero,
                test_perfect_diamond_has_no_forces):
        try:
            pin()
        except AssertionError:
            failed = True
            break
    assert failed, f"mutation {name} passed every pin"
