"""The k-th eigen level and vector (Section 2, the paragraph on the k-th eigen
level and Eq. 3; the inner-product sign rule of the Appendix).

CPU pins of the oracle: in the dense limit (nu = the full Krylov dimension)
eps_k is the k-th generalized eigenvalue and phi_k the S-normalised
eigenvector of a dense eigensolve, up to one overall sign; the integrated
density of states counts every real orbital; below the dense limit the
overlap of phi_k with the exact eigenvector grows toward 1 with nu.  GPU:
marnoldi_eigenstate against the oracle.
"""

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from tbsynth import config_c1, tiny_hydrocarbon, tiny_system

SIGMA = 1e-3


def _exact(t):
    Hd, Sd = t.dense()
    real = t.orbital_mask.astype(bool)
    ev, V = sla.eigh(Hd[np.ix_(real, real)], Sd[np.ix_(real, real)])
    return ev, V, real, Sd[np.ix_(real, real)]


@pytest.mark.parametrize("maker,ks", [(lambda: tiny_system(10, seed=4), (1, 5, 20, 21, 33, 40)),
                                      (lambda: tiny_hydrocarbon(12, 4, seed=1), (3, 14, 15, 30))])
def test_dense_limit_is_the_exact_eigenpair(maker, ks):
    t = maker()
    ev, V, real, _ = _exact(t)
    m_real = int(real.sum())
    for k in ks:
        gap = min(ev[k - 1] - ev[k - 2] if k > 1 else np.inf, ev[k] - ev[k - 1] if k < m_real else np.inf)
        assert gap > 50 * SIGMA   # an isolated level, so the smoothing does not mix neighbours
        ek, phi, info = oracle.eigenstate(t, k, m_real, SIGMA)
        assert abs(ek - ev[k - 1]) <= 1e-9 * max(1.0, abs(ev[k - 1]))
        ex = np.zeros(t.M)
        ex[real] = V[:, k - 1]
        sgn = 1.0 if phi @ ex >= 0 else -1.0
        assert np.abs(phi - sgn * ex).max() <= 1e-8 * np.abs(ex).max()
        assert np.all(phi[~real] == 0.0)


def test_idos_counts_every_orbital():
    t = tiny_hydrocarbon(12, 4, seed=1)
    c = oracle.columns(t, t.real_columns(), 16)
    e, _ = oracle.valid_levels(c)
    m_real = t.real_columns().size
    assert oracle.idos(c, e.max() + 60 * SIGMA, SIGMA) == pytest.approx(m_real, rel=1e-12)
    assert oracle.idos(c, e.min() - 60 * SIGMA, SIGMA) == pytest.approx(0.0, abs=1e-12)
    grid = np.linspace(e.min(), e.max(), 50)
    vals = [oracle.idos(c, g, 0.1) for g in grid]
    assert np.all(np.diff(vals) >= -1e-12)


def test_overlap_grows_with_nu():
    t = tiny_system(24, seed=3)
    ev, V, real, Sr = _exact(t)
    k = int(round(t.n_electrons / 2))   # the highest occupied level
    ov = []
    for nu in (30, 60, int(real.sum())):
        _, phi, _ = oracle.eigenstate(t, k, nu, SIGMA)
        p = phi[real]
        ov.append(abs(p @ Sr @ V[:, k - 1]) / np.sqrt(p @ Sr @ p))
    assert ov[0] < ov[1] < ov[2] and ov[2] > 1 - 1e-6


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
@pytest.mark.parametrize("maker,nu,ks,sigma", [
    (lambda: tiny_system(10, seed=4), 40, (1, 20, 21), SIGMA),          # dense limit
    (lambda: tiny_hydrocarbon(30, 10, seed=2), 30, (45, 46), 0.05),     # HO, LU of a hydrocarbon cluster
    (lambda: config_c1(), 30, (100, 128, 129), 0.05),
    (lambda: tiny_hydrocarbon(50, 10, seed=4), 160, (85, 86), 0.05),   # nu > 128: the matrix in device memory
])
def test_gpu_eigenstate_matches_oracle(m, maker, nu, ks, sigma):
    t = maker()
    ctx = m.setup_system(t, 0)
    m.marnoldi_solve(ctx, None, nu, 0, t.n_electrons, 0.1)
    for k in ks:
        ek, phi, (lo, hi) = m.marnoldi_eigenstate(ctx, k, sigma)
        ek_o, phi_o, info = oracle.eigenstate(t, k, nu, sigma)
        assert ek == pytest.approx(ek_o, rel=1e-10, abs=1e-12)
        assert lo == pytest.approx(info["eta"][0], rel=1e-10) and hi == pytest.approx(info["eta"][1], rel=1e-10)
        sgn = 1.0 if phi @ phi_o >= 0 else -1.0
        assert np.abs(phi - sgn * phi_o).max() <= 1e-8 * np.abs(phi_o).max()
    # the context's solve is untouched
    E, mu, N = m.marnoldi_energy(ctx)
    assert N == pytest.approx(t.n_electrons, rel=1e-10)
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_eigenstate(ctx, 0, sigma)
    m.marnoldi_destroy(ctx)


@pytest.mark.gpu
def test_gpu_eigenstate_mixed_and_errors(m):
    t = tiny_hydrocarbon(30, 10, seed=2)
    ctx = m.setup_system(t, 1)
    m.marnoldi_solve(ctx, None, 30, 0, t.n_electrons, 0.1)
    ek, phi, _ = m.marnoldi_eigenstate(ctx, 45, 0.05)
    ek_o, phi_o, _ = oracle.eigenstate(t, 45, 30, 0.05)
    assert abs(ek - ek_o) <= 1e-4
    sgn = 1.0 if phi @ phi_o >= 0 else -1.0
    assert np.abs(phi - sgn * phi_o).max() <= 1e-3 * np.abs(phi_o).max()
    m.marnoldi_solve(ctx, t.real_columns()[:10], 30, 0, 0.0, 0.1, mu_fixed=0.0)
    with pytest.raises(m.MarnoldiError):   # needs every real orbital
        m.marnoldi_eigenstate(ctx, 45, 0.05)
    m.marnoldi_destroy(ctx)


@pytest.mark.gpu
def test_gpu_polymer_frontier_state_against_dense(m):
    """The check the paper makes for its poly-fluorene: the eigenstate method's
    state against exact diagonalisation.  On an 8-unit fluorene-like chain the
    lowest unoccupied state (0.22 eV above the level below it, 0.10 eV below
    the next) comes out at nu = 300 with an overlap above 0.97 and its level
    within 3 meV."""
    from tbsynth import polymer_system
    t = polymer_system(8, seed=5)
    ev, V, real, Sr = _exact(t)
    k = int(t.n_electrons // 2) + 1
    ctx = m.setup_system(t, 0)
    m.marnoldi_solve(ctx, None, 300, 0, t.n_electrons, 0.1)
    ek, phi, _ = m.marnoldi_eigenstate(ctx, k, 0.01)
    m.marnoldi_destroy(ctx)
    p = phi[real]
    overlap = abs(p @ Sr @ V[:, k - 1]) / np.sqrt(p @ Sr @ p)
    assert overlap > 0.97
    assert abs(ek - ev[k - 1]) < 3e-3
