"""The paper-scale structure on one GPU: amorphous carbon of 1,048,576 atoms
(M = 4,194,304, about 11.8 million 4x4 blocks) in regional mode with 256-atom
regions (Section 1's order-N form of the method).

Two launch configurations: every column at nu = 30 in mixed precision with the
Fermi level by bisection, and one batch of the first 65,536 columns at nu = 100
in mixed precision and in FP64 at a fixed Fermi level.  The oracle recomputes
seeded samples of columns one by one (regional mode) at the GPU's Fermi level;
FP64 agrees to 1e-10 of the largest entry, mixed precision within 1e-5 on rho
and 1e-4 eV on rho^E.
"""

import numpy as np
import pytest

import oracle
from tbsynth import amorphous_system

pytestmark = pytest.mark.gpu

KT = 0.1
N_ATOMS = 1 << 20
N_REG = 256
BATCH = 65536


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_3218_gb300 as mm
    from paper_1307_3218_gb300 import build as b
    mm.load(b.build())
    return mm


@pytest.fixture(scope="module")
def big():
    return amorphous_system(N_ATOMS, seed=0)


def _at_rows(t, vals, c):
    """The GPU's [nnzb, 4, 4] values on the oracle's pattern rows of its columns."""
    out = []
    for q, j in enumerate(c.cols):
        J, b = int(j) // 4, int(j) % 4
        rows = c.rows[c.row_off[q]:c.row_off[q + 1]]
        I, a = rows // 4, rows % 4
        k = np.array([int(t.row_ptr[i]) + int(np.searchsorted(t.col_idx[t.row_ptr[i]:t.row_ptr[i + 1]], J))
                      for i in I])
        assert np.all(t.col_idx[k] == J)
        out.append(vals[k, a, b])
    return np.concatenate(out)


def _compare(t, g_rho, g_rhoE, cols, nu, mu, fp64):
    c = oracle.regional_columns(t, cols, nu, N_REG)
    rr, rre = oracle.density_rows(c, mu, KT)
    drho = np.abs(_at_rows(t, g_rho, c) - rr).max()
    drhoE = np.abs(_at_rows(t, g_rhoE, c) - rre).max()
    print(f"{t.n_block_rows} atoms nu={nu} fp64={fp64}: drho={drho:.2e} drhoE={drhoE:.2e}")
    if fp64:
        assert drho <= 1e-10 * np.abs(rr).max()
        assert drhoE <= 1e-10 * np.abs(rre).max()
    else:
        assert drho <= 1e-5 and drhoE <= 1e-4


def test_every_column_nu30_mixed(m, big):
    t = big
    assert t.M == 4 * N_ATOMS
    ctx = m.setup_system(t, 1)
    m.marnoldi_solve(ctx, None, 30, N_REG, float(t.n_electrons), KT)
    E, mu, N = m.marnoldi_energy(ctx)
    rho, rhoE = m.marnoldi_density(ctx)
    m.marnoldi_destroy(ctx)
    assert N == pytest.approx(t.n_electrons, rel=1e-8)
    sample = np.sort(np.random.default_rng(3).choice(t.M, size=8, replace=False))
    _compare(t, rho, rhoE, sample, 30, mu, False)


@pytest.mark.parametrize("prec", [1, 0])
def test_batch_of_65536_columns_nu100(m, big, prec):
    t = big
    mu = 3.62   # near the structure's Fermi level at nu = 30; the oracle uses the same value
    ctx = m.setup_system(t, prec)
    cols = np.arange(BATCH, dtype=np.int64)
    m.marnoldi_solve(ctx, cols, 100, N_REG, 0.0, KT, mu_fixed=mu)
    rho, rhoE = m.marnoldi_density(ctx)
    m.marnoldi_destroy(ctx)
    sample = np.sort(np.random.default_rng(4 + prec).choice(BATCH, size=6, replace=False))
    _compare(t, rho, rhoE, sample, 100, mu, prec == 0)
