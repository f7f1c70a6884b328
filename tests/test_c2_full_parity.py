"""The benchmark workload against the full oracle: every column of 4,096-atom
amorphous carbon (M = 16,384) at nu = 30, FP64 and mixed precision, each side
with its own Fermi level by bisection; mixed precision at nu = 100 on a seeded
sample of its columns, column by column; and mixed precision at nu = 100
against the full oracle on a 512-atom structure.

The oracle runs once per module over all 16,384 columns (about 85 s on 16 host
cores).  Tolerances: FP64 1e-10 relative on E_band and N and 1e-10 of the
largest entry on every rho and rho^E entry; mixed |dE_band| per atom <= 1e-6 eV,
|dN| <= 1e-8 N_e, max |d rho| <= 1e-5, max |d rho^E| <= 1e-4 eV.
"""

import numpy as np
import pytest

import oracle
from tbsynth import config_c2

pytestmark = pytest.mark.gpu

KT = 0.1


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_3218_gb300 as mm
    from paper_1307_3218_gb300 import build as b
    b.build()
    mm.load()
    return mm


@pytest.fixture(scope="module")
def c2():
    return config_c2(seed=0)


@pytest.fixture(scope="module")
def ref30(c2):
    # every real column, the oracle's own bisection for N_e = 4 per atom
    return oracle.solve(c2, nu=30, kT=KT)


def gpu_full(m, t, nu, prec):
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, nu, 0, t.n_electrons, KT)
    rho, rhoE = m.marnoldi_density(ctx)
    E, mu, N = m.marnoldi_energy(ctx)
    nue, eps, w = m.marnoldi_column_stats(ctx)
    m.marnoldi_destroy(ctx)
    return dict(rho=rho, rhoE=rhoE, E=E, mu=mu, N=N, nu_eff=nue, eps=eps, w=w)


@pytest.mark.parametrize("prec", [0, 1])
def test_c2_every_column_nu30(m, c2, ref30, prec):
    g = gpu_full(m, c2, 30, prec)
    n_atoms = c2.n_block_rows
    assert not np.isnan(ref30.rho).any()       # every block's column was solved
    dE_atom = abs(g["E"] - ref30.E_band) / n_atoms
    dN = abs(g["N"] - ref30.N)
    drho = float(np.abs(g["rho"] - ref30.rho).max())
    drhoE = float(np.abs(g["rhoE"] - ref30.rhoE).max())
    print(f"C2 nu=30 prec={prec} all {c2.M} columns: dE/atom={dE_atom:.3e} eV dN={dN:.3e} "
          f"drho={drho:.3e} drhoE={drhoE:.3e} eV dmu={abs(g['mu'] - ref30.mu):.3e} eV")
    if prec == 0:
        assert g["E"] == pytest.approx(ref30.E_band, rel=1e-10)
        assert g["N"] == pytest.approx(ref30.N, rel=1e-10)
        assert drho <= 1e-10 * np.abs(ref30.rho).max()
        assert drhoE <= 1e-10 * np.abs(ref30.rhoE).max()
        np.testing.assert_array_equal(g["nu_eff"], ref30.cols.nu_eff)
    else:
        assert dE_atom <= 1e-6
        assert dN <= 1e-8 * c2.n_electrons
        assert drho <= 1e-5
        assert drhoE <= 1e-4


SHAPE_CHILD = """
import sys, numpy as np, paper_1307_3218_gb300 as m
from tbsynth import config_c2
t = config_c2(seed=0)
ctx = m.setup_system(t, 1)
m.marnoldi_solve(ctx, None, 30, 0, t.n_electrons, %r)
rho, rhoE = m.marnoldi_density(ctx)
E, mu, N = m.marnoldi_energy(ctx)
np.savez(sys.argv[1], rho=rho, rhoE=rhoE, E=E, mu=mu, N=N, shape=np.array(m.marnoldi_gs_shape(ctx)))
""" % KT


@pytest.mark.parametrize("shape", [(32, 544), (16, 1024)])
def test_c2_every_column_nu30_other_shapes(m, c2, ref30, shape, tmp_path):
    """The other Gram-Schmidt launch shapes of 16,384-entry FP32 vectors (the streamed kernel with
    512 consumer threads and one CTA per SM, and the 1,024-thread kernel without a ring; the
    default is the streamed kernel with 256 consumer threads and two CTAs per SM), chosen through
    a tune cache in a child process, against the full oracle at the mixed tolerances."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "shapes.txt"
    cache.write_text(f"1 30 0 16384 {shape[0]} {shape[1]}\n")
    out = tmp_path / "g.npz"
    env = dict(os.environ, MARNOLDI_AUTOTUNE="1", MARNOLDI_TUNE_CACHE=str(cache), PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", SHAPE_CHILD, str(out)], env=env, cwd=root, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    g = np.load(out)
    assert tuple(g["shape"]) == shape
    dE_atom = abs(float(g["E"]) - ref30.E_band) / c2.n_block_rows
    drho = float(np.abs(g["rho"] - ref30.rho).max())
    drhoE = float(np.abs(g["rhoE"] - ref30.rhoE).max())
    print(f"C2 nu=30 mixed shape={shape}: dE/atom={dE_atom:.3e} eV drho={drho:.3e} drhoE={drhoE:.3e} eV")
    assert dE_atom <= 1e-6
    assert abs(float(g["N"]) - ref30.N) <= 1e-8 * c2.n_electrons
    assert drho <= 1e-5
    assert drhoE <= 1e-4


def column_band_energy(eps, w, nu_eff, mu):
    """Each column's share of E_band: sum_a 2 f((eps_a - mu) / kT) eps_a w_a over its valid levels."""
    valid = np.arange(eps.shape[1])[None, :] < nu_eff[:, None]
    f2 = 2.0 * oracle._fermi_np((eps - mu) / KT)
    return np.sum(np.where(valid, f2 * eps * w, 0.0), axis=1)


def test_c2_mixed_nu100_sampled(m, c2):
    """nu = 100 in mixed precision, every column on the GPU, 48 seeded columns recomputed by the
    oracle at the GPU's mu.  Each column's share of E_band, e_j = sum_a 2 f eps_a w_a, equals
    (S rho^E)_jj (the pattern trace of its rho^E column), so the rho^E tolerance bounds its error
    by ||S_j,:||_1 x 1e-4 eV; the sample's signed errors also estimate the error of the total."""
    g = gpu_full(m, c2, 100, 1)
    assert g["N"] == pytest.approx(c2.n_electrons, rel=1e-8)
    sample = np.sort(np.random.default_rng(23).choice(c2.M, size=48, replace=False))
    ref = oracle.solve(c2, nu=100, kT=KT, mu_fixed=g["mu"], cols=sample)
    mask = ~np.isnan(ref.rho)
    drho = float(np.abs(g["rho"][mask] - ref.rho[mask]).max())
    drhoE = float(np.abs(g["rhoE"][mask] - ref.rhoE[mask]).max())
    eg = column_band_energy(g["eps"][sample], g["w"][sample], g["nu_eff"][sample], g["mu"])
    eo = column_band_energy(ref.cols.eps, ref.cols.w, ref.cols.nu_eff, g["mu"])
    de = eg - eo
    s_row = np.array([np.abs(c2.S[c2.row_ptr[j // 4]:c2.row_ptr[j // 4 + 1], j % 4, :]).sum() for j in sample])
    # the total's error per atom, extrapolated from the sample (M columns, 4 per atom)
    est_atom = float(de.mean()) * c2.M / c2.n_block_rows
    print(f"C2 nu=100 mixed, 48 columns: drho={drho:.3e} drhoE={drhoE:.3e} eV "
          f"max|d e_j|={np.abs(de).max():.3e} eV (bound {1e-4 * s_row.min():.2e}), "
          f"total per atom estimated {est_atom:.2e} eV")
    assert drho <= 1e-5
    assert drhoE <= 1e-4
    assert np.all(np.abs(de) <= 1e-4 * s_row)


@pytest.fixture(scope="module")
def a512():
    from tbsynth import amorphous_system
    t = amorphous_system(512, seed=2)
    return t, oracle.solve(t, nu=100, kT=KT)     # every column, about 18 s on 8 host cores


@pytest.mark.parametrize("prec", [0, 1])
def test_nu100_every_column_512_atoms(m, a512, prec):
    """nu = 100 against the full oracle on 512-atom amorphous carbon (global mode, every column,
    each side with its own bisection)."""
    t, ref = a512
    g = gpu_full(m, t, 100, prec)
    dE_atom = abs(g["E"] - ref.E_band) / t.n_block_rows
    drho = float(np.abs(g["rho"] - ref.rho).max())
    drhoE = float(np.abs(g["rhoE"] - ref.rhoE).max())
    print(f"512 atoms nu=100 prec={prec}, every column: dE/atom={dE_atom:.3e} eV drho={drho:.3e} "
          f"drhoE={drhoE:.3e} eV")
    if prec == 0:
        assert g["E"] == pytest.approx(ref.E_band, rel=1e-10)
        assert g["N"] == pytest.approx(ref.N, rel=1e-10)
        assert drho <= 1e-10 * np.abs(ref.rho).max()
        assert drhoE <= 1e-10 * np.abs(ref.rhoE).max()
    else:
        assert dE_atom <= 1e-6
        assert abs(g["N"] - ref.N) <= 1e-8 * t.n_electrons
        assert drho <= 1e-5
        assert drhoE <= 1e-4
