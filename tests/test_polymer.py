"""The synthetic fluorene-like polymer chains (tbsynth.polymer): sound geometry
and a valid tight-binding pair, so that they can stand in for the paper's
poly-fluorene (Section 2)."""

import numpy as np
import pytest

from tbsynth import polymer_system
from tbsynth.polymer import polyfluorene
from tbsynth.structures import CARBON, HYDROGEN, min_image


@pytest.mark.parametrize("units,seed", [(1, 0), (6, 3)])
def test_chain_geometry(units, seed):
    s = polyfluorene(units, seed=seed)
    assert s.n_atoms == 69 * units + 2
    sp = s.species
    assert (sp == CARBON).sum() == 29 * units and (sp == HYDROGEN).sum() == 40 * units + 2
    d = np.linalg.norm(min_image(s.positions[None] - s.positions[:, None], s.box), axis=2)
    d += np.eye(s.n_atoms) * 99
    bonded = (d < 1.65).sum(axis=1)
    assert set(bonded[sp == CARBON]) <= {3, 4}      # aromatic or sp3 carbons
    assert np.all(bonded[sp == HYDROGEN] == 1)      # every hydrogen on one carbon
    hh = d[np.ix_(sp == HYDROGEN, sp == HYDROGEN)]
    assert hh.min() > 1.7
    assert d[np.ix_(sp == CARBON, sp == CARBON)].min() >= 1.42 - 1e-9


def test_chain_tight_binding():
    t = polymer_system(4, seed=1)
    assert t.lambda_min_S > 0.05
    assert t.n_electrons == 4 * (29 * 4) + (40 * 4 + 2)
    assert t.real_columns().size == 4 * 29 * 4 + 40 * 4 + 2


# ---------------------------------------------------------------- GPU

KT = 0.1

# (units, seed, precision, nu, region atoms): chains of uneven length with nu from
# {30, 100, 300}, the longest one beyond the global-mode size limit in regional mode
CHAINS = [
    (4, 1, 0, 300, 0),
    (6, 2, 1, 300, 0),
    (9, 3, 1, 100, 0),
    (17, 4, 1, 30, 0),
    (31, 5, 0, 100, 0),
    (52, 6, 0, 30, 0),
    (400, 7, 1, 30, 256),
]


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
def test_gpu_served_chains_match_oracle(m):
    """Polymer chains of 4 to 400 units (278 to 27,602 atoms), nu of 30, 100 and
    300, FP64 and mixed, all submitted at once to a server with three workers.
    Every result: N equal to the electron count; a seeded sample of real columns
    recomputed by the oracle at the served Fermi level (FP64 to 1e-10 of the
    largest entry, mixed within 1e-5 on rho and 1e-4 eV on rho^E)."""
    import oracle
    chains = [(polymer_system(u, seed=s), p, nu, reg) for u, s, p, nu, reg in CHAINS]
    with m.Server(workers=3, hbm_budget_bytes=24 << 30) as srv:
        ids = [srv.submit_system(t, p, nu, reg, t.n_electrons, KT) for t, p, nu, reg in chains]
        got = [srv.wait(i) for i in ids]
    for q, ((t, p, nu, reg), g) in enumerate(zip(chains, got)):
        assert g["N"] == pytest.approx(t.n_electrons, rel=1e-12 if p == 0 else 1e-8)
        real = t.real_columns()
        sample = np.sort(np.random.default_rng(q).choice(real, size=6, replace=False))
        ref = oracle.solve(t, nu=nu, kT=KT, mu_fixed=g["mu"], cols=sample, region_atoms=reg)
        mask = ~np.isnan(ref.rho)
        drho = np.abs(g["rho"][mask] - ref.rho[mask]).max()
        drhoE = np.abs(g["rhoE"][mask] - ref.rhoE[mask]).max()
        print(f"{t.n_block_rows} atoms prec={p} nu={nu} region={reg}: drho={drho:.2e} drhoE={drhoE:.2e}")
        if p == 0:
            assert drho <= 1e-10 * np.abs(ref.rho[mask]).max()
            assert drhoE <= 1e-10 * np.abs(ref.rhoE[mask]).max()
        else:
            assert drho <= 1e-5 and drhoE <= 1e-4
