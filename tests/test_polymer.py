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
