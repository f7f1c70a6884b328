"""tbsynth.amorphous_carbon takes its candidates a batch at a time; it must
accept exactly the atoms that testing one candidate at a time accepts.  The
reference below is that one-at-a-time random sequential addition, written out
(a cell dictionary and Python loops), on the same seeded candidate stream."""

import numpy as np
import pytest

from tbsynth.structures import amorphous_carbon, number_density


def _one_at_a_time(n_atoms, density_gcc=3.0, d_min=1.3, seed=0):
    L = (n_atoms / number_density(density_gcc)) ** (1.0 / 3.0)
    nc = max(1, int(L // d_min))
    cs = L / nc
    rng = np.random.default_rng(seed)
    cells = {}
    out = []
    d2min = d_min * d_min
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    batch = rng.random((4096, 3)) * L
    bi = 0
    while len(out) < n_atoms:
        if bi == batch.shape[0]:
            batch = rng.random((4096, 3)) * L
            bi = 0
        x, y, z = batch[bi]
        bi += 1
        cx, cy, cz = int(x / cs) % nc, int(y / cs) % nc, int(z / cs) % nc
        ok = True
        for a, b, c in offs:
            for k in cells.get(((cx + a) % nc, (cy + b) % nc, (cz + c) % nc), ()):
                dx, dy, dz = out[k][0] - x, out[k][1] - y, out[k][2] - z
                dx -= L * round(dx / L)
                dy -= L * round(dy / L)
                dz -= L * round(dz / L)
                if dx * dx + dy * dy + dz * dz < d2min:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            cells.setdefault((cx, cy, cz), []).append(len(out))
            out.append((x, y, z))
    return np.array(out), L


@pytest.mark.parametrize("n,seed", [(20, 0), (64, 2), (512, 1), (4096, 0), (12000, 5)])
def test_batched_packing_equals_one_at_a_time(n, seed):
    want, L = _one_at_a_time(n, seed=seed)
    got = amorphous_carbon(n, seed=seed, sort=False)
    assert got.box[0] == L
    np.testing.assert_array_equal(got.positions, want)
