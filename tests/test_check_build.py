"""The index-check build of the library (-DMARNOLDI_CHECK, the build script's
"check" variant): its kernels test every index they take from data before using
it, record a failure instead of trapping, and skip the access.  On diamond-64
(global and regional mode, FP64 and mixed precision) no check fails and the
results match the oracle.  The solves run in a child process that loads the
check build through MARNOLDI_LIB."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from tbsynth import config_c1

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KT = 0.1

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_1307_3218_gb300 as m
from tbsynth import config_c1, amorphous_system
m.load()
out = {"compiled": m.marnoldi_check_status()[0], "runs": []}
for name, t, prec, region in [("c1", config_c1(seed=0), 0, 0), ("c1", config_c1(seed=0), 1, 0),
                              ("c1", config_c1(seed=0), 0, 24), ("a300", amorphous_system(300, seed=5), 1, 0)]:
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, 30, region, t.n_electrons, 0.1)
    rho, rhoE = m.marnoldi_density(ctx)
    E, mu, N = m.marnoldi_energy(ctx)
    m.marnoldi_destroy(ctx)
    comp, site, idx = m.marnoldi_check_status()
    out["runs"].append(dict(name=name, prec=prec, region=region, E=E, mu=mu, N=N, site=site, index=idx,
                            rho=float(np.abs(rho).sum())))
print(json.dumps(out))
"""


def test_default_build_reports_no_checks():
    import paper_1307_3218_gb300 as m
    m.load()
    compiled, site, index = m.marnoldi_check_status()
    assert not compiled and site == 0 and index == 0


@pytest.mark.gpu
def test_check_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3218_gb300 import build as b
    path = b.build(variant="check")
    env = dict(os.environ, MARNOLDI_LIB=path)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["compiled"] is True
    c1 = config_c1(seed=0)
    ref = oracle.solve(c1, nu=30, kT=KT)
    ref_reg = oracle.solve(c1, nu=30, kT=KT, region_atoms=24)
    for run in out["runs"]:
        assert run["site"] == 0, run
        if run["name"] != "c1":
            assert run["N"] == pytest.approx(300 * 4, rel=1e-8)
            continue
        want = ref_reg if run["region"] else ref
        if run["prec"] == 0:
            assert run["E"] == pytest.approx(want.E_band, rel=1e-10)
        else:
            assert abs(run["E"] - want.E_band) / c1.n_block_rows <= 1e-6
