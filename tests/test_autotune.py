"""Launch-shape autotuner of the Gram-Schmidt kernel (marnoldi_set_autotune).

The tuned shape only reorders the kernel's partial sums, so a tuned solve
agrees with the oracle at the FP64 tolerance and with the fixed-rule solve to
rounding; a key is tuned once per process, and the cache file carries the
choice to another process.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_1307_3218_gb300 as m
from paper_1307_3218_gb300 import build as mbuild
from tbsynth import amorphous_system

KT = 0.1
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return m.load(mbuild.build())


def test_mode_values(lib):
    assert lib.marnoldi_set_autotune(2) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_set_autotune(-1) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_gs_shape(None, None, None) == m.marnoldi.MARNOLDI_EINVAL


@pytest.fixture(scope="module")
def tuned(lib, tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path_factory.mktemp("tune") / "shapes.txt"
    os.environ["MARNOLDI_TUNE_CACHE"] = str(cache)   # read on the first tuned solve
    m.marnoldi_set_autotune(1)
    yield cache
    m.marnoldi_set_autotune(0)


def _solve(t, prec, nu):
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, nu, 0, t.n_electrons, KT)
    out = dict(zip(("E", "mu", "N"), m.marnoldi_energy(ctx)))
    out["rho"], out["rhoE"] = m.marnoldi_density(ctx)
    out["shape"] = m.marnoldi_gs_shape(ctx)
    out["gs_launches"] = m.marnoldi_kernel_stats(ctx)["gs"][0]
    m.marnoldi_destroy(ctx)
    return out


@pytest.mark.gpu
def test_tuned_solve_matches_oracle(tuned):
    t = amorphous_system(128, seed=3)     # M = 512: shapes 2 x 256 and 1 x 512
    g = _solve(t, 0, 30)
    assert g["shape"] in ((2, 256), (1, 512))
    ref = oracle.solve(t, nu=30, kT=KT)
    rel = 1e-10
    assert g["N"] == pytest.approx(ref.N, rel=rel)
    assert g["E"] == pytest.approx(ref.E_band, rel=rel)
    mask = ~np.isnan(ref.rho)
    assert np.abs(g["rho"][mask] - ref.rho[mask]).max() <= rel * np.abs(ref.rho[mask]).max()
    assert np.abs(g["rhoE"][mask] - ref.rhoE[mask]).max() <= rel * np.abs(ref.rhoE[mask]).max()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_tuned_once_and_agrees_with_fixed_rule(tuned, prec):
    t = amorphous_system(512, seed=1)     # M = 2048: shapes 8 x 256, 4 x 512, 2 x 1024
    first = _solve(t, prec, 30)
    again = _solve(t, prec, 30)
    assert first["gs_launches"] == 30 * (1 + 2 * 3)   # the tuning runs: 3 shapes, 2 runs each
    assert again["gs_launches"] == 30 and again["shape"] == first["shape"]
    np.testing.assert_array_equal(first["rho"], again["rho"])
    m.marnoldi_set_autotune(0)
    fixed = _solve(t, prec, 30)
    m.marnoldi_set_autotune(1)
    assert fixed["shape"] == (8, 256)
    # the same calculation with another order of partial sums
    tol_e = 1e-12 if prec == 0 else 1e-9
    tol_rho = 1e-12 if prec == 0 else 1e-6
    assert abs(first["E"] - fixed["E"]) <= tol_e * abs(fixed["E"])
    assert np.abs(first["rho"] - fixed["rho"]).max() <= tol_rho * np.abs(fixed["rho"]).max()
    lines = [ln.split() for ln in open(tuned).read().splitlines()]
    assert [str(prec), "30", "0", "2048", str(first["shape"][0]), str(first["shape"][1])] in lines


@pytest.mark.gpu
def test_cache_carries_the_choice_to_another_process(tuned):
    t = amorphous_system(512, seed=1)
    want = _solve(t, 1, 30)["shape"]
    code = (
        "import json, paper_1307_3218_gb300 as m\n"
        "from tbsynth import amorphous_system\n"
        "t = amorphous_system(512, seed=1)\n"
        "ctx = m.setup_system(t, 1)\n"
        "m.marnoldi_solve(ctx, None, 30, 0, t.n_electrons, 0.1)\n"
        "print(json.dumps([m.marnoldi_gs_shape(ctx), m.marnoldi_kernel_stats(ctx)['gs'][0]]))\n"
    )
    env = dict(os.environ, MARNOLDI_AUTOTUNE="1", MARNOLDI_TUNE_CACHE=str(tuned), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    shape, launches = json.loads(out.stdout.strip().splitlines()[-1])
    assert tuple(shape) == want and launches == 30   # no tuning runs
