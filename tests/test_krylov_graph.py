"""The Krylov build as one CUDA graph (marnoldi_set_krylov_graph).

The graph holds the same kernels with the same arguments in the same order as
the direct launches, so every result must equal theirs bit for bit: FP64 and
mixed, global and regional, several batches per solve (the executable graph
updated in place from batch to batch), a second solve on the same context, a
change of nu (a new topology, so a new instantiation), members, and requests
of the request server whose contexts take the default from
MARNOLDI_KRYLOV_GRAPH.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

from tbsynth import amorphous_system, config_c1

KT = 0.1
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_graph_entry_points_check_arguments():
    import paper_1307_3218_gb300 as m
    from paper_1307_3218_gb300 import build as b
    if not os.path.exists(b.lib_path()):
        pytest.skip("library not built")
    lib = m.load()
    assert lib.marnoldi_set_krylov_graph(None, 1) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_krylov_graph_launches(None, None) == m.marnoldi.MARNOLDI_EINVAL


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_3218_gb300 as mm
    from paper_1307_3218_gb300 import build as b
    mm.load(b.build())
    return mm


def _solve(m, ctx, t, nu, region=0):
    m.marnoldi_solve(ctx, None, nu, region, t.n_electrons, KT)
    rho, rhoE = m.marnoldi_density(ctx)
    E, mu, N = m.marnoldi_energy(ctx)
    nue, eps, w = m.marnoldi_column_stats(ctx)
    return dict(rho=rho, rhoE=rhoE, E=E, mu=mu, N=N, nu_eff=nue, eps=eps, w=w)


def _same(a, b):
    for k in a:
        np.testing.assert_array_equal(np.asarray(a[k]), np.asarray(b[k]), err_msg=k)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("region", [0, 32])
def test_graph_equals_direct_launches(m, prec, region):
    t = amorphous_system(512, seed=4)
    direct = m.setup_system(t, prec)
    m.marnoldi_set_krylov_graph(direct, False)
    m.marnoldi_set_batch(direct, 600)     # several batches, the last one ragged
    ref = _solve(m, direct, t, 30, region)
    ref40 = _solve(m, direct, t, 40, region)
    m.marnoldi_destroy(direct)

    g = m.setup_system(t, prec)
    m.marnoldi_set_krylov_graph(g, True)
    m.marnoldi_set_batch(g, 600)
    first = _solve(m, g, t, 30, region)
    nbatch = m.marnoldi_krylov_graph_launches(g)
    assert nbatch >= 3
    again = _solve(m, g, t, 30, region)     # the kept graph, updated in place
    other = _solve(m, g, t, 40, region)     # another nu: another topology
    assert m.marnoldi_krylov_graph_launches(g) == 3 * nbatch
    m.marnoldi_destroy(g)
    _same(ref, first)
    _same(ref, again)
    _same(ref40, other)


@pytest.mark.gpu
def test_graph_is_not_used_while_profiling(m):
    t = config_c1(seed=0)
    ctx = m.setup_system(t, 1)
    m.marnoldi_set_krylov_graph(ctx, True)
    m.marnoldi_set_profiling(ctx, True)
    m.marnoldi_kernel_stats(ctx, reset=True)
    _solve(m, ctx, t, 30)
    assert m.marnoldi_krylov_graph_launches(ctx) == 0
    assert m.marnoldi_kernel_stats(ctx)["gs"][0] == 30
    m.marnoldi_set_profiling(ctx, False)
    _solve(m, ctx, t, 30)
    assert m.marnoldi_krylov_graph_launches(ctx) == 1
    m.marnoldi_destroy(ctx)


@pytest.mark.gpu
def test_graph_with_members(m):
    systems = [config_c1(seed=s) for s in range(3)]
    n, rp, ci, H, S, mask, offs, _ = m.union_of(systems)
    out = []
    for graph in (False, True):
        ctx = m.marnoldi_setup(n, rp, ci, H, S, mask, precision=1)
        m.marnoldi_set_krylov_graph(ctx, graph)
        m.marnoldi_set_members(ctx, offs, [t.n_electrons for t in systems])
        m.marnoldi_solve(ctx, None, 30, 0, 0.0, KT)
        rho, rhoE = m.marnoldi_density(ctx)
        out.append((rho, rhoE, [m.marnoldi_member_energy(ctx, q) for q in range(3)],
                    m.marnoldi_krylov_graph_launches(ctx)))
        m.marnoldi_destroy(ctx)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    assert out[0][3] == 0 and out[1][3] == 1


SERVER_CHILD = """
import json, sys, numpy as np, paper_1307_3218_gb300 as m
from tbsynth import config_c1
cells = [config_c1(seed=s) for s in range(4)]
with m.Server(workers=2, hbm_budget_bytes=8 << 30) as srv:
    ids = [srv.submit_system(c, 1, 30, 0, c.n_electrons, 0.1) for c in cells]
    res = [srv.wait(i) for i in ids]
np.savez(sys.argv[1], rho=np.concatenate([r["rho"].ravel() for r in res]),
         rhoE=np.concatenate([r["rhoE"].ravel() for r in res]),
         E=np.array([r["band_energy"] for r in res]), mu=np.array([r["mu"] for r in res]))
"""


@pytest.mark.gpu
def test_server_requests_with_graphs(m, tmp_path):
    got = []
    for flag in ("0", "1"):
        out = tmp_path / f"s{flag}.npz"
        env = dict(os.environ, MARNOLDI_KRYLOV_GRAPH=flag, PYTHONPATH=ROOT)
        r = subprocess.run([sys.executable, "-c", SERVER_CHILD, str(out)], env=env, cwd=ROOT,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        got.append(np.load(out))
    for k in ("rho", "rhoE", "E", "mu"):
        np.testing.assert_array_equal(got[0][k], got[1][k], err_msg=k)
