"""Several structures in one context (marnoldi_set_members): one launch per step
covers the columns of every member, each member keeps its own Fermi level.

A member whose padded vector length equals the largest member's gets the
results of solving it alone, bit for bit (same tile order, same launch shape,
same reductions over its own columns); other members agree to rounding; the
union's host-side checks reject what would mix members.
"""

import numpy as np
import pytest

from tbsynth import amorphous_system, build_tb_derivatives, config_c1, tiny_hydrocarbon

pytestmark = pytest.mark.gpu
KT = 0.1


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_3218_gb300 as mm
    from paper_1307_3218_gb300 import build as b
    mm.load(b.build())
    return mm


def _alone(m, t, prec, nu):
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, nu, 0, t.n_electrons, KT)
    out = dict(zip(("E", "mu", "N"), m.marnoldi_energy(ctx)))
    out["rho"], out["rhoE"] = m.marnoldi_density(ctx)
    out["shape"] = m.marnoldi_gs_shape(ctx)
    m.marnoldi_destroy(ctx)
    return out


def _union(m, systems, prec, nu):
    n, rp, ci, H, S, mask, offs, boffs = m.union_of(systems)
    ctx = m.marnoldi_setup(n, rp, ci, H, S, mask, precision=prec)
    m.marnoldi_set_members(ctx, offs, [t.n_electrons for t in systems])
    m.marnoldi_solve(ctx, None, nu, 0, 0.0, KT)
    rho, rhoE = m.marnoldi_density(ctx)
    out = []
    for q, t in enumerate(systems):
        E, mu, N = m.marnoldi_member_energy(ctx, q)
        sl = slice(boffs[q], boffs[q] + t.nnzb)
        out.append(dict(E=E, mu=mu, N=N, rho=rho[sl], rhoE=rhoE[sl]))
    return ctx, out, boffs


@pytest.mark.parametrize("prec", [0, 1])
def test_same_class_members_equal_alone_bitwise(m, prec):
    systems = [amorphous_system(160, seed=11), amorphous_system(256, seed=12), amorphous_system(200, seed=13)]
    ctx, got, _ = _union(m, systems, prec, 30)
    m.marnoldi_destroy(ctx)
    for t, g in zip(systems, got):
        a = _alone(m, t, prec, 30)
        assert a["shape"] == (4, 256)   # M = 640 .. 1,024: the same padded length as the union's
        assert (g["E"], g["mu"], g["N"]) == (a["E"], a["mu"], a["N"])
        np.testing.assert_array_equal(g["rho"], a["rho"])
        np.testing.assert_array_equal(g["rhoE"], a["rhoE"])


def test_mixed_classes_agree_to_rounding(m):
    systems = [config_c1(), tiny_hydrocarbon(30, 10, seed=2), amorphous_system(256, seed=12)]
    ctx, got, _ = _union(m, systems, 0, 24)
    E_tot, _, N_tot = m.marnoldi_energy(ctx)
    m.marnoldi_destroy(ctx)
    assert E_tot == pytest.approx(sum(g["E"] for g in got), rel=1e-14)
    assert N_tot == pytest.approx(sum(g["N"] for g in got), rel=1e-14)
    for t, g in zip(systems, got):
        a = _alone(m, t, 0, 24)
        assert g["E"] == pytest.approx(a["E"], rel=1e-10)
        assert g["N"] == pytest.approx(a["N"], rel=1e-10)
        assert np.abs(g["rho"] - a["rho"]).max() <= 1e-10 * np.abs(a["rho"]).max()


def test_member_forces(m):
    systems = [amorphous_system(150, seed=11), config_c1(seed=1)]   # 2 padding atoms after the first
    ctx, _, _ = _union(m, systems, 0, 20)
    n, rp, ci, H, S, mask, offs, boffs = m.union_of(systems)
    dH = np.zeros((3, len(ci), 4, 4))
    dS = np.zeros_like(dH)
    for q, t in enumerate(systems):
        dh, ds = build_tb_derivatives(t)
        dH[:, boffs[q]:boffs[q] + t.nnzb] = dh
        dS[:, boffs[q]:boffs[q] + t.nnzb] = ds
    F = m.marnoldi_forces(ctx, dH, dS)
    m.marnoldi_destroy(ctx)
    for q, t in enumerate(systems):
        c = m.setup_system(t, 0)
        m.marnoldi_solve(c, None, 20, 0, t.n_electrons, KT)
        Fa = m.marnoldi_forces(c, *build_tb_derivatives(t))
        m.marnoldi_destroy(c)
        Fq = F[offs[q]:offs[q] + t.n_block_rows]
        assert np.abs(Fq - Fa).max() <= 1e-9 * np.abs(Fa).max()
    assert np.abs(F[offs[0] + systems[0].n_block_rows:offs[1]]).max() == 0.0   # padding atoms


def test_member_checks(m):
    systems = [config_c1(), amorphous_system(160, seed=11)]
    n, rp, ci, H, S, mask, offs, boffs = m.union_of(systems)
    ctx = m.marnoldi_setup(n, rp, ci, H, S, mask, precision=0)
    ne = [t.n_electrons for t in systems]
    E = m.marnoldi.MARNOLDI_EINVAL
    for bad_offs in ([0, 60, n], [0, 64, n - 1], [0, n, n]):
        with pytest.raises(m.MarnoldiError) as ei:
            m.marnoldi_set_members(ctx, bad_offs, ne)
        assert ei.value.code == E
    with pytest.raises(m.MarnoldiError) as ei:   # block (0, 64) would couple the members
        m.marnoldi_set_members(ctx, [0, 32, n], ne)
    assert ei.value.code == E and "couples" in str(ei.value)
    m.marnoldi_set_members(ctx, offs, ne)
    for kw in (dict(columns=[0, 1, 2]), dict(region_atoms=16), dict(mu_fixed=0.0), dict(nu=260)):
        args = dict(columns=None, nu=20, region_atoms=0, electron_count=0.0, kT=KT, mu_fixed=None)
        args.update(kw)
        with pytest.raises(m.MarnoldiError) as ei:
            m.marnoldi_solve(ctx, **args)
        assert ei.value.code == E
    m.marnoldi_solve(ctx, None, 20, 0, 0.0, KT)
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_level_range(ctx)
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_member_energy(ctx, 2)
    m.marnoldi_set_members(ctx, [], [])           # back to one structure
    m.marnoldi_solve(ctx, None, 20, 0, float(sum(ne)), KT)
    m.marnoldi_destroy(ctx)


def _alone_kT(m, t, prec, nu, kT):
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, nu, 0, t.n_electrons, kT)
    out = dict(zip(("E", "mu", "N"), m.marnoldi_energy(ctx)))
    out["rho"], out["rhoE"] = m.marnoldi_density(ctx)
    m.marnoldi_destroy(ctx)
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_members_with_their_own_temperatures(m, prec):
    """kT enters only each member's Fermi step: members of the same padded length solved at
    kT 0.05, 0.1 and 0.2 in one union equal their solves alone, bit for bit."""
    systems = [amorphous_system(160, seed=11), amorphous_system(256, seed=12), amorphous_system(200, seed=13)]
    temps = [0.05, 0.2, 0.1]
    n, rp, ci, H, S, mask, offs, boffs = m.union_of(systems)
    ctx = m.marnoldi_setup(n, rp, ci, H, S, mask, precision=prec)
    m.marnoldi_set_members(ctx, offs, [t.n_electrons for t in systems])
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_set_member_temperatures(ctx, temps[:2])          # one per member
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_set_member_temperatures(ctx, [0.05, -0.1, 0.1])  # positive
    m.marnoldi_set_member_temperatures(ctx, temps)
    m.marnoldi_solve(ctx, None, 30, 0, 0.0, 0.1)
    rho, rhoE = m.marnoldi_density(ctx)
    for q, (t, kT) in enumerate(zip(systems, temps)):
        E, mu, N = m.marnoldi_member_energy(ctx, q)
        a = _alone_kT(m, t, prec, 30, kT)
        assert (E, mu, N) == (a["E"], a["mu"], a["N"])
        sl = slice(boffs[q], boffs[q] + t.nnzb)
        np.testing.assert_array_equal(rho[sl], a["rho"])
        np.testing.assert_array_equal(rhoE[sl], a["rhoE"])
    m.marnoldi_destroy(ctx)
