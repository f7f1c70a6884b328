"""Request server and device-memory footprint (marnoldi_server_*, marnoldi_footprint).

GPU tests: every request's result, computed while other structures of other
sizes, subspace dimensions and precisions run beside it, equals the result of
the same calculation run alone through a context (bit for bit: the kernels of
a request see only its own data and its reductions run in a fixed order), and
one of them also matches the oracle; admission keeps the running footprints
under the budget; the footprint predicts the device memory a run holds, to the
byte.  CPU tests: the footprint's host-side rules and the server's argument
checks.
"""

import numpy as np
import pytest

import oracle
import paper_1307_3218_gb300 as m
from paper_1307_3218_gb300 import build as mbuild
from tbsynth import amorphous_system, config_c1, tiny_hydrocarbon, tiny_system

KT = 0.1


@pytest.fixture(scope="module")
def lib():
    return m.load(mbuild.build())


# ---------------------------------------------------------------- CPU (host logic)

def test_footprint_grows_with_batch_and_clamps(lib):
    t = config_c1()
    ncols = t.real_columns().size
    last = 0
    for B in (1, 2, 7, 64, ncols):
        b, used = m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, None, 0, 30, 0, B)
        assert used == B
        assert b > last
        last = b
    b_all, used = m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, None, 0, 30, 0, 1 << 40)
    assert used == ncols and b_all == last
    # FP32 Krylov vectors halve the per-column vector bytes: mixed needs less
    b_mixed, _ = m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, None, 1, 30, 0, ncols)
    assert b_mixed < b_all


def test_regional_batches_hold_whole_groups_of_four(lib):
    """In regional mode a batch below the column count is rounded down to a
    multiple of 4 (the orbitals of one atom stay together); global mode and
    batches of 1 to 3 columns are not rounded."""
    t = config_c1()
    box = t.structure.box
    ncols = t.real_columns().size
    for B, want in ((1, 1), (3, 3), (7, 4), (65, 64), (ncols - 1, ncols - 4), (ncols, ncols), (1 << 40, ncols)):
        _, used = m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, box, 1, 30, 32, B)
        assert used == want, (B, used)
    _, used = m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, None, 1, 30, 0, 7)
    assert used == 7


def test_footprint_counts_only_real_orbitals(lib):
    t = tiny_hydrocarbon(24, 8, seed=3)
    nreal = t.real_columns().size
    assert nreal < 4 * t.n_block_rows
    _, used = m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, None, 0, 12, 0, 1 << 40)
    assert used == nreal


def test_footprint_rejects_bad_arguments(lib):
    t = config_c1()
    E = m.marnoldi.MARNOLDI_EINVAL
    for kw in (dict(nu=0), dict(nu=321), dict(batch_columns=0), dict(precision=5),
               dict(region_atoms=16, nu=30)):   # regional mode without a box
        with pytest.raises(m.MarnoldiError) as ei:
            args = dict(precision=0, nu=30, region_atoms=0, batch_columns=8)
            args.update(kw)
            m.marnoldi_footprint(t.n_block_rows, t.row_ptr, t.orbital_mask, None, **args)
        assert ei.value.code == E


def test_server_argument_checks(lib):
    import ctypes as C
    out = C.c_void_p()
    assert lib.marnoldi_server_create(C.byref(out), 0, 1 << 30) == m.marnoldi.MARNOLDI_EINVAL
    assert b"workers" in lib.marnoldi_server_last_error()
    assert lib.marnoldi_server_create(C.byref(out), 2, 1024) == m.marnoldi.MARNOLDI_EINVAL
    rid = C.c_int64()
    assert lib.marnoldi_server_submit(None, 1, None, None, None, None, None, None, None, 0, 8, 0,
                                      1.0, 0.1, 0, None, None, C.byref(rid)) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_server_wait(None, 1, 0.0, None, None, None, 0) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_server_stats(None, None) == m.marnoldi.MARNOLDI_EINVAL
    lib.marnoldi_server_destroy(None)


# ---------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def gpu(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib


def _mix():
    """(system, precision, nu, region_atoms) of structures of several sizes."""
    c1 = config_c1()
    a256 = amorphous_system(256, seed=2)
    a512 = amorphous_system(512, seed=1)
    a1024 = amorphous_system(1024, seed=4)
    hc = tiny_hydrocarbon(24, 8, seed=3)
    return [
        (a1024, 1, 30, 0),
        (c1, 0, 30, 0),
        (a512, 1, 30, 0),
        (hc, 0, 12, 0),
        (a256, 0, 60, 0),
        (a1024, 1, 40, 128),
        (c1, 1, 100, 0),
        (tiny_system(40, seed=5), 0, 20, 0),
    ]


def _alone(sysm, prec, nu, region):
    ctx = m.setup_system(sysm, prec)
    m.marnoldi_solve(ctx, None, nu, region, sysm.n_electrons, KT)
    rho, rhoE = m.marnoldi_density(ctx)
    E, mu, N = m.marnoldi_energy(ctx)
    m.marnoldi_destroy(ctx)
    return dict(band_energy=E, mu=mu, N=N, rho=rho, rhoE=rhoE)


@pytest.mark.gpu
def test_results_in_the_mix_equal_results_alone(gpu):
    mix = _mix()
    with m.Server(workers=4, hbm_budget_bytes=8 << 30) as srv:
        ids = [srv.submit_system(s, p, nu, reg, s.n_electrons, KT) for s, p, nu, reg in mix]
        got = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(mix) and st["queued"] == 0 and st["running"] == 0
    assert st["peak_bytes"] <= 8 << 30
    for (s, p, nu, reg), g in zip(mix, got):
        a = _alone(s, p, nu, reg)
        assert g["band_energy"] == a["band_energy"] and g["mu"] == a["mu"] and g["N"] == a["N"], \
            (s.meta, p, nu, reg)
        np.testing.assert_array_equal(g["rho"], a["rho"])
        np.testing.assert_array_equal(g["rhoE"], a["rhoE"])
        assert g["t_submit"] <= g["t_start"] <= g["t_end"]


@pytest.mark.gpu
def test_served_result_matches_oracle(gpu):
    t = config_c1()
    with m.Server(workers=2, hbm_budget_bytes=2 << 30) as srv:
        other = srv.submit_system(amorphous_system(512, seed=1), 1, 30)   # runs beside it
        rid = srv.submit_system(t, 0, 30, 0, t.n_electrons, KT)
        g = srv.wait(rid)
        srv.wait(other)
    ref = oracle.solve(t, nu=30, kT=KT)
    rel = 1e-10
    assert g["N"] == pytest.approx(ref.N, rel=rel)
    assert g["band_energy"] == pytest.approx(ref.E_band, rel=rel)
    mask = ~np.isnan(ref.rho)
    assert np.abs(g["rho"][mask] - ref.rho[mask]).max() <= rel * np.abs(ref.rho[mask]).max()
    assert np.abs(g["rhoE"][mask] - ref.rhoE[mask]).max() <= rel * np.abs(ref.rhoE[mask]).max()


@pytest.mark.gpu
def test_admission_by_footprint(gpu):
    a = amorphous_system(512, seed=1)
    fp, _ = m.marnoldi_footprint(a.n_block_rows, a.row_ptr, a.orbital_mask, None, 1, 30, 0, 1 << 40)
    budget = int(1.5 * fp)   # one request at a time fits, two do not
    with m.Server(workers=4, hbm_budget_bytes=budget) as srv:
        srv.set_group_limit(1)   # requests one by one (grouping is tested below)
        ids = [srv.submit_system(a, 1, 30, 0, a.n_electrons, KT, batch_columns=1 << 40) for _ in range(4)]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
        # a structure larger than the whole budget is refused at submission
        big = amorphous_system(1024, seed=4)
        with pytest.raises(m.MarnoldiError) as ei:
            srv.submit_system(big, 0, 30, batch_columns=1 << 40)
        assert ei.value.code == m.marnoldi.MARNOLDI_ENOMEM
    assert st["peak_running"] == 1 and st["peak_bytes"] == fp
    ends = sorted((r["t_start"], r["t_end"]) for r in res)
    for (s0, e0), (s1, _) in zip(ends, ends[1:]):
        assert s1 >= e0   # admitted one after another
    assert all(r["band_energy"] == res[0]["band_energy"] for r in res)


@pytest.mark.gpu
def test_automatic_batch_fits_the_share(gpu):
    a = amorphous_system(1024, seed=4)
    full, ncols = m.marnoldi_footprint(a.n_block_rows, a.row_ptr, a.orbital_mask, None, 1, 30, 0, 1 << 40)
    budget = full // 2
    with m.Server(workers=3, hbm_budget_bytes=budget) as srv:
        r = srv.wait(srv.submit_system(a, 1, 30, 0, a.n_electrons, KT))
    assert r["batch"] < ncols
    assert r["footprint_bytes"] <= budget // 3
    nxt, _ = m.marnoldi_footprint(a.n_block_rows, a.row_ptr, a.orbital_mask, None, 1, 30, 0, r["batch"] + 1)
    assert nxt > budget // 3
    alone = _alone(a, 1, 30, 0)
    assert r["band_energy"] == alone["band_energy"]
    np.testing.assert_array_equal(r["rho"], alone["rho"])


@pytest.mark.gpu
def test_failed_request_reports_and_server_continues(gpu):
    t = tiny_system(16, seed=0)
    S = t.S.copy()
    rows = np.repeat(np.arange(t.n_block_rows), np.diff(t.row_ptr))
    S[rows != t.col_idx] *= 40.0   # overlaps too large: S indefinite
    with m.Server(workers=2, hbm_budget_bytes=1 << 30) as srv:
        bad = srv.submit(t.n_block_rows, t.row_ptr, t.col_idx, t.H, S, t.orbital_mask, nu=8,
                         electron_count=t.n_electrons, kT=KT)
        good = srv.submit_system(t, 0, 8, 0, t.n_electrons, KT)
        with pytest.raises(m.MarnoldiError) as ei:
            srv.wait(bad)
        assert ei.value.code == m.marnoldi.MARNOLDI_ENOTSPD
        assert "positive definite" in str(ei.value)
        r = srv.wait(good)
        with pytest.raises(m.MarnoldiError):
            srv.wait(good)   # released after its result was read
        # kT and N_e are checked at submission
        for ne, kt in ((0.0, KT), (float("nan"), KT), (t.n_electrons, 0.0), (t.n_electrons, float("inf"))):
            with pytest.raises(m.MarnoldiError) as ei:
                srv.submit_system(t, 0, 8, electron_count=ne, kT=kt)
            assert ei.value.code == m.marnoldi.MARNOLDI_EINVAL and "positive" in str(ei.value)
    assert np.isfinite(r["band_energy"])


@pytest.mark.gpu
@pytest.mark.parametrize("prec,region", [(0, 0), (1, 0), (1, 96)])
def test_footprint_equals_device_peak(gpu, prec, region):
    a = amorphous_system(512, seed=1)
    for B in (37, 1 << 40):
        fp, used = m.marnoldi_footprint(a.n_block_rows, a.row_ptr, a.orbital_mask,
                                        a.structure.box if region else None, prec, 30, region, B)
        ctx = m.setup_system(a, prec)
        m.marnoldi_set_batch(ctx, used)
        m.marnoldi_solve(ctx, None, 30, region, a.n_electrons, KT)
        m.marnoldi_density(ctx)
        cur, peak = m.marnoldi_device_bytes(ctx)
        m.marnoldi_destroy(ctx)
        assert peak == fp, (B, peak, fp)
        assert cur < peak


@pytest.mark.gpu
def test_queued_requests_share_launches(gpu):
    """Requests of one class that wait together run as members of one union."""
    small = [amorphous_system(160, seed=11), amorphous_system(256, seed=12), amorphous_system(200, seed=13),
             amorphous_system(256, seed=14)]                 # M 640..1024: vectors of 1,024 entries
    tiny = [config_c1(seed=1), config_c1(seed=2)]           # M 256
    with m.Server(workers=1, hbm_budget_bytes=8 << 30) as srv:
        big = srv.submit_system(amorphous_system(1024, seed=4), 1, 30)   # keeps the worker busy
        ids = [srv.submit_system(t, 1, 30, 0, t.n_electrons, KT) for t in small + tiny]
        srv.wait(big)
        got = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["groups"] >= 2 and st["largest_group"] >= 3
    starts = {round(g["t_start"], 9) for g in got}
    assert len(starts) <= 3                                   # a few launch groups, not six requests
    for t, g in zip(small + tiny, got):
        a = _alone(t, 1, 30, 0)
        assert (g["band_energy"], g["mu"], g["N"]) == (a["band_energy"], a["mu"], a["N"])
        np.testing.assert_array_equal(g["rho"], a["rho"])
        np.testing.assert_array_equal(g["rhoE"], a["rhoE"])
