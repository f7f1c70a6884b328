"""Columns split over ranks with one shared Fermi level (the multi-GPU protocol).

CPU: two gloo ranks, each with the oracle on its spatial domain's columns, run
the shared bisection; the result must equal the single-process oracle solve.
GPU: two contexts on one GPU stand for two ranks (run one after the other in
one process, so no kernel waits on another) and must reproduce one context's
solve of all columns.
"""
import os
import socket

import numpy as np
import pytest

from paper_1307_3218_gb300 import shard
from tbsynth import amorphous_system, config_c1, tiny_hydrocarbon

KT = 0.1
NU = 12


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_domain_columns_partition():
    t = tiny_hydrocarbon(8, 6, seed=2)
    s = t.structure
    real = t.real_columns()
    for world in (1, 2, 3, 5):
        parts = [shard.domain_columns(s.positions, s.box, t.orbital_mask, world, r) for r in range(world)]
        allc = np.concatenate(parts)
        assert np.array_equal(np.sort(allc), np.sort(real))          # every real column once
        assert len(np.unique(allc)) == allc.size
        owner = {}
        for r, p in enumerate(parts):
            for j in p:
                assert owner.setdefault(int(j) // 4, r) == r             # an atom's columns together
    with pytest.raises(ValueError):
        shard.domain_columns(s.positions, s.box, t.orbital_mask, 2, 2)


def test_fermi_bisect_single_rank_matches_oracle():
    import oracle
    t = config_c1()
    c = oracle.columns(t, t.real_columns(), NU)
    eps, w = oracle.valid_levels(c)
    lo, hi = shard.level_bracket(eps.min(), eps.max(), KT, lambda v: v, lambda v: v)
    mu, N, E, _ = shard.fermi_bisect(lambda x: oracle.count(eps, w, x, KT), lo, hi,
                                     float(t.n_electrons), lambda a: a)
    mu0, N0, E0, _ = oracle.bisect(eps, w, float(t.n_electrons), KT)
    assert mu == mu0 and N == N0 and E == E0


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = config_c1()
        s = t.structure
        cols = shard.domain_columns(s.positions, s.box, t.orbital_mask, world, rank)
        c = oracle.columns(t, cols, NU)
        eps, w = oracle.valid_levels(c)
        red_sum, red_min, red_max = shard.torch_reducers()
        lo, hi = shard.level_bracket(eps.min(), eps.max(), KT, red_min, red_max)
        mu, N, E, it = shard.fermi_bisect(lambda x: oracle.count(eps, w, x, KT), lo, hi,
                                          float(t.n_electrons), red_sum)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([mu, N, E, it, cols.size]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_fermi_level(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    assert res[0][:3].tolist() == res[1][:3].tolist()                 # same mu, N, E on every rank
    assert res[0][4] + res[1][4] == config_c1().real_columns().size
    t = config_c1()
    ref = oracle.solve(t, nu=NU, kT=KT)
    mu, N, E = res[0][:3]
    assert abs(N - t.n_electrons) <= 1e-12 * t.n_electrons
    assert abs(E - ref.E_band) <= 1e-10 * abs(ref.E_band)
    assert abs(mu - ref.mu) <= 1e-6


@pytest.mark.gpu
def test_two_contexts_as_ranks_reproduce_one_context():
    import paper_1307_3218_gb300 as m
    t = config_c1()
    s = t.structure
    whole = m.setup_system(t, m.MARNOLDI_FP64)
    m.marnoldi_solve(whole, None, NU, 0, float(t.n_electrons), KT)
    E0, mu0, N0 = m.marnoldi_energy(whole)
    rho0, rhoE0 = m.marnoldi_density(whole)
    ctxs = [m.setup_system(t, m.MARNOLDI_FP64) for _ in range(2)]
    cols = [shard.domain_columns(s.positions, s.box, t.orbital_mask, 2, r) for r in range(2)]
    for ctx, cl in zip(ctxs, cols):
        m.marnoldi_solve(ctx, cl, NU, 0, float(t.n_electrons), KT, mu_fixed=0.0)
    # in-process reductions over the two "ranks"
    lo = min(m.marnoldi_level_range(c)[0] for c in ctxs) - shard.BRACKET_KT * KT
    hi = max(m.marnoldi_level_range(c)[1] for c in ctxs) + shard.BRACKET_KT * KT
    count = lambda x: np.sum([m.marnoldi_fermi_at(c, x, KT) for c in ctxs], axis=0)
    mu, N, E, _ = shard.fermi_bisect(count, lo, hi, float(t.n_electrons), lambda a: a)
    for c in ctxs:
        m.marnoldi_fermi_at(c, mu, KT)
    assert abs(N - N0) <= 1e-10 * N0 and abs(E - E0) <= 1e-10 * abs(E0)
    rho = sum(m.marnoldi_density(c)[0] for c in ctxs)
    rhoE = sum(m.marnoldi_density(c)[1] for c in ctxs)
    assert np.max(np.abs(rho - rho0)) <= 1e-10 * np.max(np.abs(rho0))
    assert np.max(np.abs(rhoE - rhoE0)) <= 1e-10 * np.max(np.abs(rhoE0))
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_fermi_at(ctxs[0], mu, 0.0)
    fresh = m.setup_system(t, m.MARNOLDI_FP64)
    with pytest.raises(m.MarnoldiError):
        m.marnoldi_level_range(fresh)
    for c in ctxs + [whole, fresh]:
        m.marnoldi_destroy(c)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_device_bisection_equals_host_loop(prec):
    """The solve's bisection (a CUDA-graph while loop on the device) takes the
    same steps as the host loop over marnoldi_fermi_at: same bracket, same
    counts, so the same mu, N and E bit for bit."""
    import paper_1307_3218_gb300 as m
    t = amorphous_system(256, seed=2)
    ctx = m.setup_system(t, prec)
    m.marnoldi_solve(ctx, None, NU, 0, float(t.n_electrons), KT)
    E0, mu0, N0 = m.marnoldi_energy(ctx)
    lo, hi = shard.level_bracket(*m.marnoldi_level_range(ctx), KT, lambda v: v, lambda v: v)
    mu, N, E, it = shard.fermi_bisect(lambda x: m.marnoldi_fermi_at(ctx, x, KT), lo, hi,
                                      float(t.n_electrons), lambda a: a)
    assert (mu, N, E) == (mu0, N0, E0)
    assert 10 < it < shard.BISECT_MAXIT
    stats = m.marnoldi_kernel_stats(ctx)
    assert stats["bisect_step"][0] == it + 3   # bracket, N(lo), N(hi), then one per halving
    m.marnoldi_destroy(ctx)
