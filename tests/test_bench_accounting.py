"""The bench's roofline accounting, recomputed independently on a small case.

bench.support_counts (tiles of 8 atoms within L pattern hops of each column's
atom, by scipy's shortest paths) and bench.gs_algorithmic_support (the bytes
the Gram-Schmidt steps must move over the vectors' supports, summed with
aggregated counts) feed the `achieved` figure of the bench's roofline.  Here
a breadth-first search written out in Python and per-column, per-step loops
give the same numbers exactly.
"""

from collections import deque

import numpy as np
import pytest

import bench
from tbsynth import amorphous_system, tiny_hydrocarbon


def _hops(t, start):
    dist = np.full(t.n_block_rows, -1, dtype=np.int64)
    dist[start] = 0
    q = deque([start])
    while q:
        a = q.popleft()
        for k in range(t.row_ptr[a], t.row_ptr[a + 1]):
            b = int(t.col_idx[k])
            if dist[b] < 0:
                dist[b] = dist[a] + 1
                q.append(b)
    return dist


def _tile_counts(t, atom, nu, m_pad):
    d = _hops(t, atom)
    ntile = m_pad // 32
    out = np.zeros(nu + 2, dtype=np.int64)
    for tile in range(ntile):
        members = [d[a] for a in range(8 * tile, min(8 * tile + 8, t.n_block_rows)) if d[a] >= 0]
        if not members:
            continue
        h = min(members)
        for L in range(nu + 2):
            out[L] += h <= L
    return out


def _gs_bytes(tc, nu, vbytes):
    total = 0
    for c in range(tc.shape[0]):
        E = 32 * tc[c]
        for n in range(nu):
            total += (2 if vbytes == 4 else 1) * E[n + 1]   # u (and its lo word)
            total += E[n]                                    # w_n
            for i in range(n + 1):
                total += 2 * E[i + 1]                        # w_i and S w_i
            if n + 1 < nu:
                for i in range(n + 1):
                    total += E[i + 1]                        # w_i again, for the subtraction
                total += E[n + 1]                            # the new w
    return total * vbytes


@pytest.mark.parametrize("maker,nu", [(lambda: amorphous_system(64, seed=2), 6),
                                      (lambda: tiny_hydrocarbon(20, 8, seed=1), 9)])
def test_support_counts_and_gs_bytes(maker, nu):
    t = maker()
    cols = t.real_columns()
    m_pad = bench.column_m_pad(t.M)
    tc = bench.support_counts(t, cols, nu, m_pad)
    want = np.array([_tile_counts(t, int(j) // 4, nu, m_pad) for j in cols])
    np.testing.assert_array_equal(tc, want)
    for vbytes in (4, 8):
        got, _ = bench.gs_algorithmic_support(nu, tc, vbytes)
        assert got == _gs_bytes(want, nu, vbytes)


def test_dram_ratio_belongs_to_the_current_kernel():
    """The DRAM/algorithmic ratio that bench.py turns into `traffic` was measured on one version of
    the kernel: every recorded ratio names the sources it was captured from, and they must be the
    files on disk (else recapture the kernel or drop the entry)."""
    import bench
    for (prec, shape) in bench.GS_DRAM_PER_ALGORITHMIC:
        assert shape in bench.GS_DRAM_KERNEL and shape in bench.GS_DRAM_SOURCES
        assert bench.capture_current(shape), f"sources of {bench.GS_DRAM_KERNEL[shape]} changed since the capture"


def test_eigensolver_flop_model():
    """bench.eig_flops against the operation counts written out step by step: the L^-1 products
    (full first product, lower triangle of the second), the Householder steps on the lower
    triangle (A v, the rank-2 update) and on R, R L^-T, nu^2 QL rotations of 20 flops and their
    replay at 6 flops per row; eig_roofline sums it over the columns' own pattern rows."""
    for nu, rows in ((7, 5), (30, 46), (100, 78)):
        first = sum(2 * (i + 1) * nu for i in range(nu))
        second = sum(2 * (i + 1) * (nu - i) for i in range(nu))
        hh = sum(2 * L * L + 2 * L * (L + 1) for L in range(nu - 1, 1, -1))   # A v, rank-2 (lower)
        r_lt = sum(2 * (i + 1) for i in range(nu)) * rows
        r_refl = sum(4 * L for L in range(nu - 1, 1, -1)) * rows
        ql, replay = 20 * nu * nu, 6 * nu * nu * rows
        exact = first + second + hh + r_lt + r_refl + ql + replay
        model = bench.eig_flops(nu, rows)
        # the model keeps the leading terms: within 1 % at the sizes the bench runs
        assert abs(model - exact) <= 0.01 * exact, (nu, model, exact)
    t = tiny_hydrocarbon(12, 4, seed=0)
    cols = t.real_columns()
    r = bench.eig_roofline(t, cols, 12, (3, 2.0), 1)
    blocks = np.diff(t.row_ptr)[cols // 4]
    want = sum(bench.eig_flops(12, 4 * int(b) + 2) for b in blocks) / 2e-3 / 1e12
    assert r["achieved"] == pytest.approx(want, rel=1e-3, abs=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS, rel=1e-2, abs=1e-4)
    assert bench.eig_roofline(t, cols, 12, (0, 0.0), 1) is None


def test_mixed_vs_fp64_statistics():
    """bench.mixed_vs_fp64's host logic on a stand-in for the library: two densities that differ in
    one known entry give that entry's size, its count above the bounds and its column."""
    from types import SimpleNamespace

    t = tiny_hydrocarbon(12, 4, seed=0)
    nu = 6
    rho64 = np.zeros((t.nnzb, 4, 4))
    rho32 = rho64.copy()
    blk, a, b = 5, 1, 2
    rho32[blk, a, b] = 3e-5
    col = 4 * int(t.col_idx[blk]) + b
    eps = np.tile(np.linspace(-2.0, 2.0, nu), (t.M, 1))

    class Ctx:
        def __init__(self, prec):
            self.prec = prec

    lib = SimpleNamespace(
        setup_system=lambda sysm, prec: Ctx(prec),
        marnoldi_solve=lambda ctx, cols, nu_, reg, ne, kT: None,
        marnoldi_energy=lambda ctx: (-10.0 - 1e-9 * ctx.prec, 0.0, 16.0),
        marnoldi_density=lambda ctx: ((rho32, 2 * rho32) if ctx.prec else (rho64, 2 * rho64)),
        marnoldi_column_stats=lambda ctx: (np.full(t.M, nu, np.int32), eps, np.ones((t.M, nu))),
        marnoldi_fermi_at=lambda ctx, mu, kT: (0.0, 0.0),
        marnoldi_gs_shape=lambda ctx: (64, 288),
        marnoldi_destroy=lambda ctx: None)
    import tbsynth   # mixed_vs_fp64 imports the generator when it runs
    saved = tbsynth.config_c2
    tbsynth.config_c2 = lambda seed=0: t
    try:
        out = bench.mixed_vs_fp64(lib, nu)
    finally:
        tbsynth.config_c2 = saved
    assert out["max_drho"] == pytest.approx(3e-5)
    assert out["drho_gt_1e-5"] == 1 and out["drhoE_gt_1e-4"] == 0
    assert out["max_drhoE_eV"] == pytest.approx(6e-5)
    assert out["worst"]["column"] == col
    assert out["dE_band_per_atom_eV"] == pytest.approx(1e-9 / t.n_block_rows)
    assert out["rho_entries"] == t.nnzb * 16
