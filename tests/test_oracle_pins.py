"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

The paper (arXiv:1307.3218) prints no worked example and no per-column numbers,
so every pin here is a closed form, an invariant, a textbook special case, a
library routine on a special case, or a high-precision brute force on a tiny
input:

* nu = 1 reduces to eps = H_jj / S_jj (closed form);
* nu = M reproduces the dense generalized eigensolve H phi = eps S phi (Eq. 2)
  and the direct solve of (z S - H) x = e_j (Eq. 1), the paper's own cross-check
  against exact diagonalisation (Section 3, last paragraph before Fig. 2);
* the Galerkin condition K^T((zS - H) x - e_j) = 0 and K^T S K = I;
* sum_a w_a = 1, and the pattern traces (S rho)_jj, (H rho)_jj;
* S = I reduces to Lanczos: a tridiagonal subspace matrix and Gauss-quadrature
  moments sum_a w_a eps_a^p = (H^p)_jj for p <= 2 nu - 1;
* the power basis [e_j, H e_j, ...] solved as a nu x nu generalized problem in
  50-digit arithmetic (span independence, brute force);
* the bisection's bracket and stopping rule; relabelling invariance;
* the Jacobi eigensolver against LAPACK, the Fermi function against tanh.
"""

import numpy as np
import pytest
import scipy.linalg as sl
from scipy.special import expit

import oracle
from tbsynth import tiny_system

KT = 0.1


def fermi2(x):
    """2 f(x) with f(x) = 1/(1 + e^x) = expit(-x), the library logistic function."""
    return 2.0 * expit(-np.asarray(x, dtype=np.float64))


def dense_reference(t, mu, kT=KT):
    H, S = t.dense()
    ev, Phi = sl.eigh(H, S)
    f2 = fermi2((ev - mu) / kT)
    rho = (Phi * f2) @ Phi.T
    rhoE = (Phi * (f2 * ev)) @ Phi.T
    return H, S, ev, Phi, rho, rhoE


def bsr_to_dense_blocks(t, vals):
    out = {}
    rows = np.repeat(np.arange(t.n_block_rows), np.diff(t.row_ptr))
    for k, (I, J) in enumerate(zip(rows, t.col_idx)):
        out[(int(I), int(J))] = vals[k]
    return out


# --------------------------------------------------------------------------- building blocks

def test_fermi_against_tanh_and_limits():
    xs = np.array([-800.0, -50.0, -3.0, -1e-9, 0.0, 1e-9, 0.7, 3.0, 50.0, 800.0])
    got = np.array([oracle.fermi(x) for x in xs])
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(2 * got, fermi2(xs), rtol=1e-14, atol=1e-300)
    # and against the tanh form where it has no cancellation (x <= 0)
    neg = xs[xs <= 0]
    np.testing.assert_allclose(2 * got[xs <= 0], 1.0 - np.tanh(0.5 * neg), rtol=1e-14)
    assert oracle.fermi(0.0) == 0.5
    for x in xs:
        assert abs(oracle.fermi(x) + oracle.fermi(-x) - 1.0) < 1e-15
    assert np.all(np.diff(got) <= 0)


@pytest.mark.parametrize("n,seed", [(7, 0), (40, 1), (100, 2)])
def test_jacobi_matches_lapack(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = A + A.T
    A[0, 1] = A[1, 0] = 0.0
    e, V = oracle.jacobi_eigh(A)
    ref = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(e, ref, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(A @ V, V * e, atol=1e-12 * np.abs(ref).max())
    assert np.all(np.diff(e) >= 0)


def test_jacobi_degenerate():
    e, V = oracle.jacobi_eigh(np.diag([3.0, 1.0, 1.0, -2.0]))
    np.testing.assert_array_equal(e, [-2.0, 1.0, 1.0, 3.0])
    np.testing.assert_allclose(np.abs(V.T @ V), np.eye(4), atol=1e-15)


# --------------------------------------------------------------------------- closed forms

def test_p1_nu1_closed_form(c1):
    H, S = c1.dense()
    for j in (0, 1, 5, 130, 255):
        r = oracle.column(c1, j, 1)
        assert r["nu_eff"] == 1
        assert r["eps"][0] == pytest.approx(H[j, j] / S[j, j], rel=1e-15)
        assert r["w"][0] == pytest.approx(1.0, abs=1e-15)
        mu = 0.3
        c = oracle.columns(c1, [j], 1, full_rows=True)
        rho, rhoE = oracle.density_rows(c, mu, KT)
        e = H[j, j] / S[j, j]
        expect = np.zeros(c1.M)
        expect[j] = fermi2((e - mu) / KT) / S[j, j]
        np.testing.assert_allclose(rho, expect, atol=1e-15)
        np.testing.assert_allclose(rhoE, expect * e, atol=1e-13)


@pytest.mark.parametrize("n,seed", [(8, 0), (10, 3)])
def test_p3_dense_limit(n, seed):
    """nu = M: rho, rho^E and G(z) columns equal the dense generalized solution."""
    t = tiny_system(n, seed=seed)
    M = t.M
    sol = oracle.solve(t, nu=M, kT=KT)
    assert np.all(sol.cols.nu_eff == M)
    H, S, ev, Phi, rho, rhoE = dense_reference(t, sol.mu)
    # electron count and band energy of the dense solution at the same mu
    f2 = fermi2((ev - sol.mu) / KT)
    assert sol.N == pytest.approx(np.sum(f2), rel=1e-12)
    assert sol.E_band == pytest.approx(np.sum(f2 * ev), rel=1e-12)
    assert sol.N == pytest.approx(t.n_electrons, rel=1e-12)
    blocks = bsr_to_dense_blocks(t, sol.rho)
    blocksE = bsr_to_dense_blocks(t, sol.rhoE)
    scale, scaleE = np.abs(rho).max(), np.abs(rhoE).max()
    for (I, J), v in blocks.items():
        np.testing.assert_allclose(v, rho[4 * I:4 * I + 4, 4 * J:4 * J + 4], atol=1e-11 * scale)
        np.testing.assert_allclose(blocksE[(I, J)], rhoE[4 * I:4 * I + 4, 4 * J:4 * J + 4],
                                   atol=1e-11 * scaleE)
    # full columns, and the Green's function against a direct solve of Eq. 1
    cols = np.array([0, 3, M // 2 + 1, M - 1])
    c = oracle.columns(t, cols, M, full_rows=True)
    rr, _ = oracle.density_rows(c, sol.mu, KT)
    for z in (sol.mu + 0.5j, -3.0 + 0.05j, 40.0 - 2.0j):
        g = oracle.green_rows(c, z)
        G = np.linalg.solve(z * S - H, np.eye(M)[:, cols])
        for q, j in enumerate(cols):
            seg = slice(c.row_off[q], c.row_off[q + 1])
            np.testing.assert_allclose(g[seg], G[:, q], atol=1e-11 * np.abs(G).max())
            np.testing.assert_allclose(rr[seg], rho[:, j], atol=1e-11 * scale)


def test_p3_standard_problem_s_identity():
    """S = I and nu = M: rho equals the standard eigendecomposition of H."""
    t = tiny_system(8, seed=0)
    t.S = np.zeros_like(t.S)
    for I in range(t.n_block_rows):
        for k in range(t.row_ptr[I], t.row_ptr[I + 1]):
            if t.col_idx[k] == I:
                t.S[k] = np.eye(4)
    mu = -1.0
    c = oracle.columns(t, t.real_columns(), t.M, full_rows=True)
    rr, _ = oracle.density_rows(c, mu, KT)
    H, _ = t.dense()
    ev, Phi = np.linalg.eigh(H)
    rho = (Phi * fermi2((ev - mu) / KT)) @ Phi.T
    np.testing.assert_allclose(rr.reshape(t.M, t.M).T, rho, atol=1e-11 * np.abs(rho).max())


# --------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("nu", [3, 7])
def test_p4_galerkin_and_s_orthonormality(nu):
    t = tiny_system(10, seed=3)
    H, S = t.dense()
    for j in (0, 5, 17, 38):
        r = oracle.column(t, j, nu)
        assert r["nu_eff"] == nu
        K = r["K"][:nu].T                     # M x nu
        np.testing.assert_allclose(K.T @ S @ K, np.eye(nu), atol=1e-12)
        np.testing.assert_allclose(r["Hsub"], K.T @ H @ K, atol=1e-11 * np.abs(H).max())
        # Y holds the full rows of K V
        for z in (0.5 + 0.2j, -7.0 + 1.0j):
            y = r["t"][:nu] / (z - r["eps"][:nu])
            x = r["Y"][:, :nu] @ y
            res = K.T @ ((z * S - H) @ x - np.eye(t.M)[:, j])
            assert np.abs(res).max() < 1e-11 * max(1.0, np.abs(x).max() * np.abs(H).max())
        # q = K^T e_j has only its first entry nonzero... in the S-orthonormal basis
        # e_j^T S K = sqrt(S_jj) e_1^T, so K^T S e_j = sqrt(S_jj) e_1
        np.testing.assert_allclose(K.T @ S[:, j], np.sqrt(S[j, j]) * np.eye(nu)[0], atol=1e-12)


def test_p5_weights_sum_to_one(c1):
    c = oracle.columns(c1, c1.real_columns(), 30)
    assert np.all(c.nu_eff == 30)
    np.testing.assert_allclose(c.w.sum(axis=1), 1.0, atol=1e-13)


def test_p6_p7_pattern_traces(c1):
    """(S rho)_jj = sum 2 f w and (H rho)_jj = sum 2 f eps w, read off the pattern."""
    sol = oracle.solve(c1, nu=30, kT=KT)
    c = sol.cols
    f2 = fermi2((c.eps - sol.mu) / KT)
    n_col = np.sum(f2 * c.w, axis=1)
    e_col = np.sum(f2 * c.eps * c.w, axis=1)
    rows = np.repeat(np.arange(c1.n_block_rows), np.diff(c1.row_ptr))
    bidx = oracle.block_index(c1)
    trS = np.zeros(c1.M)
    trH = np.zeros(c1.M)
    for k, (J, I) in enumerate(zip(rows, c1.col_idx)):     # block (J, I) of row J
        kt = bidx[(int(I), int(J))]                          # rho block (I, J)
        for b in range(4):
            j = 4 * J + b
            trS[j] += c1.S[k][b, :] @ sol.rho[kt][:, b]
            trH[j] += c1.H[k][b, :] @ sol.rho[kt][:, b]
    np.testing.assert_allclose(trS, n_col, atol=1e-12)
    np.testing.assert_allclose(trH, e_col, atol=1e-12 * np.abs(e_col).max())
    assert trS.sum() == pytest.approx(c1.n_electrons, rel=1e-11)
    assert trH.sum() == pytest.approx(sol.E_band, rel=1e-11)


def test_p8_lanczos_gauss_quadrature():
    """S = I: tridiagonal H_sub, w_a = V[0,a]^2 >= 0, moments exact up to 2 nu - 1."""
    t = tiny_system(10, seed=0)
    t.S = np.zeros_like(t.S)
    for I in range(t.n_block_rows):
        for k in range(t.row_ptr[I], t.row_ptr[I + 1]):
            if t.col_idx[k] == I:
                t.S[k] = np.eye(4)
    H, _ = t.dense()
    nu = 6
    rad = np.abs(np.linalg.eigvalsh(H)).max()
    for j in (0, 9, 22):
        r = oracle.column(t, j, nu)
        T = r["Hsub"]
        off = np.triu(np.abs(T), 2)
        assert off.max() < 1e-12 * rad
        assert np.all(r["w"] >= -1e-15)
        Hp = np.eye(t.M)
        for p in range(2 * nu):
            mom = np.sum(r["w"] * r["eps"] ** p)
            assert abs(mom - Hp[j, j]) <= 1e-11 * rad ** p + 1e-13, (j, p)
            Hp = Hp @ H


def test_p9_power_basis_brute_force_50_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    t = tiny_system(6, seed=2)
    H, S = t.dense()
    M = t.M
    Hm = mp.matrix(H.tolist())
    Sm = mp.matrix(S.tolist())
    mu = 0.7
    for j, nu in ((0, 2), (5, 3), (13, 5), (20, 7)):
        B = mp.matrix(M, nu)
        v = mp.matrix(M, 1)
        v[j] = 1
        for i in range(nu):
            for r in range(M):
                B[r, i] = v[r]
            v = Hm * v
        A = B.T * Hm * B
        Cm = B.T * Sm * B
        L = mp.cholesky(Cm)
        Li = mp.inverse(L)
        E, U = mp.eigsy(Li * A * Li.T)
        Y = Li.T * U                               # Cm-orthonormal generalized eigenvectors
        order = sorted(range(nu), key=lambda a: E[a])
        eps = np.array([float(E[a]) for a in order])
        BY = B * Y
        ej = mp.matrix(M, 1)
        ej[j] = 1
        SB = (Sm * BY).T * ej                      # e_j^T S B y_a
        Bt = BY.T * ej                             # y_a^T B^T e_j
        w = np.array([float(SB[a] * Bt[a]) for a in order])
        rho = mp.matrix(M, 1)
        for a in range(nu):
            f2 = 1 - mp.tanh((E[a] - mu) / (2 * mp.mpf(KT)))
            for r in range(M):
                rho[r] += BY[r, a] * f2 * Bt[a]
        rho = np.array([float(x) for x in rho])
        r_or = oracle.column(t, j, nu)
        assert r_or["nu_eff"] == nu
        np.testing.assert_allclose(r_or["eps"], eps, atol=1e-11 * np.abs(eps).max())
        np.testing.assert_allclose(r_or["w"], w, atol=1e-11)
        c = oracle.columns(t, [j], nu, full_rows=True)
        rr, _ = oracle.density_rows(c, mu, KT)
        np.testing.assert_allclose(rr, rho, atol=1e-11 * max(1.0, np.abs(rho).max()))


def test_p10_bisection(c1):
    c = oracle.columns(c1, c1.real_columns(), 30)
    e, w = oracle.valid_levels(c)
    mu, N, E, it = oracle.bisect(e, w, c1.n_electrons, KT)
    assert abs(N - c1.n_electrons) <= oracle.BISECT_RTOL * c1.n_electrons
    assert 1 <= it <= oracle.BISECT_MAXIT
    grid = np.linspace(e.min() - 4, e.max() + 4, 301)
    Ns = np.array([oracle.count(e, w, m, KT)[0] for m in grid])
    assert np.all(np.diff(Ns) >= -1e-9)
    lo, hi = e.min() - 40 * KT, e.max() + 40 * KT
    assert oracle.count(e, w, lo, KT)[0] <= c1.n_electrons <= oracle.count(e, w, hi, KT)[0]
    assert np.sum(w) == pytest.approx(c1.M, rel=1e-12)     # f == 1 limit: N = 2 M_real / 2 per column
    with pytest.raises(RuntimeError):
        oracle.bisect(e, w, 2.5 * c1.M, KT)


def test_p12_relabelling(c1):
    rng = np.random.default_rng(7)
    perm = rng.permutation(c1.n_block_rows)
    t2 = c1.permuted(perm)
    a = oracle.solve(c1, nu=12, kT=KT)
    b = oracle.solve(t2, nu=12, kT=KT)
    assert b.E_band == pytest.approx(a.E_band, rel=1e-11)
    assert b.N == pytest.approx(a.N, rel=1e-11)
    ia = oracle.block_index(c1)
    ib = oracle.block_index(t2)
    for (I2, J2), k2 in ib.items():
        k1 = ia[(int(perm[I2]), int(perm[J2]))]
        np.testing.assert_allclose(b.rho[k2], a.rho[k1], atol=1e-10)
        np.testing.assert_allclose(b.rhoE[k2], a.rhoE[k1], atol=1e-8)


def test_breakdown_isolated_atom():
    """An atom with no neighbour: its columns stop at nu_eff = 1 with the exact result."""
    t = tiny_system(8, seed=1)
    deg = np.diff(t.row_ptr)
    iso = int(np.nonzero(deg == 1)[0][0])
    H, S = t.dense()
    c = oracle.columns(t, t.real_columns(), 12, full_rows=True)
    for q in range(4 * iso, 4 * iso + 4):
        assert c.nu_eff[q] == 1
        assert c.eps[q, 0] == pytest.approx(H[q, q] / S[q, q], rel=1e-15)
        assert c.w[q, 0] == pytest.approx(1.0, abs=1e-15)
    others = [q for q in range(t.M) if q // 4 != iso]
    assert np.all(c.nu_eff[others] == 12)
    # the connected rest reaches its own full Krylov dimension and the dense answer
    sol = oracle.solve(t, nu=t.M, kT=KT)
    assert sol.cols.nu_eff.max() == t.M - 4
    _, _, _, _, rho, _ = dense_reference(t, sol.mu)
    blocks = bsr_to_dense_blocks(t, sol.rho)
    for (I, J), v in blocks.items():
        np.testing.assert_allclose(v, rho[4 * I:4 * I + 4, 4 * J:4 * J + 4], atol=1e-11)


def rescaled(t, seed=11):
    """H' = D H D, S' = D S D with a random positive diagonal D (orbital rescaling, S'_jj != 1)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.5, 2.0, t.M)
    rows = np.repeat(np.arange(t.n_block_rows), np.diff(t.row_ptr))
    for k, (I, J) in enumerate(zip(rows, t.col_idx)):
        DI = d[4 * I:4 * I + 4][:, None]
        DJ = d[4 * J:4 * J + 4][None, :]
        t.H[k] = DI * t.H[k] * DJ
        t.S[k] = DI * t.S[k] * DJ
    return t, d


def test_p1_p3_p5_rescaled_orbitals():
    """S_jj != 1: nu = 1 closed form, sum w = 1, and the dense limit of the rescaled pencil."""
    t, d = rescaled(tiny_system(8, seed=0))
    H, S = t.dense()
    assert np.abs(np.diag(S) - 1.0).max() > 0.5
    for j in (0, 7, 30):
        r = oracle.column(t, j, 1)
        assert r["eps"][0] == pytest.approx(H[j, j] / S[j, j], rel=1e-14)
        assert r["w"][0] == pytest.approx(1.0, abs=1e-14)
    c = oracle.columns(t, t.real_columns(), 7)
    np.testing.assert_allclose(c.w.sum(axis=1), 1.0, atol=1e-13)
    sol = oracle.solve(t, nu=t.M, kT=KT)
    assert np.all(sol.cols.nu_eff == t.M)
    _, _, _, _, rho, rhoE = dense_reference(t, sol.mu)
    blocks = bsr_to_dense_blocks(t, sol.rho)
    for (I, J), v in blocks.items():
        np.testing.assert_allclose(v, rho[4 * I:4 * I + 4, 4 * J:4 * J + 4],
                                   atol=1e-11 * np.abs(rho).max())


def test_p11_region_of_all_atoms_is_global(c1):
    """Regional mode with the region = every atom is the global problem, bit for bit."""
    a = oracle.solve(c1, nu=20, kT=KT)
    b = oracle.solve(c1, nu=20, kT=KT, region_atoms=c1.n_block_rows)
    assert b.E_band == a.E_band and b.N == a.N
    np.testing.assert_array_equal(b.rho, a.rho)
    np.testing.assert_array_equal(b.rhoE, a.rhoE)


def test_region_definition_and_convergence(c1):
    """Regions hold the n nearest atoms (ties by index), contain the column's atom and
    every pattern neighbour once large enough; the error shrinks as regions grow."""
    s = c1.structure
    for J in (0, 17, 63):
        R = oracle.region(s.positions, s.box, J, 20)
        assert R.size == 20 and J in R and np.all(np.diff(R) > 0)
        d = s.positions - s.positions[J]
        d -= s.box * np.round(d / s.box)
        d2 = np.sum(d * d, axis=1)
        outside = np.setdiff1d(np.arange(c1.n_block_rows), R)
        assert d2[R].max() <= d2[outside].min()
        nbrs = c1.col_idx[c1.row_ptr[J]:c1.row_ptr[J + 1]]
        assert set(nbrs.tolist()) <= set(R.tolist())
    ref = oracle.solve(c1, nu=16, kT=KT)
    errs = []
    for nr in (16, 40, 64):
        r = oracle.solve(c1, nu=16, kT=KT, region_atoms=nr, mu_fixed=ref.mu)
        errs.append(np.nanmax(np.abs(r.rho - ref.rho)))
    assert errs[-1] == 0.0 and errs[1] < errs[0]


@pytest.mark.parametrize("seed", [4, 1])
def test_padding_orbitals_dense_limit(seed):
    """Hydrogen atoms padded to 4x4 blocks: the masked dummy orbitals never enter, and
    nu = (real orbitals) reproduces the dense eigensolve on the real orbitals."""
    from tbsynth import tiny_hydrocarbon
    t = tiny_hydrocarbon(10, 4, seed=seed)
    r = t.orbital_mask.astype(bool)
    nr = int(r.sum())
    sol = oracle.solve(t, nu=nr, kT=KT)
    assert sol.N == pytest.approx(t.n_electrons, rel=1e-12)
    H, S = t.dense()
    ev, Phi = sl.eigh(H[np.ix_(r, r)], S[np.ix_(r, r)])
    P = np.zeros((t.M, ev.size))
    P[r] = Phi
    rho = (P * fermi2((ev - sol.mu) / KT)) @ P.T
    for (I, J), v in bsr_to_dense_blocks(t, sol.rho).items():
        if not np.all(np.isnan(v)):
            vv = np.where(np.isnan(v), 0.0, v)
            np.testing.assert_allclose(vv, rho[4 * I:4 * I + 4, 4 * J:4 * J + 4], atol=1e-12)
    # padding columns are never solved
    assert set(sol.cols.cols.tolist()) == set(np.nonzero(r)[0].tolist())
