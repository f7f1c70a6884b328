"""Plain FP64 CPU oracle of the multiple Arnoldi (mArnoldi) method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or runs anything here, and nothing here imports the product.

The arithmetic lives in ``marnoldi_oracle.c`` (plain loops, OpenMP over columns
only); this module compiles it with gcc, calls it through ctypes and arranges
its per-column outputs into BSR density values.  The steps follow
Hoshi, Yamazaki, Akiyama, arXiv:1307.3218, Section 2 (Eq. 1, Eq. 2 and the
paragraph after Eq. 2); the readings of points the paper leaves open are listed
at the top of ``marnoldi_oracle.c``.
"""

from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "marnoldi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None

TAU_FP64 = 1e-10      # relative breakdown threshold
BISECT_RTOL = 1e-12   # |N - Ne| <= rtol * Ne
BISECT_MAXIT = 200


def lib_path() -> str:
    return os.path.join(_BUILD, f"libmarnoldi_oracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    out = lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(build())
        P = C.c_void_p
        i64, i32, d = C.c_int64, C.c_int, C.c_double
        L.oracle_column.restype = i32
        L.oracle_column.argtypes = [i64, P, P, P, P, i64, i32, d, i64, P, P, P, P, P, P, P]
        L.oracle_columns.restype = i32
        L.oracle_columns.argtypes = [i64, P, P, P, P, i64, P, i32, d, P, P, P, P, P, P, P, i32]
        L.oracle_jacobi_eigh.restype = i32
        L.oracle_jacobi_eigh.argtypes = [i32, P, P, P]
        L.oracle_fermi.restype = d
        L.oracle_fermi.argtypes = [d]
        L.oracle_count.restype = None
        L.oracle_count.argtypes = [i64, P, P, d, d, P, P]
        L.oracle_bisect.restype = i32
        L.oracle_bisect.argtypes = [i64, P, P, d, d, d, i32, P, P, P]
        L.oracle_density.restype = None
        L.oracle_density.argtypes = [i64, i32, P, P, P, P, d, d, P, P]
        L.oracle_threads.restype = i32
        L.oracle_threads.argtypes = []
        _LIB = L
    return _LIB


class use_library:
    """Context manager: run the oracle functions against another build of the oracle source.

    Only the mutation tests use it, to check that planted mistakes fail the pins.
    """

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _LIB
        self.saved = _LIB
        _LIB = None
        real_build = globals()["build"]
        globals()["build"] = lambda force=False: self.path
        try:
            _lib()
        finally:
            globals()["build"] = real_build
        return self

    def __exit__(self, *exc):
        global _LIB
        _LIB = self.saved
        return False


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def threads() -> int:
    return int(_lib().oracle_threads())


def fermi(x: float) -> float:
    return float(_lib().oracle_fermi(float(x)))


def jacobi_eigh(A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    n = A.shape[0]
    e = np.zeros(n)
    V = np.zeros((n, n))
    if _lib().oracle_jacobi_eigh(n, _p(A), _p(e), _p(V)) < 0:
        raise RuntimeError("Jacobi did not converge")
    return e, V


def pattern_rows(sysm, j: int) -> np.ndarray:
    """Orbital rows of column j's pattern: the 4 rows of every block in block-row j//4, in block order."""
    J = j // 4
    blocks = sysm.col_idx[sysm.row_ptr[J]:sysm.row_ptr[J + 1]].astype(np.int64)
    return (4 * blocks[:, None] + np.arange(4)[None, :]).reshape(-1)


def _csr_args(sysm):
    rp = np.ascontiguousarray(sysm.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(sysm.col_idx, dtype=np.int32)
    Hv = np.ascontiguousarray(sysm.H, dtype=np.float64)
    Sv = np.ascontiguousarray(sysm.S, dtype=np.float64)
    return rp, ci, Hv, Sv


@dataclass
class Columns:
    cols: np.ndarray        # (nc,) int64 orbital columns
    nu: int
    nu_eff: np.ndarray      # (nc,) int32
    eps: np.ndarray         # (nc, nu)
    w: np.ndarray           # (nc, nu)
    t: np.ndarray           # (nc, nu)
    row_off: np.ndarray     # (nc+1,) offsets into rows / Y
    rows: np.ndarray        # concatenated orbital rows per column
    Y: np.ndarray           # (row_off[-1], nu): rows of K V


def column(sysm, j: int, nu: int, tau: float = TAU_FP64, rows: np.ndarray | None = None):
    """One column with its subspace matrix and basis (small systems; for the pins)."""
    rp, ci, Hv, Sv = _csr_args(sysm)
    M = sysm.M
    rows = np.arange(M, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    eps = np.zeros(nu); w = np.zeros(nu); t = np.zeros(nu)
    Y = np.zeros((rows.size, nu)); Hsub = np.zeros((nu, nu)); K = np.zeros((nu, M))
    r = _lib().oracle_column(sysm.n_block_rows, _p(rp), _p(ci), _p(Hv), _p(Sv), int(j), int(nu),
                             float(tau), rows.size, _p(rows), _p(eps), _p(w), _p(t), _p(Y),
                             _p(Hsub), _p(K))
    if r < 0:
        raise RuntimeError(f"oracle column failed: {r}")
    return dict(nu_eff=r, eps=eps, w=w, t=t, Y=Y, Hsub=Hsub, K=K, rows=rows)


def columns(sysm, cols, nu: int, tau: float = TAU_FP64, full_rows: bool = False,
            nthreads: int = 0) -> Columns:
    rp, ci, Hv, Sv = _csr_args(sysm)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    nc = cols.size
    if full_rows:
        rows_l = [np.arange(sysm.M, dtype=np.int64)] * nc
    else:
        rows_l = [pattern_rows(sysm, int(j)) for j in cols]
    row_off = np.zeros(nc + 1, np.int64)
    row_off[1:] = np.cumsum([r.size for r in rows_l])
    rows = np.ascontiguousarray(np.concatenate(rows_l) if nc else np.zeros(0, np.int64))
    nu_eff = np.zeros(nc, np.int32)
    eps = np.zeros((nc, nu)); w = np.zeros((nc, nu)); t = np.zeros((nc, nu))
    Y = np.zeros((int(row_off[-1]), nu))
    r = _lib().oracle_columns(sysm.n_block_rows, _p(rp), _p(ci), _p(Hv), _p(Sv), nc, _p(cols),
                              int(nu), float(tau), _p(row_off), _p(rows), _p(nu_eff), _p(eps),
                              _p(w), _p(t), _p(Y), int(nthreads))
    if r < 0:
        raise RuntimeError(f"oracle columns failed: {r}")
    return Columns(cols, nu, nu_eff, eps, w, t, row_off, rows, Y)


def region(positions: np.ndarray, box: np.ndarray, J: int, n_reg: int) -> np.ndarray:
    """Projection region of atom J: the n_reg atoms nearest J, ascending atom index.

    Distance: squared minimum-image distance, each component
    d = x_i - x_J - L rint((x_i - x_J) / L), summed as (dx^2 + dy^2) + dz^2;
    ties go to the lower atom index.  J itself (distance 0) is always inside.
    """
    d = positions - positions[J]
    d = d - box * np.round(d / box)
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    order = np.lexsort((np.arange(positions.shape[0]), d2))[:n_reg]
    return np.sort(order)


def local_system(sysm, R: np.ndarray):
    """Principal sub-pair of (H, S) on the atoms R (ascending): BSR arrays in local numbering."""
    R = np.asarray(R, dtype=np.int64)
    rows, cols, ks = [], [], []
    for q, I in enumerate(R):
        k0, k1 = int(sysm.row_ptr[I]), int(sysm.row_ptr[I + 1])
        J = sysm.col_idx[k0:k1].astype(np.int64)
        pos = np.searchsorted(R, J)
        ok = (pos < R.size) & (R[np.minimum(pos, R.size - 1)] == J)
        rows.append(np.full(ok.sum(), q))
        cols.append(pos[ok])
        ks.append(np.arange(k0, k1)[ok])
    rows = np.concatenate(rows)
    rp = np.zeros(R.size + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    ks = np.concatenate(ks)
    return (R.size, rp, np.concatenate(cols).astype(np.int32),
            np.ascontiguousarray(sysm.H[ks]), np.ascontiguousarray(sysm.S[ks]))


def regional_columns(sysm, cols, nu: int, n_reg: int, positions=None, box=None,
                     tau: float = TAU_FP64, nthreads: int = 0) -> Columns:
    """Columns solved in regional mode: each column's Krylov process runs on the
    principal sub-pair of (H, S) over its atom's projection region.  Pattern rows
    of atoms outside the region are zero."""
    import concurrent.futures as cf
    s = sysm.structure
    positions = s.positions if positions is None else positions
    box = s.box if box is None else box
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    nc = cols.size
    rows_l = [pattern_rows(sysm, int(j)) for j in cols]
    row_off = np.zeros(nc + 1, np.int64)
    row_off[1:] = np.cumsum([r.size for r in rows_l])
    rows = np.concatenate(rows_l) if nc else np.zeros(0, np.int64)
    nu_eff = np.zeros(nc, np.int32)
    eps = np.zeros((nc, nu)); w = np.zeros((nc, nu)); t = np.zeros((nc, nu))
    Y = np.zeros((int(row_off[-1]), nu))
    cache: dict = {}

    def one(q):
        j = int(cols[q])
        J, b = j // 4, j % 4
        if J not in cache:
            R = region(positions, box, J, n_reg)
            cache[J] = (R, local_system(sysm, R))
        R, (nb, lrp, lci, lH, lS) = cache[J]
        jl = 4 * int(np.searchsorted(R, J)) + b
        grows = rows_l[q]
        gatoms = grows // 4
        pos = np.searchsorted(R, gatoms)
        inside = (pos < R.size) & (R[np.minimum(pos, R.size - 1)] == gatoms)
        lrows = np.ascontiguousarray(4 * pos[inside] + grows[inside] % 4, dtype=np.int64)
        e_ = np.zeros(nu); w_ = np.zeros(nu); t_ = np.zeros(nu)
        Yl = np.zeros((lrows.size, nu))
        r = _lib().oracle_column(nb, _p(lrp), _p(lci), _p(lH), _p(lS), jl, int(nu), float(tau),
                                 lrows.size, _p(lrows), _p(e_), _p(w_), _p(t_), _p(Yl), None, None)
        if r < 0:
            raise RuntimeError(f"oracle column {j} failed: {r}")
        nu_eff[q] = r
        eps[q], w[q], t[q] = e_, w_, t_
        seg = np.zeros((grows.size, nu))
        seg[inside] = Yl
        Y[row_off[q]:row_off[q + 1]] = seg

    # per-atom regions first (serial), then the columns in parallel (the C calls release the GIL)
    for J in sorted({int(j) // 4 for j in cols}):
        R = region(positions, box, J, n_reg)
        cache[J] = (R, local_system(sysm, R))
    with cf.ThreadPoolExecutor(max_workers=nthreads or os.cpu_count() or 1) as ex:
        list(ex.map(one, range(nc)))
    return Columns(cols, nu, nu_eff, eps, w, t, row_off, rows, Y)


def valid_levels(c: Columns) -> tuple[np.ndarray, np.ndarray]:
    """(eps, w) of the nu_eff valid levels of every column, concatenated."""
    mask = np.arange(c.nu)[None, :] < c.nu_eff[:, None]
    return np.ascontiguousarray(c.eps[mask]), np.ascontiguousarray(c.w[mask])


def count(eps, w, mu: float, kT: float) -> tuple[float, float]:
    eps = np.ascontiguousarray(eps, np.float64); w = np.ascontiguousarray(w, np.float64)
    N = C.c_double(); E = C.c_double()
    _lib().oracle_count(eps.size, _p(eps), _p(w), float(mu), float(kT), C.byref(N), C.byref(E))
    return N.value, E.value


def bisect(eps, w, Ne: float, kT: float, rtol: float = BISECT_RTOL,
           maxit: int = BISECT_MAXIT) -> tuple[float, float, float, int]:
    eps = np.ascontiguousarray(eps, np.float64); w = np.ascontiguousarray(w, np.float64)
    mu = C.c_double(); N = C.c_double(); E = C.c_double()
    it = _lib().oracle_bisect(eps.size, _p(eps), _p(w), float(Ne), float(kT), float(rtol),
                              int(maxit), C.byref(mu), C.byref(N), C.byref(E))
    if it < 0:
        raise RuntimeError("electron count outside the bisection bracket")
    return mu.value, N.value, E.value, it


def density_rows(c: Columns, mu: float, kT: float) -> tuple[np.ndarray, np.ndarray]:
    rho = np.zeros(c.Y.shape[0]); rhoE = np.zeros(c.Y.shape[0])
    _lib().oracle_density(c.cols.size, c.nu, _p(c.row_off), _p(np.ascontiguousarray(c.eps)),
                          _p(np.ascontiguousarray(c.t)), _p(c.Y), float(mu), float(kT),
                          _p(rho), _p(rhoE))
    return rho, rhoE


def green_rows(c: Columns, z: complex) -> np.ndarray:
    """G(z) e_j on each column's rows: (K V) diag(1/(z - eps)) t (valid levels only)."""
    out = np.zeros(c.Y.shape[0], np.complex128)
    for ci_ in range(c.cols.size):
        ne = int(c.nu_eff[ci_])
        y = c.t[ci_, :ne] / (z - c.eps[ci_, :ne])
        sl = slice(c.row_off[ci_], c.row_off[ci_ + 1])
        out[sl] = c.Y[sl, :ne] @ y
    return out


def block_index(sysm) -> dict:
    """(I, J) -> BSR block index."""
    rows = np.repeat(np.arange(sysm.n_block_rows), np.diff(sysm.row_ptr))
    return {(int(I), int(J)): k for k, (I, J) in enumerate(zip(rows, sysm.col_idx))}


def scatter_pattern(sysm, c: Columns, vals_rows: np.ndarray) -> np.ndarray:
    """Put pattern-row values of columns j into BSR values [nnzb, 4, 4] (entry [I,J][a][b] = col 4J+b, row 4I+a).

    Blocks whose column was not computed stay NaN.
    """
    out = np.full((sysm.nnzb, 4, 4), np.nan, dtype=vals_rows.dtype)
    bidx = block_index(sysm)
    for ci_, j in enumerate(c.cols):
        J, b = int(j) // 4, int(j) % 4
        seg = vals_rows[c.row_off[ci_]:c.row_off[ci_ + 1]]
        for r, row in enumerate(c.rows[c.row_off[ci_]:c.row_off[ci_ + 1]]):
            I, a = int(row) // 4, int(row) % 4
            out[bidx[(I, J)], a, b] = seg[r]
    return out


@dataclass
class Solution:
    mu: float
    N: float
    E_band: float
    rho: np.ndarray       # [nnzb, 4, 4]
    rhoE: np.ndarray      # [nnzb, 4, 4]
    cols: Columns
    iters: int


def solve(sysm, nu: int, kT: float, Ne: float | None = None, mu_fixed: float | None = None,
          cols=None, tau: float = TAU_FP64, nthreads: int = 0, region_atoms: int = 0) -> Solution:
    """The whole path: every column's subspace, the Fermi level, rho and rho^E on H's pattern, E_band."""
    if cols is None:
        cols = sysm.real_columns()
    if region_atoms:
        c = regional_columns(sysm, cols, nu, region_atoms, tau=tau, nthreads=nthreads)
    else:
        c = columns(sysm, cols, nu, tau=tau, nthreads=nthreads)
    e, w = valid_levels(c)
    if mu_fixed is None:
        Ne = sysm.n_electrons if Ne is None else Ne
        mu, N, E, it = bisect(e, w, Ne, kT)
    else:
        mu = float(mu_fixed)
        N, E = count(e, w, mu, kT)
        it = 0
    rr, rre = density_rows(c, mu, kT)
    return Solution(mu, N, E, scatter_pattern(sysm, c, rr), scatter_pattern(sysm, c, rre), c, it)


def forces(sysm, rho: np.ndarray, rhoE: np.ndarray, dH: np.ndarray, dS: np.ndarray) -> np.ndarray:
    """Atomic forces F_K = -Tr(rho dH/dR_K) + Tr(rho^E dS/dR_K), shape (n_atoms, 3).

    Section 2: the Green's function (here its density and energy-density
    matrices) gives the total energy and the force; the paper prints no force
    formula, so this is the standard one for a non-orthogonal basis, with the
    unsymmetrised column results symmetrised, rho_bar = (rho + rho^T) / 2.
    dH, dS: (3, nnzb, 4, 4), block (I, J) differentiated with respect to
    d = R_J - R_I, so dH_IJ/dR_I = -dH[., k] and dH_IJ/dR_J = +dH[., k].
    Entries of columns that were not computed (NaN) count as 0.
    """
    nb = sysm.nnzb
    rows = np.repeat(np.arange(sysm.n_block_rows), np.diff(sysm.row_ptr))
    cols = np.asarray(sysm.col_idx, dtype=np.int64)
    bidx = block_index(sysm)
    kt = np.array([bidx[(int(J), int(I))] for I, J in zip(rows, cols)], dtype=np.int64)
    r = np.nan_to_num(np.asarray(rho, dtype=np.float64).reshape(nb, 4, 4))
    rE = np.nan_to_num(np.asarray(rhoE, dtype=np.float64).reshape(nb, 4, 4))
    rbar = 0.5 * (r + r[kt].transpose(0, 2, 1))
    rEbar = 0.5 * (rE + rE[kt].transpose(0, 2, 1))
    F = np.zeros((sysm.n_block_rows, 3))
    for x in range(3):
        trH = np.einsum("kab,kab->k", rbar, dH[x])     # Tr(rho_bar_k^T dH_k), one block
        trS = np.einsum("kab,kab->k", rEbar, dS[x])
        # -Tr(rho dH/dR_K) + Tr(rho^E dS/dR_K): block k = (I, J) enters K = I with
        # dH/dR_I = -dH_k and K = J with dH/dR_J = +dH_k
        np.add.at(F[:, x], rows, trH - trS)
        np.add.at(F[:, x], cols, -trH + trS)
    return F


def _fermi_np(x):
    """f(x) = 1 / (1 + e^x) elementwise, through e^(-|x|); +-inf give 0 and 1."""
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(-np.abs(x))
    return np.where(x >= 0, e / (1.0 + e), 1.0 / (1.0 + e))


def idos(c: Columns, eta: float, sigma: float) -> float:
    """Integrated density of states n(eta) = sum_j sum_a w_a f((eps_a - eta) / sigma), one state per
    level (no spin factor): the count of levels below eta, each step smoothed by the Fermi function
    of width sigma (Section 2, the paragraph on the k-th eigen level)."""
    e, w = valid_levels(c)
    return float(np.sum(w * _fermi_np((e - eta) / sigma)))


def eigenstate(sysm, k: int, nu: int, sigma: float, tau: float = TAU_FP64):
    """The k-th eigen level and vector from the subspace levels and vectors (Section 2, Eq. 3 of the
    paper's eigenstate paragraph, and the inner-product sign rule of its Appendix).

    n(eta) as in idos(); eta(n) its inverse by the bisection of bisect() on 2 n (the count there
    carries the spin factor 2), eta(0) = -inf and eta(M_real) = +inf; eps_k = eta(k - 1/2).  The
    smoothed delta of Eq. 3 is read as the derivative of the Fermi step of width sigma, so
    int_{eta(k-1)}^{eta(k)} delta(eps - eps_a) = f((eps_a - eta(k)) / sigma) - f((eps_a - eta(k-1)) / sigma)
    =: W_a.  Component j of phi_k: sum_a s_a t_a W_a with t_a = e_j^T K v_a.  Signs: the reference is
    the subspace eigenvector (full-space K v_a over all columns j and levels a) of largest |t_a W_a|
    (first in column, then level order among equals); s_a = sign(v_ref^T K v_a), +1 when it is 0.
    Returns (eps_k, phi (M,), info).  Small systems only: it keeps every column's full vectors.
    """
    cols = sysm.real_columns()
    c = columns(sysm, cols, nu, tau=tau, full_rows=True)
    e, w = valid_levels(c)
    m_real = cols.size

    def eta(n):
        if n <= 0:
            return -np.inf
        if n >= m_real:
            return np.inf
        return bisect(e, w, 2.0 * n, sigma)[0]

    lo, ek, hi = eta(k - 1), eta(k - 0.5), eta(k)
    valid = np.arange(nu)[None, :] < c.nu_eff[:, None]
    W = np.where(valid, _fermi_np((c.eps - hi) / sigma) - _fermi_np((c.eps - lo) / sigma), 0.0)
    a = np.where(valid, c.t * W, 0.0)
    q, al = np.unravel_index(int(np.argmax(np.abs(a))), a.shape)
    M = sysm.M
    Yc = c.Y.reshape(cols.size, M, nu)
    vref = Yc[q, :, al]
    dots = np.einsum("r,crl->cl", vref, Yc)
    s = np.where(dots < 0.0, -1.0, 1.0)
    phi = np.zeros(M)
    phi[cols] = np.sum(s * a, axis=1)
    return ek, phi, dict(eta=(lo, hi), ref=(int(cols[q]), int(al)), columns=c)
