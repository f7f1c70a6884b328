"""Two-centre Slater-Koster tight-binding model -> BSR pair (H, S) with 4x4 blocks.

The paper works with LCAO matrices H and S, sparse and real-symmetric, S positive
definite (Section 2, the text around Eq. 1).  Its own model parameters are not
given, so this module states one model:

* carbon: orbitals (s, px, py, pz); on-site s = -5.0 eV, p = +2.0 eV; hoppings
  ss-sigma = -5.0, sp-sigma = +4.7, pp-sigma = +5.5, pp-pi = -1.8 eV, all scaled
  by (1.54 A / r)^2, hard cutoff 2.6 A;
* overlap: S = I on site; off-site the same angular form with every amplitude
  multiplied by 0.1 / 5.5 eV^-1, so that the largest overlap amplitude is 0.1
  (the literal "0.1 x H" makes S indefinite on these structures);
* hydrogen (for polymer-like inputs): one s orbital padded to a 4x4 block with
  three dummy orbitals (zero coupling, unit overlap, masked out); on-site -3.0
  eV, C-H ss-sigma = -4.0, sp-sigma = +4.5 eV scaled by (1.09 A / r)^2.

Textbook two-centre forms (Slater & Koster 1954), with (l, m, n) the direction
cosines from atom i to atom j and a, b in {x, y, z}:
    E_ss = V_sss,  E_s,b = c_b V_sps,  E_a,s = -c_a V_sps,
    E_a,b = c_a c_b (V_pps - V_ppp) + delta_ab V_ppp.
They give block(j, i) = block(i, j)^T, so H and S are symmetric.

BSR layout: ``row_ptr[n_block_rows + 1]`` (int64), ``col_idx[nnzb]`` (int32,
ascending within a row, diagonal block included), ``vals[nnzb][4][4]`` row-major
(float64).  Orbital index of (atom I, orbital a) is 4 I + a.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .structures import CARBON, HYDROGEN, Structure, amorphous_carbon, diamond, min_image

OVERLAP_FACTOR = 0.1 / 5.5     # eV^-1: S amplitudes = OVERLAP_FACTOR x H amplitudes


def carbon_params() -> dict:
    return {
        "onsite": {CARBON: (-5.0, 2.0, 2.0, 2.0), HYDROGEN: (-3.0, 0.0, 0.0, 0.0)},
        # (V_sss, V_sps, V_pps, V_ppp, r0) per unordered species pair
        "hop": {
            (CARBON, CARBON): (-5.0, 4.7, 5.5, -1.8, 1.54),
            (CARBON, HYDROGEN): (-4.0, 4.5, 0.0, 0.0, 1.09),
            (HYDROGEN, HYDROGEN): None,
        },
        "cutoff": 2.6,
        "overlap_factor": OVERLAP_FACTOR,
        "electrons": {CARBON: 4, HYDROGEN: 1},
        "real_orbitals": {CARBON: (1, 1, 1, 1), HYDROGEN: (1, 0, 0, 0)},
    }


@dataclass
class TBSystem:
    n_block_rows: int
    row_ptr: np.ndarray          # int64 [n_block_rows + 1]
    col_idx: np.ndarray          # int32 [nnzb]
    H: np.ndarray                # float64 [nnzb, 4, 4]
    S: np.ndarray                # float64 [nnzb, 4, 4]
    orbital_mask: np.ndarray     # uint8 [4 n_block_rows]
    n_electrons: float
    structure: Structure | None = None
    lambda_min_S: float | None = None
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return 4 * self.n_block_rows

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    def real_columns(self) -> np.ndarray:
        return np.nonzero(self.orbital_mask)[0].astype(np.int64)

    def dense(self) -> tuple[np.ndarray, np.ndarray]:
        """Dense (H, S) as M x M float64 arrays (small systems only)."""
        M = self.M
        Hd = np.zeros((M, M))
        Sd = np.zeros((M, M))
        for I in range(self.n_block_rows):
            for k in range(self.row_ptr[I], self.row_ptr[I + 1]):
                J = int(self.col_idx[k])
                Hd[4 * I:4 * I + 4, 4 * J:4 * J + 4] = self.H[k]
                Sd[4 * I:4 * I + 4, 4 * J:4 * J + 4] = self.S[k]
        return Hd, Sd

    def scipy_bsr(self, which: str = "H"):
        import scipy.sparse as sp
        vals = self.H if which == "H" else self.S
        return sp.bsr_matrix((vals, self.col_idx, self.row_ptr), shape=(self.M, self.M))

    def permuted(self, perm: np.ndarray) -> "TBSystem":
        """Relabel atoms: new atom a is old atom perm[a]."""
        perm = np.asarray(perm, dtype=np.int64)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        rows, cols, hb, sb = [], [], [], []
        for a in range(perm.size):
            I = perm[a]
            for k in range(self.row_ptr[I], self.row_ptr[I + 1]):
                rows.append(a)
                cols.append(inv[self.col_idx[k]])
                hb.append(self.H[k])
                sb.append(self.S[k])
        rows = np.array(rows)
        cols = np.array(cols)
        order = np.lexsort((cols, rows))
        rp = np.zeros(perm.size + 1, np.int64)
        np.add.at(rp, rows + 1, 1)
        rp = np.cumsum(rp)
        mask = self.orbital_mask.reshape(-1, 4)[perm].reshape(-1).copy()
        return TBSystem(perm.size, rp, cols[order].astype(np.int32), np.array(hb)[order],
                        np.array(sb)[order], mask, self.n_electrons, None, self.lambda_min_S,
                        dict(self.meta))


def _sk_blocks(d: np.ndarray, V: np.ndarray) -> np.ndarray:
    """4x4 two-centre blocks for displacements d (P,3) and amplitudes V (P,4)=(sss,sps,pps,ppp)."""
    r = np.linalg.norm(d, axis=1)
    c = d / r[:, None]
    P = d.shape[0]
    B = np.zeros((P, 4, 4))
    B[:, 0, 0] = V[:, 0]
    B[:, 0, 1:] = c * V[:, 1:2]
    B[:, 1:, 0] = -c * V[:, 1:2]
    B[:, 1:, 1:] = (c[:, :, None] * c[:, None, :]) * (V[:, 2] - V[:, 3])[:, None, None] \
        + np.eye(3)[None] * V[:, 3][:, None, None]
    return B


def _sk_block_derivatives(d: np.ndarray, V: np.ndarray) -> np.ndarray:
    """d/d(d_x) of the blocks of _sk_blocks when every amplitude scales as r^-2.

    Returns (P, 3, 4, 4).  With c = d / r, g_p = (delta_px - c_p c_x) / r
    (= dc_p / dd_x) and dV/dd_x = -2 V c_x / r:
        dB/dd_x = -2 (c_x / r) B + [0, V_sps g_b; -V_sps g_a, (g_a c_b + c_a g_b)(V_pps - V_ppp)].
    """
    r = np.linalg.norm(d, axis=1)
    c = d / r[:, None]
    B = _sk_blocks(d, V)
    P = d.shape[0]
    out = np.zeros((P, 3, 4, 4))
    eye = np.eye(3)
    for x in range(3):
        g = (eye[x][None, :] - c * c[:, x:x + 1]) / r[:, None]          # (P, 3)
        D = -2.0 * (c[:, x] / r)[:, None, None] * B
        D[:, 0, 1:] += g * V[:, 1:2]
        D[:, 1:, 0] -= g * V[:, 1:2]
        D[:, 1:, 1:] += (g[:, :, None] * c[:, None, :] + c[:, :, None] * g[:, None, :]) \
            * (V[:, 2] - V[:, 3])[:, None, None]
        out[:, x] = D
    return out


def pair_amplitudes(si: np.ndarray, sj: np.ndarray, r: np.ndarray, params: dict) -> tuple[np.ndarray, np.ndarray]:
    """(V, coupled): Slater-Koster amplitudes V0 (r0 / r)^2 of each pair and whether the pair couples."""
    V = np.zeros((si.size, 4))
    keep = np.ones(si.size, bool)
    for (a, b), hop in params["hop"].items():
        sel = ((si == a) & (sj == b)) | ((si == b) & (sj == a))
        if hop is None:
            keep &= ~sel
            continue
        V[sel] = np.array(hop[:4])[None, :] * ((hop[4] / r[sel]) ** 2)[:, None]
    return V, keep


def build_tb_derivatives(sysm: "TBSystem", params: dict | None = None) -> tuple[np.ndarray, np.ndarray]:
    """dH, dS of shape (3, nnzb, 4, 4): block (I, J) differentiated with respect to
    the displacement d = R_J - R_I (minimum image) along x, y, z; on-site blocks 0.

    Aligned with sysm's blocks; couplings to padding orbitals stay 0.
    """
    p = params or carbon_params()
    s = sysm.structure
    rows = np.repeat(np.arange(sysm.n_block_rows), np.diff(sysm.row_ptr))
    cols = sysm.col_idx.astype(np.int64)
    off = np.nonzero(rows != cols)[0]
    i, j = rows[off], cols[off]
    d = min_image(s.positions[j] - s.positions[i], s.box)
    V, keep = pair_amplitudes(s.species[i], s.species[j], np.linalg.norm(d, axis=1), p)
    dH = np.zeros((3, sysm.nnzb, 4, 4))
    dS = np.zeros((3, sysm.nnzb, 4, 4))
    Dh = _sk_block_derivatives(d, V) * keep[:, None, None, None]
    Ds = _sk_block_derivatives(d, V * p["overlap_factor"]) * keep[:, None, None, None]
    real = sysm.orbital_mask.reshape(-1, 4).astype(bool)
    pad = ~(real[i][:, :, None] & real[j][:, None, :])                     # (P, 4, 4)
    for D in (Dh, Ds):
        D *= ~pad[:, None, :, :]
    dH[:, off] = np.moveaxis(Dh, 1, 0)
    dS[:, off] = np.moveaxis(Ds, 1, 0)
    return dH, dS


def neighbour_pairs(s: Structure, cutoff: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """All ordered pairs (i, j), i != j, closer than cutoff; displacement j - i (minimum image)."""
    from scipy.spatial import cKDTree
    if np.any(s.box <= 2.0 * cutoff):
        raise ValueError("box must exceed twice the cutoff for minimum-image neighbours")
    tree = cKDTree(s.positions, boxsize=s.box)
    pairs = tree.query_pairs(cutoff, output_type="ndarray")
    if pairs.size == 0:
        pairs = np.zeros((0, 2), np.int64)
    i = np.concatenate([pairs[:, 0], pairs[:, 1]]).astype(np.int64)
    j = np.concatenate([pairs[:, 1], pairs[:, 0]]).astype(np.int64)
    d = min_image(s.positions[j] - s.positions[i], s.box)
    return i, j, d


def build_tb(s: Structure, params: dict | None = None, check_spd: bool = True,
             spd_floor: float = 0.05) -> TBSystem:
    p = params or carbon_params()
    n = s.n_atoms
    i, j, d = neighbour_pairs(s, p["cutoff"])
    V, keep = pair_amplitudes(s.species[i], s.species[j], np.linalg.norm(d, axis=1), p)
    i, j, d, V = i[keep], j[keep], d[keep], V[keep]
    Hoff = _sk_blocks(d, V)
    Soff = _sk_blocks(d, V * p["overlap_factor"])
    real = np.array([p["real_orbitals"][int(x)] for x in s.species], dtype=np.uint8)  # (n,4)
    # zero couplings to padding orbitals (rows of i, columns of j)
    pad_i = (1 - real[i]).astype(bool)
    pad_j = (1 - real[j]).astype(bool)
    for B in (Hoff, Soff):
        B[pad_i[:, :, None] & np.ones((1, 1, 4), bool)] = 0.0
        B[np.ones((1, 4, 1), bool) & pad_j[:, None, :]] = 0.0
    Hon = np.zeros((n, 4, 4))
    Son = np.zeros((n, 4, 4))
    for sp_, e in p["onsite"].items():
        sel = s.species == sp_
        Hon[sel] = np.diag(e)
        Son[sel] = np.eye(4)
    rows = np.concatenate([np.arange(n), i])
    cols = np.concatenate([np.arange(n), j])
    Hall = np.concatenate([Hon, Hoff])
    Sall = np.concatenate([Son, Soff])
    order = np.lexsort((cols, rows))
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    sysm = TBSystem(
        n_block_rows=n,
        row_ptr=rp,
        col_idx=cols[order].astype(np.int32),
        H=np.ascontiguousarray(Hall[order]),
        S=np.ascontiguousarray(Sall[order]),
        orbital_mask=real.reshape(-1).copy(),
        n_electrons=float(sum(p["electrons"][int(x)] for x in s.species)),
        structure=s,
    )
    if check_spd:
        lam = lambda_min(sysm)
        sysm.lambda_min_S = lam
        if not lam > spd_floor:
            raise ValueError(f"overlap matrix not safely positive definite: lambda_min = {lam:.4g}")
    return sysm


def lambda_min(sysm: TBSystem) -> float:
    """Smallest eigenvalue of S (dense for small M, Lanczos otherwise)."""
    if sysm.M <= 4096:
        _, Sd = sysm.dense()
        return float(np.linalg.eigvalsh(Sd)[0])
    import scipy.sparse.linalg as sla
    S = sysm.scipy_bsr("S")   # 4x4-block products are faster than CSR's
    v0 = np.random.default_rng(1).standard_normal(S.shape[0])
    # a relative tolerance of 1e-5 is ample for the positivity check
    val = sla.eigsh(S, k=1, which="SA", v0=v0, tol=1e-5, return_eigenvectors=False)
    return float(val[0])


def config_c1(seed: int = 0) -> TBSystem:
    """64-atom jittered diamond (2x2x2 cubic cells), M = 256."""
    t = build_tb(diamond(2, seed=seed))
    t.meta.update(name="diamond-64", seed=seed)
    return t


def config_c2(seed: int = 0) -> TBSystem:
    """4,096-atom random-packed amorphous carbon at 3.0 g/cm^3, M = 16,384."""
    t = build_tb(amorphous_carbon(4096, seed=seed))
    t.meta.update(name="amorphous-4096", seed=seed)
    return t


def amorphous_system(n_atoms: int, seed: int = 0, check_spd: bool = True) -> TBSystem:
    """Amorphous carbon of n_atoms atoms.  check_spd=False skips the host eigensolve that
    refuses lambda_min(S) <= 0.05 (the library's setup runs its own SPD check)."""
    t = build_tb(amorphous_carbon(n_atoms, seed=seed), check_spd=check_spd)
    t.meta.update(name=f"amorphous-{n_atoms}", seed=seed)
    return t


def tiny_system(n_atoms: int, seed: int = 0, radius: float | None = None,
                box: float = 12.0) -> TBSystem:
    """A small carbon cluster in a large periodic box (no image interactions).

    Atoms are added at random inside a sphere with a 1.3 A minimum distance; the
    sphere is sized for about 0.1 atoms per cubic Angstrom so that most atoms
    have neighbours inside the 2.6 A cutoff.
    """
    rng = np.random.default_rng(seed)
    R = radius if radius is not None else (3.0 * n_atoms / (4.0 * np.pi * 0.1)) ** (1.0 / 3.0)
    pts: list[np.ndarray] = []
    tries = 0
    while len(pts) < n_atoms:
        tries += 1
        if tries > 100000:
            raise RuntimeError("tiny_system packing failed")
        x = rng.uniform(-R, R, 3)
        if x @ x > R * R:
            continue
        if all(np.sum((x - q) ** 2) >= 1.3 ** 2 for q in pts):
            pts.append(x)
    pos = np.array(pts) + box / 2.0
    s = Structure(pos, np.zeros(n_atoms, np.uint8), np.full(3, box))
    t = build_tb(s)
    t.meta.update(name=f"cluster-{n_atoms}", seed=seed)
    return t


def polymer_system(n_units: int, seed: int = 0, check_spd: bool = True, **kw) -> TBSystem:
    """A fluorene-like chain of n_units units (69 atoms each; see tbsynth.polymer).  check_spd=False
    skips the host eigensolve of S (the library's setup runs its own SPD check)."""
    from .polymer import polyfluorene
    t = build_tb(polyfluorene(n_units, seed=seed, **kw), check_spd=check_spd)
    t.meta.update(name=f"polyfluorene-{n_units}", seed=seed)
    return t


def tiny_hydrocarbon(n_atoms: int, n_hydrogen: int, seed: int = 0, box: float = 12.0) -> TBSystem:
    """A small cluster in which n_hydrogen of the atoms are hydrogen (one s
    orbital padded to a 4x4 block with three masked dummy orbitals)."""
    from .structures import HYDROGEN
    base = tiny_system(n_atoms, seed=seed, box=box)
    s = base.structure
    species = s.species.copy()
    rng = np.random.default_rng(seed + 1000)
    species[rng.choice(n_atoms, size=n_hydrogen, replace=False)] = HYDROGEN
    t = build_tb(Structure(s.positions.copy(), species, s.box.copy()))
    t.meta.update(name=f"hydrocarbon-{n_atoms}-{n_hydrogen}", seed=seed)
    return t
