"""Synthetic conjugated-polymer chains: fluorene-like units with two octyl side chains.

A stand-in for the poly-fluorene of the paper's eigenstate study (Section 2,
the poly-fluorene paragraph; the paper's structure model is not available).
Each unit is 69 atoms: a planar C13 backbone (two six-membered rings fused to
a five-membered ring, ring bonds 1.42 A), six ring hydrogens (C-H 1.09 A),
and two C8H17 chains on the bridging carbon, one above and one below the
ring plane (C-C 1.53 A zig-zag, C-H 1.09 A).  Units are bonded ring to ring
(1.48 A) along the chain axis, each turned about that axis by a seeded
torsion: mostly small, with occasional near-perpendicular twists that break
the pi conjugation, so that the frontier states localise on a few units.
End units carry a hydrogen on their free linking carbon.  Geometry only: no
arithmetic of the method lives here.
"""

from __future__ import annotations

import numpy as np

from .structures import CARBON, HYDROGEN, Structure, spatial_sort

RING = 1.42      # aromatic C-C, Angstrom
LINK = 1.48      # inter-unit C-C
SP3 = 1.53       # alkyl C-C
CH = 1.09        # C-H


def _regular_polygon_on_edge(p, q, n, away_from):
    """Vertices of the regular n-gon with edge p -> q, on the side away from `away_from`
    (in the xy plane); returns the n - 2 new vertices following q."""
    mid = 0.5 * (p + q)
    e = q - p
    side = np.linalg.norm(e)
    normal = np.array([-e[1], e[0], 0.0]) / side
    if np.dot(normal, mid - away_from) < 0:
        normal = -normal
    apothem = side / (2.0 * np.tan(np.pi / n))
    centre = mid + apothem * normal
    radius = side / (2.0 * np.sin(np.pi / n))
    a0 = np.arctan2(q[1] - centre[1], q[0] - centre[0])
    ap = np.arctan2(p[1] - centre[1], p[0] - centre[0])
    step = 2.0 * np.pi / n
    # go around from q away from p
    direction = 1.0 if np.isclose((ap - a0) % (2 * np.pi), (-step) % (2 * np.pi)) else -1.0
    out = []
    for k in range(1, n - 1):
        a = a0 + direction * k * step
        out.append(centre + radius * np.array([np.cos(a), np.sin(a), 0.0]))
    return out


def _backbone():
    """C13 backbone in the xy plane; returns (positions (13, 3), names)."""
    r5 = RING / (2.0 * np.sin(np.pi / 5))
    ang = {"C9": 90.0, "C9a": 162.0, "C4a": 234.0, "C4b": 306.0, "C8a": 18.0}
    P = {k: r5 * np.array([np.cos(np.radians(a)), np.sin(np.radians(a)), 0.0]) for k, a in ang.items()}
    c5 = np.zeros(3)
    a_ring = _regular_polygon_on_edge(P["C4a"], P["C9a"], 6, c5)      # C1, C2, C3, C4 after C9a
    P["C1"], P["C2"], P["C3"], P["C4"] = a_ring
    b_ring = _regular_polygon_on_edge(P["C8a"], P["C4b"], 6, c5)      # C5, C6, C7, C8 after C4b
    P["C5"], P["C6"], P["C7"], P["C8"] = b_ring
    names = ["C1", "C2", "C3", "C4", "C4a", "C4b", "C5", "C6", "C7", "C8", "C8a", "C9", "C9a"]
    return np.array([P[n] for n in names]), names


def _unit(rng):
    """One 69-atom unit in its own frame (chain axis x, ring plane xy), with the
    positions of the linking carbons C2 (left) and C7 (right)."""
    bb, names = _backbone()
    idx = {n: i for i, n in enumerate(names)}
    # orient the C2 -> C7 axis along +x
    axis = bb[idx["C7"]] - bb[idx["C2"]]
    th = -np.arctan2(axis[1], axis[0])
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    bb = bb @ R.T
    bb -= bb[idx["C2"]]
    pos = [p for p in bb]
    spec = [CARBON] * 13
    ring_a = [idx[n] for n in ("C1", "C2", "C3", "C4", "C4a", "C9a")]
    ring_b = [idx[n] for n in ("C4b", "C5", "C6", "C7", "C8", "C8a")]
    ca, cb = bb[ring_a].mean(axis=0), bb[ring_b].mean(axis=0)
    for n in ("C1", "C3", "C4"):
        d = bb[idx[n]] - ca
        pos.append(bb[idx[n]] + CH * d / np.linalg.norm(d))
        spec.append(HYDROGEN)
    for n in ("C5", "C6", "C8"):
        d = bb[idx[n]] - cb
        pos.append(bb[idx[n]] + CH * d / np.linalg.norm(d))
        spec.append(HYDROGEN)
    # two octyl chains on C9, above and below the plane, pointing away from the
    # rings: zig-zag C-C bonds b_k = cos(34) u +- sin(34) z (C-C-C 112 degrees),
    # hydrogens at 54.75 degrees either side of the C-C-C plane
    c9 = bb[idx["C9"]]
    out = c9 - 0.5 * (bb[idx["C9a"]] + bb[idx["C8a"]])
    out /= np.linalg.norm(out)
    th = np.radians(34.0)
    hh = np.radians(54.75)
    xax = np.array([1.0, 0.0, 0.0])
    for side in (+1.0, -1.0):
        u = np.cos(np.radians(35.0)) * np.array([0.0, 0.0, side]) + np.sin(np.radians(35.0)) * out
        u /= np.linalg.norm(u)
        z = np.cross(xax, u)    # zig-zag across the chain axis; hydrogens along it
        z /= np.linalg.norm(z)
        nrm = np.cross(u, z)
        bonds = [np.cos(th) * u + (1.0 if k % 2 == 0 else -1.0) * np.sin(th) * z for k in range(9)]
        prev = c9
        for k in range(8):
            cur = prev + SP3 * bonds[k]
            pos.append(cur)
            spec.append(CARBON)
            d = bonds[k] - bonds[k + 1]
            d /= np.linalg.norm(d)
            hs = [np.cos(hh) * d + np.sin(hh) * nrm, np.cos(hh) * d - np.sin(hh) * nrm]
            if k == 7:
                hs.append(bonds[k + 1])
            for h in hs:
                pos.append(cur + CH * h / np.linalg.norm(h))
                spec.append(HYDROGEN)
            prev = cur
    return np.array(pos), np.array(spec, dtype=np.uint8), idx["C2"], idx["C7"]


def polyfluorene(n_units: int, seed: int = 0, twist_small: float = 25.0, twist_break: float = 80.0,
                 p_break: float = 0.25, vacuum: float = 12.0) -> Structure:
    """A chain of n_units fluorene-like units (69 atoms each, plus two end hydrogens).

    Unit u + 1 is the mirror image of unit u (the bridging carbons alternate
    sides, so the chain runs straight on average), bonded C7 -> C2' along the
    outward para direction of the C7 ring, and turned about that bond by the
    seeded torsion.
    """
    rng = np.random.default_rng(seed)
    local, uspec, i2, i7 = _unit(rng)
    bb = local[:13]
    ring_a = bb[[0, 1, 2, 3, 4, 12]].mean(axis=0)
    ring_b = bb[[5, 6, 7, 8, 9, 10]].mean(axis=0)
    allpos, allspec = [], []
    E = None            # world basis (columns) of the current unit, at its C2
    origin = None
    for u in range(n_units):
        m = local.copy()
        ca, cb = ring_a.copy(), ring_b.copy()
        if u % 2:
            m[:, 1] *= -1.0
            ca[1] *= -1.0
            cb[1] *= -1.0
        dA = m[i2] - ca
        dA /= np.linalg.norm(dA)
        e3 = np.array([0.0, 0.0, 1.0])
        e2 = np.cross(e3, dA)
        B_loc = np.stack([dA, e2, e3], axis=1)           # local frame at C2 (columns)
        if u == 0:
            E1, E3 = np.array([-1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
            origin = np.zeros(3)
        else:
            E1 = -link_dir
            if rng.random() < p_break:
                tau = np.radians(rng.choice([-1.0, 1.0]) * rng.uniform(twist_break - 10, twist_break + 10))
            else:
                tau = np.radians(rng.normal(0.0, twist_small))
            # turn the previous plane normal about the bond axis by tau (Rodrigues)
            k = link_dir
            v = prev_normal
            E3 = v * np.cos(tau) + np.cross(k, v) * np.sin(tau) + k * np.dot(k, v) * (1 - np.cos(tau))
            E3 -= np.dot(E3, E1) * E1
            E3 /= np.linalg.norm(E3)
            origin = link_end
        E2 = np.cross(E3, E1)
        E = np.stack([E1, E2, E3], axis=1)
        W = (m - m[i2]) @ B_loc @ E.T + origin          # local -> world
        allpos.append(W)
        allspec.append(uspec)
        dB = m[i7] - cb
        dB /= np.linalg.norm(dB)
        link_dir = dB @ B_loc @ E.T
        link_dir /= np.linalg.norm(link_dir)
        link_end = W[i7] + LINK * link_dir
        prev_normal = E3
        if u == 0:   # hydrogen on the free C2 of the first unit
            dir0 = (m[i2] - ca) @ B_loc @ E.T
            allpos.append((W[i2] + CH * dir0 / np.linalg.norm(dir0))[None, :])
            allspec.append(np.array([HYDROGEN], np.uint8))
        if u == n_units - 1:
            allpos.append((W[i7] + CH * link_dir)[None, :])
            allspec.append(np.array([HYDROGEN], np.uint8))
    pos = np.concatenate(allpos)
    spec = np.concatenate(allspec)
    lo = pos.min(axis=0) - vacuum / 2
    pos = pos - lo
    box = pos.max(axis=0) + vacuum / 2
    return spatial_sort(Structure(pos, spec, box))
