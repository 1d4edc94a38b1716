"""Energy, slice geometry, held-spin fields and local weights (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Follows:
* the EA energy E(s) = -sum_<ij> J_ij s_i s_j (main text, "Sampling 3D spin
  glasses"; SM I.A) and the Potts energy E = -J sum delta(s_i, s_j)
  (main text, "Sampling the 3-state 3D Potts model");
* the TNMCMC-1 decomposition (SM II.A): a 2D layer is the active set, the two
  adjacent layers are its Markov blanket and act on it as a site-dependent
  field;
* the periodic-slice rule of the Potts experiments: the spins on one randomly
  chosen line of the slice are held fixed (reading R1); reading R2 also holds
  one random column, which leaves an open rectangle.

Geometry of a slice normal to axis ``a`` at position ``k``: the in-plane column
axis is ``(a + 1) % 3`` and the row axis is ``(a + 2) % 3``. Active rows are
``r = 1..m`` and active columns ``x = 0..Lc-1``; the rows form rings when the
column axis is periodic and no column is fixed.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from . import philox

J_FRAC_BITS = 20
J_SCALE = 2.0 ** -J_FRAC_BITS

MODEL_EA_PM, MODEL_EA_GAUSS, MODEL_POTTS = 0, 1, 2

FIX_R1 = 0   # one random line fixed on a periodic row axis
FIX_R2 = 1   # additionally one random column fixed on a periodic column axis


def pair_e(model: int, v: int, w: int) -> int:
    """Integer bond factor e(v, w): s(v) s(w) for Ising indices, delta for Potts."""
    if model == MODEL_POTTS:
        return 1 if v == w else 0
    return (1 - 2 * v) * (1 - 2 * w)


def pair_table(model: int, d: int) -> np.ndarray:
    return np.array([[pair_e(model, v, w) for w in range(d)] for v in range(d)], dtype=np.int64)


def full_energy_int(model: int, spins: np.ndarray, J: np.ndarray) -> int:
    """E(s) in units of 2**-20 as an exact integer: -sum over all 3 L^3 bond records of J e."""
    d = 3 if model == MODEL_POTTS else 2
    table = pair_table(model, d)
    s = spins.astype(np.int64)
    total = 0
    for a, ax in ((0, 2), (1, 1), (2, 0)):  # axis a is numpy axis 2 - a for [z, y, x] layout
        nb = np.roll(s, -1, axis=ax)
        total += int(np.sum(J[a].astype(np.int64) * table[s, nb]))
    return -total


@dataclass
class SliceGeom:
    """Where the active sites of one slice update sit in the 3D lattice."""

    axis: int
    k: int
    ra: int            # row axis
    ca: int            # column axis
    n_r: int
    n_c: int
    m: int             # active rows
    Lc: int            # active columns
    ring: bool         # active rows are periodic rings
    row0: int          # plane row of active row r is (row0 + r) % n_r ... see plane_row
    col0: int          # plane column of active column x is (col0 + x) % n_c
    y0: int            # fixed row (-1 if none)
    x0: int            # fixed column (-1 if none)

    def plane_row(self, r: int) -> int:
        return (self.row0 + r) % self.n_r

    def plane_col(self, x: int) -> int:
        return (self.col0 + x) % self.n_c

    def coord(self, r: int, x: int) -> Tuple[int, int, int]:
        """(x, y, z) lattice coordinates of active site (r, x)."""
        c = [0, 0, 0]
        c[self.axis] = self.k
        c[self.ra] = self.plane_row(r)
        c[self.ca] = self.plane_col(x)
        return c[0], c[1], c[2]


def slice_geometry(dims, bc, axis: int, k: int, fix_mode: int, seed: int, step: int, chain: int,
                   kind: int = 0) -> SliceGeom:
    """Active region of slice (axis, k); the fixed line/column are Philox draws (independent of the state).

    ``kind`` selects the Philox axis word axis | kind << 4 of the draws: 0 for TNMCMC-1 slices, 1 for
    TNMCMC-2 composite layers (oracle.superspin), so the two updates never share a draw."""
    ca, ra = (axis + 1) % 3, (axis + 2) % 3
    n_r, n_c = int(dims[ra]), int(dims[ca])
    axw = axis | (kind << 4)
    if bc[ra]:
        u = philox.uniform(seed, philox.PURPOSE_FIXED_ROW, 0, k, axw, step, chain)
        y0 = min(int(u * n_r), n_r - 1)
        m, row0 = n_r - 1, y0          # active row r (1..m) sits at plane row y0 + r
    else:
        y0, m, row0 = -1, n_r, -1      # active row r sits at plane row r - 1
    if bc[ca] and fix_mode == FIX_R2:
        u = philox.uniform(seed, philox.PURPOSE_FIXED_COL, 0, k, axw, step, chain)
        x0 = min(int(u * n_c), n_c - 1)
        Lc, col0, ring = n_c - 1, x0 + 1, False
    else:
        x0, Lc, col0, ring = -1, n_c, 0, bool(bc[ca])
    return SliceGeom(axis, k, ra, ca, n_r, n_c, m, Lc, ring, row0, col0, y0, x0)


def _site_index(dims, c):
    return c[2], c[1], c[0]  # numpy [z, y, x]


def _step(dims, c, a, delta):
    c = list(c)
    c[a] = (c[a] + delta) % int(dims[a])
    return tuple(c)


def tn_bonds(g: SliceGeom):
    """Bonds carried by the slice tensor network: (r, x) -> neighbour, kind, owner site of J."""
    hor = []   # (r, x, x2): bond between (r,x) and (r,x2), J stored at (r,x) along column axis
    for r in range(1, g.m + 1):
        for x in range(g.Lc - 1):
            hor.append((r, x, x + 1))
        if g.ring:
            hor.append((r, g.Lc - 1, 0))
    ver = [(r, x) for r in range(1, g.m) for x in range(g.Lc)]  # bond (r,x)-(r+1,x), J stored at (r,x) along row axis
    return hor, ver


def slice_terms(model: int, dims, spins: np.ndarray, J: np.ndarray, g: SliceGeom):
    """Integer energy terms of the active sites.

    Returns (Jh, Jv, hfield):
      Jh[r-1, x]   coupling of in-row bond x -> x+1 (wrap at x = Lc-1 on rings; else 0)
      Jv[r-1, x]   coupling of bond between rows r and r+1 (r < m; else 0)
      hfield[r-1, x, v]  sum over the bonds of (r, x) that the network does not carry
                         of J * e(v, neighbour spin): held layers, fixed line/column
                         and (zero-valued) open wraps.
    All in units of 2**-20, exact integers.
    """
    d = 3 if model == MODEL_POTTS else 2
    m, Lc = g.m, g.Lc
    Jh = np.zeros((m, Lc), dtype=np.int64)
    Jv = np.zeros((m, Lc), dtype=np.int64)
    hfield = np.zeros((m, Lc, d), dtype=np.int64)
    active = {}
    for r in range(1, m + 1):
        for x in range(Lc):
            active[g.coord(r, x)] = (r, x)
    carried = set()
    hor, ver = tn_bonds(g)
    for (r, x, x2) in hor:
        c = g.coord(r, x)
        Jh[r - 1, x] = J[(g.ca,) + _site_index(dims, c)]
        carried.add((c, g.ca))
    for (r, x) in ver:
        c = g.coord(r, x)
        Jv[r - 1, x] = J[(g.ra,) + _site_index(dims, c)]
        carried.add((c, g.ra))
    for (pos, (r, x)) in active.items():
        for a in range(3):
            # bond leaving pos along +a, stored at pos
            if (pos, a) not in carried:
                nb = _step(dims, pos, a, +1)
                jv = int(J[(a,) + _site_index(dims, pos)])
                sv = int(spins[_site_index(dims, nb)])
                for v in range(d):
                    hfield[r - 1, x, v] += jv * pair_e(model, v, sv)
            # bond arriving at pos from -a, stored at the neighbour
            nb = _step(dims, pos, a, -1)
            if (nb, a) not in carried:
                jv = int(J[(a,) + _site_index(dims, nb)])
                sv = int(spins[_site_index(dims, nb)])
                for v in range(d):
                    hfield[r - 1, x, v] += jv * pair_e(model, v, sv)
    return Jh, Jv, hfield


def active_spins(spins: np.ndarray, dims, g: SliceGeom) -> np.ndarray:
    out = np.zeros((g.m, g.Lc), dtype=np.int64)
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            out[r - 1, x] = spins[_site_index(dims, g.coord(r, x))]
    return out


def write_active(spins: np.ndarray, dims, g: SliceGeom, s: np.ndarray) -> None:
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            spins[_site_index(dims, g.coord(r, x))] = s[r - 1, x]


def slice_energy_int(model: int, g: SliceGeom, Jh, Jv, hfield, s: np.ndarray) -> int:
    """E of every bond touching the active set, for active configuration s [m, Lc] (exact integer)."""
    m, Lc = g.m, g.Lc
    e = 0
    for r in range(m):
        for x in range(Lc):
            v = int(s[r, x])
            e -= int(hfield[r, x, v])
            if x + 1 < Lc:
                e -= int(Jh[r, x]) * pair_e(model, v, int(s[r, x + 1]))
            elif g.ring:
                e -= int(Jh[r, x]) * pair_e(model, v, int(s[r, 0]))
            if r + 1 < m:
                e -= int(Jv[r, x]) * pair_e(model, v, int(s[r + 1, x]))
    return e


@dataclass
class SliceWeights:
    """Boltzmann factors of the slice network, each normalised to a maximum of 1.

    phi[r, x, v]       field factor exp(beta * h(v))
    psih[r, x, v, w]   in-row pair factor of the bond (r, x) -> (r, x+1) (wrap on rings)
    psiv[r, x, u, v]   pair factor between (r, x) in state u and (r+1, x) in state v
    log_scale          sum of the logs divided out by the normalisation
    """

    phi: np.ndarray
    psih: np.ndarray
    psiv: np.ndarray
    log_scale: float


def slice_weights(model: int, beta: float, g: SliceGeom, Jh, Jv, hfield) -> SliceWeights:
    d = hfield.shape[2]
    table = pair_table(model, d).astype(np.float64)
    m, Lc = g.m, g.Lc
    b = beta * J_SCALE
    hmax = hfield.max(axis=2, keepdims=True)
    phi = np.exp(b * (hfield - hmax).astype(np.float64))
    log_scale = float(b * hmax.astype(np.float64).sum())

    def pair(Jarr, present):
        out = np.ones((m, Lc, d, d))
        for r in range(m):
            for x in range(Lc):
                if not present(r, x):
                    continue
                jv = float(Jarr[r, x])
                ex = jv * table
                mx = ex.max()
                out[r, x] = np.exp(b * (ex - mx))
                nonlocal_scale[0] += b * mx
        return out

    nonlocal_scale = [0.0]
    psih = pair(Jh, lambda r, x: x + 1 < Lc or g.ring)
    psiv = pair(Jv, lambda r, x: r + 1 < m)
    return SliceWeights(phi, psih, psiv, log_scale + nonlocal_scale[0])
