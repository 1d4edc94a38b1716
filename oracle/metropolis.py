"""Single-spin Metropolis for the Ising / EA models (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

The paper compares TNMCMC with single-spin Metropolis (main text, "Sampling 3D
spin glasses"; SM III): a spin s_i is flipped with probability
min(1, exp(-beta dE)), dE = 2 s_i h_i, h_i = sum_j J_ij s_j. One sweep visits
the sites in two checkerboard half-sweeps (colour (x + y + z) mod 2), which
is a valid order of single-site updates because sites of one colour share no
bond; it needs a bipartite lattice (open axes or even periodic extents). The
uniform of site i in half-sweep c of sweep t is Philox purpose 7, index i,
slice c, axis 0, step t, chain.
"""
from __future__ import annotations

import numpy as np

from . import model, philox

PURPOSE_METRO = 7


def bipartite(dims, bc) -> bool:
    return all((not b) or (L % 2 == 0) for L, b in zip(dims, bc))


def local_field_int(spins: np.ndarray, J: np.ndarray, z: int, y: int, x: int) -> int:
    """h_i in units of 2^-20 (Ising values s = 1 - 2 index)."""
    Lz, Ly, Lx = spins.shape
    s = lambda zz, yy, xx: 1 - 2 * int(spins[zz % Lz, yy % Ly, xx % Lx])
    h = 0
    h += int(J[0, z, y, x]) * s(z, y, x + 1) + int(J[0, z, y, (x - 1) % Lx]) * s(z, y, x - 1)
    h += int(J[1, z, y, x]) * s(z, y + 1, x) + int(J[1, z, (y - 1) % Ly, x]) * s(z, y - 1, x)
    h += int(J[2, z, y, x]) * s(z + 1, y, x) + int(J[2, (z - 1) % Lz, y, x]) * s(z - 1, y, x)
    return h


def sweep(spins: np.ndarray, J: np.ndarray, beta: float, seed: int, t: int, chain: int) -> int:
    """One checkerboard Metropolis sweep of one chain in place; returns accepted flips."""
    Lz, Ly, Lx = spins.shape
    acc = 0
    for colour in (0, 1):
        # sites of one colour share no bond, so their updates commute: use the fields of the half-sweep start
        flips = []
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    if (x + y + z) % 2 != colour:
                        continue
                    si = 1 - 2 * int(spins[z, y, x])
                    dE = 2 * si * local_field_int(spins, J, z, y, x)       # units of 2^-20
                    i = (z * Ly + y) * Lx + x
                    u = philox.uniform(seed, PURPOSE_METRO, i, colour, 0, t, chain)
                    if u < np.exp(min(0.0, -beta * dE * model.J_SCALE)):
                        flips.append((z, y, x))
        for z, y, x in flips:
            spins[z, y, x] = 1 - spins[z, y, x]
        acc += len(flips)
    return acc
