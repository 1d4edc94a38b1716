"""Seeded synthetic inputs for the slice-update path.

This module only draws random lattices, couplings and chain layouts. It holds
none of the method's arithmetic (no weights, contractions, sampling or
acceptance), so both the GPU path and the CPU oracle may use it.

Conventions shared by every consumer:

* A lattice has extents ``(Lx, Ly, Lz)`` and per-axis boundary flags
  ``bc = (bx, by, bz)`` with 1 = periodic, 0 = open (free).
* Spins are stored as state indices ``v`` in ``[0, d)`` as ``int8`` with
  layout ``[Lz][Ly][Lx]`` (x fastest). For Ising ``d = 2``, index 0 is spin
  +1 and index 1 is spin -1 (the basis-vector convention of SM I.C).
* Couplings are ``int32`` fixed point in units of ``2**-J_FRAC_BITS`` with
  layout ``[3][Lz][Ly][Lx]``: ``J[a][z][y][x]`` is the bond from site
  ``(x, y, z)`` to its neighbour one step along axis ``a`` (0 = x, 1 = y,
  2 = z), wrapping around the lattice. On an open axis the wrapping bond is
  stored as 0 and never contributes energy.
* The three models follow the paper's workloads: the +/-J Edwards-Anderson
  glass with ``P(J = +1) = 1/2`` (main text, "Sampling 3D spin glasses"),
  Gaussian couplings rounded to the fixed-point grid, and the ferromagnetic
  3-state Potts model with ``J = 1`` ("Sampling the 3-state 3D Potts model").
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

J_FRAC_BITS = 20
J_ONE = 1 << J_FRAC_BITS

MODEL_EA_PM = 0
MODEL_EA_GAUSS = 1
MODEL_POTTS = 2

MODEL_NAMES = {"ea_pm": MODEL_EA_PM, "ea_gauss": MODEL_EA_GAUSS, "potts": MODEL_POTTS}


def model_states(model: int, potts_q: int = 3) -> int:
    """Local dimension d of a model: 2 for Ising glasses, q for Potts."""
    return potts_q if model == MODEL_POTTS else 2


def make_couplings(model: int, dims: Sequence[int], bc: Sequence[int], seed: int) -> np.ndarray:
    """Draw one disorder instance: int32 ``[3, Lz, Ly, Lx]`` fixed-point couplings."""
    Lx, Ly, Lz = (int(v) for v in dims)
    rng = np.random.default_rng(np.uint64(seed) + np.uint64(0x5EED0000))
    shape = (3, Lz, Ly, Lx)
    if model == MODEL_EA_PM:
        J = np.where(rng.random(shape) < 0.5, J_ONE, -J_ONE).astype(np.int32)
    elif model == MODEL_EA_GAUSS:
        J = np.rint(rng.standard_normal(shape) * J_ONE).astype(np.int64)
        J = np.clip(J, -(1 << 30), (1 << 30)).astype(np.int32)
    elif model == MODEL_POTTS:
        J = np.full(shape, J_ONE, dtype=np.int32)
    else:
        raise ValueError(f"unknown model {model}")
    # open axes: zero the bond that wraps from the last layer to the first
    if not bc[0]:
        J[0, :, :, Lx - 1] = 0
    if not bc[1]:
        J[1, :, Ly - 1, :] = 0
    if not bc[2]:
        J[2, Lz - 1, :, :] = 0
    return J


def make_spins(n_chains: int, dims: Sequence[int], d: int, seed: int, cold: bool = False) -> np.ndarray:
    """Initial spins ``int8 [n_chains, Lz, Ly, Lx]``: uniform (hot) or all index 0 (cold, M = 1)."""
    Lx, Ly, Lz = (int(v) for v in dims)
    if cold:
        return np.zeros((n_chains, Lz, Ly, Lx), dtype=np.int8)
    rng = np.random.default_rng(np.uint64(seed) + np.uint64(0xC0FFEE))
    return rng.integers(0, d, size=(n_chains, Lz, Ly, Lx), dtype=np.int8)


@dataclass
class Workload:
    """A batch of chains sharing one lattice geometry and model.

    Chains are laid out instance-major: chain ``c`` has instance
    ``c // (n_beta * n_rep)``, inverse temperature index
    ``(c // n_rep) % n_beta`` and replica ``c % n_rep``. Replicas of the same
    (instance, beta) pair share couplings and differ only in their random
    stream, which is what the overlap q needs.
    """

    model: int
    dims: Tuple[int, int, int]
    bc: Tuple[int, int, int]
    chi: int
    betas: List[float]
    n_inst: int
    n_rep: int = 2
    potts_q: int = 3
    seed: int = 1
    couplings: np.ndarray = field(default=None, repr=False)  # [n_inst, 3, Lz, Ly, Lx]

    def __post_init__(self):
        if self.couplings is None:
            self.couplings = np.stack(
                [make_couplings(self.model, self.dims, self.bc, self.seed * 1000003 + i) for i in range(self.n_inst)]
            )

    @property
    def d(self) -> int:
        return model_states(self.model, self.potts_q)

    @property
    def n_chains(self) -> int:
        return self.n_inst * len(self.betas) * self.n_rep

    def chain_beta(self) -> np.ndarray:
        nb = len(self.betas)
        return np.array([self.betas[(c // self.n_rep) % nb] for c in range(self.n_chains)], dtype=np.float64)

    def chain_instance(self) -> np.ndarray:
        nb = len(self.betas)
        return np.array([c // (nb * self.n_rep) for c in range(self.n_chains)], dtype=np.int32)

    def initial_spins(self, cold: bool = False) -> np.ndarray:
        return make_spins(self.n_chains, self.dims, self.d, self.seed, cold=cold)


def linspace_betas(lo: float, hi: float, n: int) -> List[float]:
    return [float(b) for b in np.linspace(lo, hi, n)]
