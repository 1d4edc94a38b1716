"""Brute-force enumeration of slice distributions and small lattices (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

The exact conditional of the active set given the held spins (SM II.A,
P(s_a | s_h)) and its autoregressive factors P(s_i | s_<i) (main text,
"TNMCMC"; SM I.C) written out by summing exp(-beta E) over every
configuration. Used only to pin the network code on tiny slices.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import model


def slice_enumerate(mdl: int, g, Jh, Jv, hf, beta: float):
    """All configurations of the active set with their exact log-weights -beta*E (E up to a constant)."""
    d = hf.shape[2]
    n = g.m * g.Lc
    confs = np.array(list(itertools.product(range(d), repeat=n)), dtype=np.int64).reshape(-1, g.m, g.Lc)
    logw = np.array([-beta * model.J_SCALE * model.slice_energy_int(mdl, g, Jh, Jv, hf, s) for s in confs])
    return confs, logw


def log_sum_exp(a):
    mx = np.max(a)
    return float(mx + np.log(np.sum(np.exp(a - mx))))


def exact_logq(confs, logw, s):
    """log P(s | held) of one configuration."""
    idx = np.where((confs == s[None]).all(axis=(1, 2)))[0][0]
    return float(logw[idx] - log_sum_exp(logw))


def exact_conditionals(confs, logw, s):
    """P(s_i = v | s_<i) in raster order for a configuration s: array [m, Lc, d]."""
    m, Lc = s.shape
    d = int(confs.max()) + 1
    flat = confs.reshape(len(confs), -1)
    sf = s.reshape(-1)
    out = np.zeros((m * Lc, d))
    mask = np.ones(len(confs), dtype=bool)
    for i in range(m * Lc):
        lw = np.array([log_sum_exp(logw[mask & (flat[:, i] == v)]) if np.any(mask & (flat[:, i] == v)) else -np.inf
                       for v in range(d)])
        out[i] = np.exp(lw - log_sum_exp(lw))
        mask &= flat[:, i] == sf[i]
    return out.reshape(m, Lc, d)


def boltzmann_lattice(mdl: int, J: np.ndarray, beta: float, d: int):
    """Exact Boltzmann distribution of a whole (tiny) lattice: (states [N, Lz, Ly, Lx], probabilities)."""
    shape = J.shape[1:]
    n = int(np.prod(shape))
    states = np.array(list(itertools.product(range(d), repeat=n)), dtype=np.int8).reshape((-1,) + shape)
    E = np.array([model.full_energy_int(mdl, s, J) for s in states], dtype=np.float64) * model.J_SCALE
    lw = -beta * E
    p = np.exp(lw - lw.max())
    return states, p / p.sum(), E
