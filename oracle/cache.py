"""Proposals from a cache of environments built for earlier held fields (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Follows the Conclusions: the slices are resampled under effective external
fields from their held neighbours, so contractions are frequent; one could
keep a list of "typical" fields so that contractions are needed only
occasionally, at the price of a lower acceptance. Reading:
* a cache entry per (chain, axis, slice) holds the fixed line / column drawn
  at build time and the environment stack E_1..E_m (SM I.B) contracted from
  the held spins at build time;
* a cached update takes the entry's geometry and environments and the row
  weights of the current held field: q_C(s | sigma) is the product over rows
  of p(s_r | s_<r) formed from phi(sigma), the in-plane pair factors and the
  cached E_r (the sampler of SM I.C with E_r replaced). It is a normalised
  distribution that depends on the held spins and the entry, not on the
  current slice, so the Metropolis-Hastings step of Eq. (1) with the exact
  energy keeps the chain exact as long as the cache does not change;
* the cache is frozen once built. Rebuilding it from a chain's own later
  state would make the proposal depend on the chain's past (the paper's
  "further approximations"); between rebuilds the chain is exact;
* sweeps mix cached and fresh updates: with fresh_every = k >= 1, sweep t
  builds environments afresh when t mod k = k - 1 and proposes from the
  cache otherwise; k = 0 always proposes from the cache. The choice does not
  depend on the state, and each of the two kernels leaves the Boltzmann
  distribution invariant. Draws of a cached update are those of the single
  update of the same (slice, step, chain).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import bmps, model, philox, update


@dataclass
class Entry:
    g: model.SliceGeom
    envs: List[List[np.ndarray]]


def build_entry(mdl: int, dims, bc, spins: np.ndarray, J: np.ndarray, beta: float, chi: int, axis: int, k: int,
                fix_mode: int, seed: int, step: int, chain: int) -> Entry:
    """Geometry drawn for (seed, step) and the environments of the current held spins."""
    g = model.slice_geometry(dims, bc, axis, k, fix_mode, seed, step, chain)
    Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
    w = model.slice_weights(mdl, beta, g, Jh, Jv, hf)
    envs, _ = bmps.environments(w, g.ring, chi)
    return Entry(g, envs)


def build(mdl: int, dims, bc, spins: np.ndarray, J_of_chain, betas, chi: int, fix_mode: int, seed: int, step: int,
          env_beta_factor: Optional[float] = None) -> Dict[Tuple[int, int, int], Entry]:
    """Entries for every chain, axis and slice from the current lattice spins [chains, Lz, Ly, Lx]."""
    cache = {}
    for c in range(spins.shape[0]):
        beta = float(betas[c]) * (1.0 if env_beta_factor is None else env_beta_factor)
        for axis in range(3):
            for k in range(int(dims[axis])):
                cache[(c, axis, k)] = build_entry(mdl, dims, bc, spins[c], J_of_chain(c), beta, chi, axis, k,
                                                  fix_mode, seed, step, c)
    return cache


def cached_update(mdl: int, dims, spins: np.ndarray, J: np.ndarray, beta: float, entry: Entry, seed: int,
                  step: int, chain: int, env_beta: Optional[float] = None,
                  write_back: bool = True) -> update.UpdateResult:
    """One slice update proposing from a cache entry; updates ``spins`` in place."""
    g = entry.g
    Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
    s_old = model.active_spins(spins, dims, g)
    w = model.slice_weights(mdl, beta if env_beta is None else env_beta, g, Jh, Jv, hf)
    u = update.site_uniforms(seed, g, chain, step)
    s_new, lq_new, ev1 = bmps.sample_slice(w, entry.envs, g.ring, uniforms=u)
    _, lq_old, ev2 = bmps.sample_slice(w, entry.envs, g.ring, forced=s_old)
    dE = model.slice_energy_int(mdl, g, Jh, Jv, hf, s_new) - model.slice_energy_int(mdl, g, Jh, Jv, hf, s_old)
    logA = (lq_old - lq_new) - beta * dE * model.J_SCALE
    u_mh = philox.uniform(seed, philox.PURPOSE_MH, 0, g.k, g.axis, step, chain)
    accept = bool(u_mh < np.exp(min(0.0, logA)))
    if accept and write_back:
        model.write_active(spins, dims, g, s_new)
    return update.UpdateResult(s_old, s_new, lq_new, lq_old, dE, accept, g.y0, g.x0, ev1 + ev2, float("nan"))


def sweep(mdl: int, dims, bc, spins: np.ndarray, J_of_chain, betas, chi: int, t: int, seed: int,
          cache: Dict[Tuple[int, int, int], Entry], fresh_every: int, fix_mode: int = model.FIX_R1,
          env_beta_factor: Optional[float] = None):
    """Sweep t (as update.sweep) proposing from the cache, except that with fresh_every = k >= 1 the
    sweeps t with t mod k = k - 1 build environments afresh (fresh_every = 0: always the cache)."""
    use = fresh_every == 0 or t % fresh_every != fresh_every - 1
    axis = t % 3
    n = int(dims[axis])
    acc = tot = 0
    for colour, ks in enumerate(update.colour_classes(n, bool(bc[axis]))):
        step = t * 4 + colour
        for c in range(spins.shape[0]):
            beta = float(betas[c])
            eb = None if env_beta_factor is None else beta * env_beta_factor
            for k in ks:
                if use:
                    res = cached_update(mdl, dims, spins[c], J_of_chain(c), beta, cache[(c, axis, k)], seed, step, c,
                                        env_beta=eb)
                else:
                    res = update.slice_update(mdl, dims, bc, spins[c], J_of_chain(c), beta, chi, axis, k, seed, step,
                                              c, fix_mode=fix_mode, env_beta=eb)
                acc += int(res.accept)
                tot += 1
    return acc, tot
