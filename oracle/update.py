"""One TNMCMC-1 slice update and the sweep schedule (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Follows Algorithm 2 (TNMCMC-1) and SM II.A:
  1. build the slice network from the held layers and couplings;
  2. contract it by boundary MPS and draw a candidate slice s' with q(s');
  3. evaluate q(s) of the current slice with the same environments;
  4. accept with the Metropolis-Hastings probability of Eq. (1),
     A = min{1, q(s) exp(-beta E(s')) / (q(s') exp(-beta E(s)))}.
     (Algorithm 2 prints the ratio with the primes swapped; Eq. (1) and the
     acceptance formula of SM II.A agree with each other and are used.)
A rejected proposal keeps the current slice.

The sweep cycles the slice normal through x, y, z (SM II.A) and updates all
slices of one colour class at once (the odd/even parallel update of SM II.A
and SM III.D): two classes for even or open axes, three for odd periodic axes.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import bmps, model, philox


@dataclass
class UpdateResult:
    s_old: np.ndarray
    s_new: np.ndarray
    logq_new: float
    logq_old: float
    dE: int
    accept: bool
    y0: int
    x0: int
    events: int
    logz: float


def site_uniforms(seed, g: model.SliceGeom, chain: int, step: int, purpose=philox.PURPOSE_SITE) -> np.ndarray:
    u = np.zeros((g.m, g.Lc))
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            u[r - 1, x] = philox.uniform(seed, purpose, (r - 1) * g.Lc + x, g.k, g.axis, step, chain)
    return u


def slice_update(mdl: int, dims, bc, spins: np.ndarray, J: np.ndarray, beta: float, chi: int,
                 axis: int, k: int, seed: int, step: int, chain: int,
                 fix_mode: int = model.FIX_R1, env_beta: Optional[float] = None,
                 write_back: bool = True) -> UpdateResult:
    """TN proposal + exact-energy MH for slice (axis, k) of one chain; updates ``spins`` in place."""
    g = model.slice_geometry(dims, bc, axis, k, fix_mode, seed, step, chain)
    Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
    s_old = model.active_spins(spins, dims, g)
    w = model.slice_weights(mdl, beta if env_beta is None else env_beta, g, Jh, Jv, hf)
    envs, logz = bmps.environments(w, g.ring, chi)
    u = site_uniforms(seed, g, chain, step)
    s_new, lq_new, ev1 = bmps.sample_slice(w, envs, g.ring, uniforms=u)
    _, lq_old, ev2 = bmps.sample_slice(w, envs, g.ring, forced=s_old)
    dE = model.slice_energy_int(mdl, g, Jh, Jv, hf, s_new) - model.slice_energy_int(mdl, g, Jh, Jv, hf, s_old)
    logA = (lq_old - lq_new) - beta * dE * model.J_SCALE
    u_mh = philox.uniform(seed, philox.PURPOSE_MH, 0, k, axis, step, chain)
    accept = bool(u_mh < np.exp(min(0.0, logA)))
    if accept and write_back:
        model.write_active(spins, dims, g, s_new)
    return UpdateResult(s_old, s_new, lq_new, lq_old, dE, accept, g.y0, g.x0, ev1 + ev2, logz + w.log_scale)


@dataclass
class MultiResult:
    s_old: np.ndarray
    s_final: np.ndarray
    logq_old: float
    logq_final: float
    dE: int              # E(final) - E(old), units of 2^-20
    accepted: int        # accepted proposals out of K
    y0: int
    x0: int


def slice_update_k(mdl: int, dims, bc, spins: np.ndarray, J: np.ndarray, beta: float, chi: int,
                   axis: int, k: int, seed: int, step: int, chain: int, n_prop: int,
                   fix_mode: int = model.FIX_R1, env_beta: Optional[float] = None,
                   write_back: bool = True) -> MultiResult:
    """n_prop proposals from one environment build (main text: "draw a batch of candidate samples";
    the environments E_r depend only on the held spins, so every proposal of the batch is drawn from
    the same q). The batch runs as an independence-sampler chain on the slice: proposal j is accepted
    against the current slice with Eq. (1), whose log q and energy then move to the accepted
    candidate. Proposal 0 uses the draws of slice_update, so n_prop = 1 is that update."""
    g = model.slice_geometry(dims, bc, axis, k, fix_mode, seed, step, chain)
    Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
    s_old = model.active_spins(spins, dims, g)
    w = model.slice_weights(mdl, beta if env_beta is None else env_beta, g, Jh, Jv, hf)
    envs, _ = bmps.environments(w, g.ring, chi)
    _, lq_cur, _ = bmps.sample_slice(w, envs, g.ring, forced=s_old)
    lq_old = lq_cur
    e_old = model.slice_energy_int(mdl, g, Jh, Jv, hf, s_old)
    s_cur, e_cur = s_old.copy(), e_old
    n_sites = g.m * g.Lc
    accepted = 0
    for j in range(n_prop):
        if j == 0:
            u = site_uniforms(seed, g, chain, step)
            u_mh = philox.uniform(seed, philox.PURPOSE_MH, 0, k, axis, step, chain)
        else:
            u = np.zeros((g.m, g.Lc))
            for r in range(1, g.m + 1):
                for x in range(g.Lc):
                    u[r - 1, x] = philox.uniform(seed, philox.PURPOSE_SITE_K, (j - 1) * n_sites + (r - 1) * g.Lc + x,
                                                 k, axis, step, chain)
            u_mh = philox.uniform(seed, philox.PURPOSE_MH_K, j - 1, k, axis, step, chain)
        s_new, lq_new, _ = bmps.sample_slice(w, envs, g.ring, uniforms=u)
        e_new = model.slice_energy_int(mdl, g, Jh, Jv, hf, s_new)
        logA = (lq_cur - lq_new) - beta * (e_new - e_cur) * model.J_SCALE
        if u_mh < np.exp(min(0.0, logA)):
            s_cur, lq_cur, e_cur = s_new, lq_new, e_new
            accepted += 1
    if write_back:
        model.write_active(spins, dims, g, s_cur)
    return MultiResult(s_old, s_cur, lq_old, lq_cur, e_cur - e_old, accepted, g.y0, g.x0)


def colour_classes(n: int, periodic: bool) -> List[List[int]]:
    """Slices of one axis grouped so that no two in a group are neighbours (Markov blanket)."""
    if periodic and n % 2 == 1 and n > 1:
        return [list(range(0, n - 1, 2)), list(range(1, n - 1, 2)), [n - 1]]
    return [list(range(0, n, 2)), list(range(1, n, 2))]


def sweep(mdl: int, dims, bc, spins: np.ndarray, J_of_chain, betas, chi: int, t: int, seed: int,
          fix_mode: int = model.FIX_R1, env_beta_factor: Optional[float] = None, n_prop: int = 1):
    """One sweep t: axis t mod 3, every colour class in order, every chain. Returns accept counts
    (accepted proposals and proposals; n_prop proposals per slice from one environment build)."""
    axis = t % 3
    n = int(dims[axis])
    acc, tot = 0, 0
    for colour, ks in enumerate(colour_classes(n, bool(bc[axis]))):
        step = t * 4 + colour
        for c in range(spins.shape[0]):
            beta = float(betas[c])
            eb = None if env_beta_factor is None else beta * env_beta_factor
            for k in ks:
                if n_prop == 1:
                    res = slice_update(mdl, dims, bc, spins[c], J_of_chain(c), beta, chi, axis, k, seed, step, c,
                                       fix_mode=fix_mode, env_beta=eb)
                    acc += int(res.accept)
                else:
                    res = slice_update_k(mdl, dims, bc, spins[c], J_of_chain(c), beta, chi, axis, k, seed, step, c,
                                         n_prop, fix_mode=fix_mode, env_beta=eb)
                    acc += res.accepted
                tot += n_prop
    return acc, tot
