"""Pins of the oracle's cached-environment proposal (NEXT-4; the Conclusions' cache of typical fields).

* Built from the current held spins (open plane: no fixed-line draw), a cached update is the single
  update of Algorithm 2, draw for draw.
* Built from another state, q_C is still a normalised distribution over the slice (enumeration at a
  truncating chi), positive wherever the Boltzmann weight is.
* A chain proposing from a frozen cache built from an unrelated state samples the exact Boltzmann
  distribution (Eq. (1)); accepting every cached proposal does not (the test has power).
"""
import itertools

import numpy as np
import pytest

from oracle import bmps, cache, exact, model, observables, update
from paper_2509_23945_gb300 import inputs


def test_cache_of_current_state_equals_single_update():
    mdl, dims, bc = model.MODEL_EA_GAUSS, (4, 5, 3), (0, 0, 0)
    J = inputs.make_couplings(mdl, dims, bc, 3)
    spins = inputs.make_spins(1, dims, 2, 3)[0]
    for axis in range(3):
        for k in range(dims[axis]):
            e = cache.build_entry(mdl, dims, bc, spins, J, 1.1, 3, axis, k, model.FIX_R1, 99, 1, 0)
            a = cache.cached_update(mdl, dims, spins.copy(), J, 1.1, e, 5, 7, 0)
            b = update.slice_update(mdl, dims, bc, spins.copy(), J, 1.1, 3, axis, k, 5, 7, 0)
            assert np.array_equal(a.s_new, b.s_new) and a.accept == b.accept and a.dE == b.dE
            assert a.logq_new == b.logq_new and a.logq_old == b.logq_old


@pytest.mark.parametrize("dims,bc,fix,axis", [((3, 3, 3), (0, 0, 0), model.FIX_R1, 2),
                                              ((3, 4, 3), (1, 1, 1), model.FIX_R1, 0),
                                              ((4, 4, 3), (1, 1, 1), model.FIX_R2, 2)])
def test_cached_proposal_is_normalised(dims, bc, fix, axis):
    mdl, beta, chi = model.MODEL_EA_PM, 1.2, 2
    J = inputs.make_couplings(mdl, dims, bc, 5)
    built_from = inputs.make_spins(1, dims, 2, 1)[0]
    now = inputs.make_spins(1, dims, 2, 2)[0]
    e = cache.build_entry(mdl, dims, bc, built_from, J, beta, chi, axis, 1, fix, 4, 0, 0)
    g = e.g
    Jh, Jv, hf = model.slice_terms(mdl, dims, now, J, g)
    w = model.slice_weights(mdl, beta, g, Jh, Jv, hf)
    total = 0.0
    for flat in itertools.product(range(2), repeat=g.m * g.Lc):
        s = np.array(flat).reshape(g.m, g.Lc)
        _, lq, _ = bmps.sample_slice(w, e.envs, g.ring, forced=s)
        assert np.isfinite(lq)
        total += np.exp(lq)
    assert abs(total - 1.0) < 1e-12


def _chain(chi, fresh_every, n_sweeps=2400, seed=8, burn=30, plant=None):
    mdl, dims, bc, beta = model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(1, dims, 2, seed)
    other = inputs.make_spins(1, dims, 2, seed + 100)     # the cache is built from an unrelated state
    C = cache.build(mdl, dims, bc, other, lambda c: J, [beta], chi, model.FIX_R1, 17, 0, env_beta_factor=0.6)
    visits, energies = [], []
    acc = tot = 0
    for t in range(n_sweeps):
        a, b = cache.sweep(mdl, dims, bc, spins, lambda c: J, [beta], chi, t, seed, C, fresh_every)
        acc, tot = acc + a, tot + b
        if t >= burn:
            visits.append(spins[0].copy())
            energies.append(model.full_energy_int(mdl, spins[0], J) * model.J_SCALE)
    states, p, _ = exact.boltzmann_lattice(mdl, J, beta, 2)
    index = {s.tobytes(): i for i, s in enumerate(states)}
    counts = np.zeros(len(states))
    for v in visits:
        counts[index[v.tobytes()]] += 1
    tv = 0.5 * np.abs(counts / counts.sum() - p).sum()
    tau, _, _ = observables.tau_int(np.array(energies))
    n_eff = max(len(visits) / (2 * max(tau, 0.5)), 1.0)
    rng = np.random.default_rng(0)
    null = [0.5 * np.abs(rng.multinomial(int(n_eff), p) / int(n_eff) - p).sum() for _ in range(200)]
    return tv, float(np.quantile(null, 0.999)), acc / tot


@pytest.mark.parametrize("chi,fresh_every", [(1, 0), (4, 0), (1, 3)])
def test_frozen_cache_chain_matches_boltzmann(chi, fresh_every):
    """fresh_every = 0: every update proposes from the frozen cache (built at 0.6 beta from another state)."""
    tv, bound, acc = _chain(chi, fresh_every)
    assert tv < bound, (tv, bound, acc)
    assert 0.0 < acc < 1.0


def test_planted_acceptance_without_ratio_fails(monkeypatch):
    real_exp = np.exp

    def always_accept(x):
        return real_exp(0.0) if np.ndim(x) == 0 else real_exp(x)

    monkeypatch.setattr(cache.np, "exp", always_accept)
    tv, bound, _ = _chain(1, 0)
    monkeypatch.undo()
    assert tv > bound, (tv, bound)
