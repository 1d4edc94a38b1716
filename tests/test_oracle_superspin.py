"""Pins of the oracle's TNMCMC-2 composite-layer update (SM II.B) against brute force.

Nothing here reuses the composite layer's own bookkeeping as its check:
* energies against a full-lattice recomputation (every bond record of the lattice);
* at exact chi, q(s) of every superspin configuration against exp(-beta E_full(s)) normalised by
  enumeration, and log Z against the same sum;
* with the couplings between the two layers set to zero the composite network is the product of
  two independent TNMCMC-1 slices (whose oracle is pinned on its own);
* a chain of composite updates samples the exact Boltzmann distribution of a small lattice.
"""
import itertools

import numpy as np
import pytest

from oracle import exact, model, observables, superspin, update
from paper_2509_23945_gb300 import inputs

# model, dims (Lx, Ly, Lz), bc, axis, k, fix_mode, beta
CASES = [
    (model.MODEL_EA_PM, (3, 2, 4), (0, 0, 1), 2, 1, model.FIX_R1, 1.0),      # open plane, n_a = 4
    (model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 2, 0, model.FIX_R1, 0.9),      # the whole lattice
    (model.MODEL_EA_GAUSS, (3, 3, 3), (1, 1, 1), 0, 1, model.FIX_R1, 1.2),   # R1 ring rows, n_a = 3
    (model.MODEL_EA_PM, (4, 3, 3), (1, 1, 1), 2, 2, model.FIX_R2, 1.1),      # R2, composite wraps (2, 0)
    (model.MODEL_EA_GAUSS, (2, 3, 2), (1, 0, 0), 0, 1, model.FIX_R1, 1.3),   # n_a = 2 periodic: two bonds
]


def _lattice(case, seed=4):
    mdl, dims, bc, axis, k, fix, beta = case
    J = inputs.make_couplings(mdl, dims, bc, seed)
    spins = inputs.make_spins(1, dims, 2, seed)[0]
    g = superspin.geometry(dims, bc, axis, k, fix, 9, 6, 0)
    return mdl, dims, bc, axis, k, fix, beta, J, spins, g


def _rest_energy(mdl, dims, spins, J, g):
    """-sum of J e over the bond records with neither end in the composite layer (full lattice)."""
    act = set()
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            for layer in (0, 1):
                act.add(superspin.layer_coord(dims, g, r, x, layer))
    e = 0
    for c in itertools.product(*(range(int(n)) for n in dims)):
        for a in range(3):
            q = model._step(dims, c, a, +1)
            if c in act or q in act:
                continue
            e -= int(J[a, c[2], c[1], c[0]]) * model.pair_e(mdl, int(spins[c[2], c[1], c[0]]),
                                                             int(spins[q[2], q[1], q[0]]))
    return e


def _with(spins, dims, g, s):
    out = spins.copy()
    superspin.write_superspins(out, dims, g, s)
    return out


@pytest.mark.parametrize("case", CASES)
def test_composite_energy_equals_full_lattice(case):
    mdl, dims, bc, axis, k, fix, beta, J, spins, g = _lattice(case)
    eh, ev, hf = superspin.terms(mdl, dims, spins, J, g)
    rest = _rest_energy(mdl, dims, spins, J, g)
    rng = np.random.default_rng(2)
    for _ in range(12):
        s = rng.integers(0, 4, size=(g.m, g.Lc))
        full = model.full_energy_int(mdl, _with(spins, dims, g, s), J)
        assert superspin.energy_int(g, eh, ev, hf, s) + rest == full


def _enumerate(mdl, dims, spins, J, g, beta):
    n = g.m * g.Lc
    confs = np.array(list(itertools.product(range(4), repeat=n)), dtype=np.int64).reshape(-1, g.m, g.Lc)
    E = np.array([model.full_energy_int(mdl, _with(spins, dims, g, s), J) for s in confs], dtype=np.float64)
    return confs, -beta * model.J_SCALE * E


@pytest.mark.parametrize("case", CASES)
def test_exact_chi_q_and_logz_equal_enumeration(case):
    mdl, dims, bc, axis, k, fix, beta, J, spins, g = _lattice(case)
    eh, ev, hf = superspin.terms(mdl, dims, spins, J, g)
    w = superspin.weights(beta, g, eh, ev, hf)
    envs, logz = superspin.bmps.environments(w, g.ring, 16)
    confs, logw = _enumerate(mdl, dims, spins, J, g, beta)
    lse = exact.log_sum_exp(logw)
    # log Z of the composite network: the Boltzmann sum with the rest of the lattice divided out
    rest = _rest_energy(mdl, dims, spins, J, g)
    assert abs(logz + w.log_scale - (lse + beta * model.J_SCALE * rest)) < 1e-10 * max(1.0, abs(lse))
    rng = np.random.default_rng(3)
    picks = rng.choice(len(confs), size=min(24, len(confs)), replace=False)
    eps = superspin.bmps.FLOOR_EPS
    for i in picks:
        probs = np.zeros((g.m, g.Lc, 4))
        _, lq, nev = superspin.bmps.sample_slice(w, envs, g.ring, forced=confs[i], probs_out=probs)
        assert nev == 0
        # exact raster-order conditionals with the floor rule of the sampler, (P + eps) / (1 + d eps)
        P = (exact.exact_conditionals(confs, logw, confs[i]) + eps) / (1.0 + 4 * eps)
        assert np.max(np.abs(probs - P)) < 1e-12
        want = float(np.sum(np.log(np.take_along_axis(P, confs[i][..., None], axis=2))))
        assert abs(lq - want) < 1e-9
        # and without the floor the product is the Boltzmann probability of s
        assert abs(want - (logw[i] - lse)) < g.m * g.Lc * eps * np.exp(lse - logw[i]) + 1e-9


@pytest.mark.parametrize("case", CASES)
def test_exact_chi_accepts_with_unit_ratio(case):
    mdl, dims, bc, axis, k, fix, beta, J, spins, g = _lattice(case)
    before = spins.copy()
    res = superspin.composite_update(mdl, dims, bc, spins, J, beta, 16, axis, k, 11, 6, 0, fix_mode=fix)
    logA = (res.logq_old - res.logq_new) - beta * res.dE * model.J_SCALE
    # at exact chi q = P(s | held) up to the sampler's floor, which moves log p(v) by at most
    # eps / p(v) per site (main text: exact conditionals give unit acceptance)
    eh, ev, hf = superspin.terms(mdl, dims, before, J, g)
    w = superspin.weights(beta, g, eh, ev, hf)
    envs, _ = superspin.bmps.environments(w, g.ring, 16)
    bound = 1e-12
    for s in (res.s_old, res.s_new):
        probs = np.zeros((g.m, g.Lc, 4))
        superspin.bmps.sample_slice(w, envs, g.ring, forced=s, probs_out=probs)
        bound += float(np.sum(superspin.bmps.FLOOR_EPS / np.take_along_axis(probs, s[..., None], axis=2)))
    assert abs(logA) < 2 * bound and res.accept
    # the move writes both layers and dE is the full-lattice energy change
    assert model.full_energy_int(mdl, spins, J) - model.full_energy_int(mdl, before, J) == res.dE
    g2 = superspin.geometry(dims, bc, axis, k, fix, 11, 6, 0)
    assert np.array_equal(superspin.active_superspins(spins, dims, g2), res.s_new)


def test_uncoupled_layers_factorise_into_two_slices():
    """With zero couplings between layers k and k+1 the composite network is the product of the
    TNMCMC-1 networks of slices k and k+1 (open plane: no fixed line), so log Z adds at exact chi."""
    mdl, dims, bc, axis, k = model.MODEL_EA_GAUSS, (3, 2, 5), (0, 0, 1), 2, 2
    J = inputs.make_couplings(mdl, dims, bc, 8)
    J[axis, k] = 0                      # bonds from layer k to layer k+1 (z = 2 -> 3)
    spins = inputs.make_spins(1, dims, 2, 8)[0]
    beta = 1.1
    sup = superspin.composite_update(mdl, dims, bc, spins.copy(), J, beta, 16, axis, k, 3, 0, 0, write_back=False)
    a = update.slice_update(mdl, dims, bc, spins.copy(), J, beta, 16, axis, k, 3, 0, 0, write_back=False)
    b = update.slice_update(mdl, dims, bc, spins.copy(), J, beta, 16, axis, k + 1, 3, 0, 0, write_back=False)
    assert abs(sup.logz - (a.logz + b.logz)) < 1e-10 * abs(sup.logz)


def test_composite_classes_are_independent_and_cover():
    for n in range(2, 9):
        for periodic in (0, 1):
            covered = set()
            for offset in (0, 1):
                classes = superspin.composite_classes(n, bool(periodic), offset)
                for cls in classes:
                    for k in cls:
                        assert periodic or k + 1 < n
                        covered |= {k, (k + 1) % n}
                    # no composite of a class touches another's layers or blanket
                    for k1, k2 in itertools.combinations(cls, 2):
                        own1 = {k1, (k1 + 1) % n}
                        reach2 = {(k2 + dk) % n if periodic else k2 + dk for dk in (-1, 0, 1, 2)}
                        assert not own1 & reach2, (n, periodic, offset, cls)
                if periodic and n % 2 == 0:
                    layers = sorted(l for cls in classes for k in cls for l in (k, (k + 1) % n))
                    assert layers == list(range(n))
            assert covered == set(range(n))


def _tv_chain(chi, ebf, n_sweeps=2400, seed=6, burn=30):
    mdl, dims, bc, beta = model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(1, dims, 2, seed)
    visits, energies = [], []
    for t in range(n_sweeps):
        superspin.sweep(mdl, dims, bc, spins, lambda c: J, [beta], chi, t, seed, env_beta_factor=ebf)
        if t >= burn and (t // 3) % 2 == 0:      # offset-1 sweeps of an extent-2 open axis move nothing
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
    return tv, float(np.quantile(null, 0.999))


@pytest.mark.parametrize("chi,ebf", [(1, None), (1, 0.6)])
def test_composite_chain_matches_boltzmann_2x2x2(chi, ebf):
    """Composite updates at a truncating chi (1 < 4) and with a proposal built at 0.6 beta keep the
    exact Boltzmann distribution of a 2x2x2 free-BC lattice (Eq. (1) corrects any proposal)."""
    tv, bound = _tv_chain(chi, ebf)
    assert tv < bound, (tv, bound)


def test_planted_wrong_acceptance_fails_composite_chain(monkeypatch):
    """Accepting every composite proposal samples the proposal, not Boltzmann: the test above has power."""
    real_exp = np.exp

    def always_accept(x):
        return real_exp(0.0) if np.ndim(x) == 0 else real_exp(x)

    monkeypatch.setattr(superspin.np, "exp", always_accept)
    tv, bound = _tv_chain(1, 0.3)
    monkeypatch.undo()
    assert tv > bound, (tv, bound)


@pytest.mark.slow
@pytest.mark.parametrize("bc,chi", [((1, 1, 0), 4), ((1, 1, 0), 1)])
def test_composite_chain_state_histogram_3x3x2(bc, chi):
    """3x3x2 lattice (2^18 states), x and y periodic: composite updates along x and y leave one layer of
    three out and fix a line of superspins (R1, ring rows of D_h = 16); along z the composite is the whole
    lattice. The visited states, lumped by energy, by exact probability and by a random partition (flip
    pairs in one bin), match exact enumeration (chi-squared at the 0.999 level), at exact chi (4) and
    truncating (1)."""
    import boltzmann_check
    mdl, dims, beta, n_chains, n_sweeps = model.MODEL_EA_PM, (3, 3, 2), 0.7, 8, 240
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(n_chains, dims, 2, 9)
    snaps = []
    acc = tot = 0
    for t in range(n_sweeps + 24):
        a, b = superspin.sweep(mdl, dims, bc, spins, lambda c: J, [beta] * n_chains, chi, t, 9)
        acc, tot = acc + a, tot + b
        if t >= 24 and b > 0:
            snaps.append(spins.copy())
    _, p, E = exact.boltzmann_lattice(mdl, J, beta, 2)
    idx = boltzmann_check.state_index(np.array(snaps).reshape(-1, *dims[::-1])).reshape(len(snaps), n_chains)
    res = boltzmann_check.lumped_chi2(idx, p, E, flip_invariant=True)
    for name, (chi2, thr, dof, tau) in res.items():
        assert chi2 < thr, (name, chi2, thr, dof, tau, acc / tot)
    if chi == 4:
        assert acc / tot > 0.999
