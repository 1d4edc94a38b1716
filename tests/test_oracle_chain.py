"""Chain-level pins: the oracle's TNMCMC-1 chain samples the exact Boltzmann distribution.

MH with the acceptance of Eq. (1) leaves the Boltzmann distribution invariant
for any positive proposal, so the stationary histogram must match exact
enumeration at a truncating chi, at exact chi and with a deliberately
mismatched proposal. A planted mistake (acceptance that ignores the proposal
ratio) must fail the same test, which shows the test has power.
"""
import numpy as np
import pytest

import boltzmann_check
from oracle import exact, model, observables, update
from paper_2509_23945_gb300 import inputs


def _run_chain(mdl, dims, bc, beta, chi, n_sweeps, seed, env_beta_factor=None, burn=20):
    d = 3 if mdl == model.MODEL_POTTS else 2
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(1, dims, d, seed)
    visits = []
    energies = []
    acc = tot = 0
    for t in range(n_sweeps):
        a, b = update.sweep(mdl, dims, bc, spins, lambda c: J, [beta], chi, t, seed,
                            env_beta_factor=env_beta_factor)
        acc += a
        tot += b
        if t >= burn:
            visits.append(spins[0].copy())
            energies.append(model.full_energy_int(mdl, spins[0], J) * model.J_SCALE)
    return J, visits, np.array(energies), acc / tot


def _tv_test(mdl, dims, beta, visits, energies, J):
    d = 3 if mdl == model.MODEL_POTTS else 2
    states, p, _ = exact.boltzmann_lattice(mdl, J, beta, d)
    index = {s.tobytes(): i for i, s in enumerate(states)}
    counts = np.zeros(len(states))
    for v in visits:
        counts[index[v.tobytes()]] += 1
    emp = counts / counts.sum()
    tv = 0.5 * np.abs(emp - p).sum()
    tau, _, _ = observables.tau_int(energies)
    n_eff = max(len(visits) / (2 * max(tau, 0.5)), 1.0)
    # null distribution of TV for n_eff independent exact draws
    rng = np.random.default_rng(0)
    null = [0.5 * np.abs(rng.multinomial(int(n_eff), p) / int(n_eff) - p).sum() for _ in range(200)]
    return tv, float(np.quantile(null, 0.999)), tau


@pytest.mark.parametrize("chi,ebf", [(1, None), (4, None), (1, 0.7)])
def test_chain_matches_boltzmann_2x2x2(chi, ebf):
    mdl, dims, bc, beta = model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    J, visits, energies, acc = _run_chain(mdl, dims, bc, beta, chi, 3000, seed=5, env_beta_factor=ebf)
    tv, bound, tau = _tv_test(mdl, dims, beta, visits, energies, J)
    assert tv < bound, (tv, bound, tau, acc)


def test_planted_wrong_acceptance_fails(monkeypatch):
    """Accepting every proposal (no q ratio, no energy) samples the proposal, not Boltzmann."""
    real_exp = np.exp

    def always_accept(x):
        return real_exp(0.0) if np.ndim(x) == 0 else real_exp(x)

    monkeypatch.setattr(update.np, "exp", always_accept)
    mdl, dims, bc, beta = model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    J, visits, energies, acc = _run_chain(mdl, dims, bc, beta, 1, 3000, seed=5, env_beta_factor=0.3)
    monkeypatch.undo()
    tv, bound, tau = _tv_test(mdl, dims, beta, visits, energies, J)
    assert tv > bound, (tv, bound)


_EXACT = {}


def _exact_3x3x2(mdl, J, beta):
    key = (mdl, J.tobytes(), beta)
    if key not in _EXACT:
        _EXACT[key] = exact.boltzmann_lattice(mdl, J, beta, 2)
    return _EXACT[key]


def _lumped_check(mdl, dims, bc, beta, chi, ebf, n_sweeps, seed, n_chains=16):
    """n_chains independent oracle chains (replicas of one instance) for n_sweeps after 20 of burn-in."""
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(n_chains, dims, 2, seed)
    snaps = []
    acc = tot = 0
    for t in range(n_sweeps + 20):
        a, b = update.sweep(mdl, dims, bc, spins, lambda c: J, [beta] * n_chains, chi, t, seed,
                            env_beta_factor=ebf)
        acc += a
        tot += b
        if t >= 20:
            snaps.append(spins.copy())
    _, p, E = _exact_3x3x2(mdl, J, beta)
    idx = boltzmann_check.state_index(np.array(snaps).reshape(-1, *dims[::-1])).reshape(n_sweeps, n_chains)
    return boltzmann_check.lumped_chi2(idx, p, E, flip_invariant=True), acc / tot


@pytest.mark.slow
@pytest.mark.parametrize("bc,chi,ebf", [((0, 0, 0), 1, None), ((0, 0, 0), 4, None), ((0, 0, 0), 1, 0.7),
                                        ((1, 1, 0), 4, None)])
def test_chain_state_histogram_3x3x2(bc, chi, ebf):
    """3x3x2 lattice (2^18 states) under the full oracle chain: the visited states, lumped by energy, by
    exact probability and by a random partition (each flip pair s, -s in one bin: the global flip is a
    slow mode of local slice moves that would only dilute the test), match exact enumeration
    (chi-squared at the 0.999 level). Free BC at a truncating chi (1), at exact chi (4) and with a proposal built at 0.7 beta;
    x and y periodic at chi 4, which runs R1 fixed lines, ring rows and the three colour classes of
    odd periodic axes."""
    res, acc = _lumped_check(model.MODEL_EA_PM, (3, 3, 2), bc, 0.7, chi, ebf, 300, seed=8)
    for name, (chi2, thr, dof, tau) in res.items():
        assert chi2 < thr, (name, chi2, thr, dof, tau, acc)
    if chi == 4 and ebf is None:
        assert acc > 0.999


@pytest.mark.slow
def test_planted_wrong_acceptance_fails_3x3x2(monkeypatch):
    """The same lumped test rejects a chain that accepts every proposal of a mismatched proposal."""
    real_exp = np.exp

    def always_accept(x):
        return real_exp(0.0) if np.ndim(x) == 0 else real_exp(x)

    monkeypatch.setattr(update.np, "exp", always_accept)
    res, acc = _lumped_check(model.MODEL_EA_PM, (3, 3, 2), (0, 0, 0), 0.7, 1, 0.3, 200, seed=8)
    monkeypatch.undo()
    assert any(chi2 > thr for chi2, thr, _, _ in res.values()), res


def test_tau_int_ar1_closed_form():
    """For an AR(1) series x_t = phi x_{t-1} + noise, tau_int = (1 + phi) / (2 (1 - phi))."""
    rng = np.random.default_rng(3)
    for phi in (0.0, 0.5, 0.8):
        n = 200000
        x = np.zeros(n)
        e = rng.standard_normal(n)
        for t in range(1, n):
            x[t] = phi * x[t - 1] + e[t]
        tau, W, err = observables.tau_int(x[:20000] if phi == 0.0 else x)
        expect = (1 + phi) / (2 * (1 - phi))
        assert abs(tau - expect) < 4 * err + 0.02, (phi, tau, expect, err)


def test_overlap_of_identical_and_flipped_replicas():
    s = inputs.make_spins(1, (4, 4, 4), 2, 3)[0]
    assert observables.overlap(s, s) == 1.0
    assert observables.overlap(s, 1 - s) == -1.0


def test_magnetisation_of_uniform_and_checkerboard_states():
    """M = mean of s with index 0 = spin +1: all-0 gives +1, all-1 gives -1, a checkerboard gives 0,
    and a single flipped site of N moves M by 2/N."""
    z = np.zeros((4, 4, 4), dtype=np.int8)
    assert observables.magnetisation(z) == 1.0
    assert observables.magnetisation(1 - z) == -1.0
    cb = (np.indices((4, 4, 4)).sum(axis=0) % 2).astype(np.int8)
    assert observables.magnetisation(cb) == 0.0
    one = z.copy()
    one[1, 2, 3] = 1
    assert observables.magnetisation(one) == 1.0 - 2.0 / 64


def test_k_proposals_with_one_proposal_is_the_single_update():
    mdl, dims, bc = model.MODEL_EA_GAUSS, (4, 4, 4), (1, 1, 1)
    J = inputs.make_couplings(mdl, dims, bc, 3)
    s1 = inputs.make_spins(1, dims, 2, 4)[0]
    s2 = s1.copy()
    a = update.slice_update(mdl, dims, bc, s1, J, 0.9, 4, 1, 2, 17, 5, 0)
    b = update.slice_update_k(mdl, dims, bc, s2, J, 0.9, 4, 1, 2, 17, 5, 0, 1)
    assert np.array_equal(s1, s2)
    assert b.accepted == int(a.accept) and b.logq_old == a.logq_old
    assert b.dE == (a.dE if a.accept else 0)


@pytest.mark.parametrize("n_prop,ebf", [(3, None), (4, 0.5)])
def test_k_proposal_chain_matches_boltzmann_2x2x2(n_prop, ebf):
    """K proposals per environment build run as an independence-sampler chain on the slice: still exact."""
    mdl, dims, bc, beta = model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(1, dims, 2, 5)
    visits, energies = [], []
    for t in range(2000):
        update.sweep(mdl, dims, bc, spins, lambda c: J, [beta], 1, t, 5, env_beta_factor=ebf, n_prop=n_prop)
        if t >= 20:
            visits.append(spins[0].copy())
            energies.append(model.full_energy_int(mdl, spins[0], J) * model.J_SCALE)
    tv, bound, tau = _tv_test(mdl, dims, beta, visits, np.array(energies), J)
    assert tv < bound, (tv, bound, tau)


def test_metropolis_matches_boltzmann_2x2x2():
    """Checkerboard single-spin Metropolis (the paper's comparison method) samples Boltzmann exactly."""
    from oracle import metropolis
    mdl, dims, bc, beta = model.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    J = inputs.make_couplings(mdl, dims, bc, 11)
    spins = inputs.make_spins(1, dims, 2, 5)
    visits, energies = [], []
    for t in range(6000):
        metropolis.sweep(spins[0], J, beta, 5, t, 0)
        if t >= 20:
            visits.append(spins[0].copy())
            energies.append(model.full_energy_int(mdl, spins[0], J) * model.J_SCALE)
    tv, bound, tau = _tv_test(mdl, dims, beta, visits, np.array(energies), J)
    assert tv < bound, (tv, bound, tau)


def test_metropolis_field_and_flip_against_full_energy():
    """dE = 2 s_i h_i equals the full-lattice energy difference of one flip (periodic and open axes)."""
    from oracle import metropolis
    for bc in ((1, 1, 1), (0, 1, 0)):
        dims = (4, 3, 4)
        J = inputs.make_couplings(model.MODEL_EA_GAUSS, dims, bc, 2)
        s = inputs.make_spins(1, dims, 2, 3)[0]
        for (z, y, x) in ((0, 0, 0), (3, 2, 1), (1, 1, 3)):
            e0 = model.full_energy_int(model.MODEL_EA_GAUSS, s, J)
            si = 1 - 2 * int(s[z, y, x])
            dE = 2 * si * metropolis.local_field_int(s, J, z, y, x)
            s2 = s.copy()
            s2[z, y, x] = 1 - s2[z, y, x]
            assert model.full_energy_int(model.MODEL_EA_GAUSS, s2, J) - e0 == dE
