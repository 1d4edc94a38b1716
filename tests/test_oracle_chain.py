"""Chain-level pins: the oracle's TNMCMC-1 chain samples the exact Boltzmann distribution.

MH with the acceptance of Eq. (1) leaves the Boltzmann distribution invariant
for any positive proposal, so the stationary histogram must match exact
enumeration at a truncating chi, at exact chi and with a deliberately
mismatched proposal. A planted mistake (acceptance that ignores the proposal
ratio) must fail the same test, which shows the test has power.
"""
import numpy as np
import pytest

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


@pytest.mark.slow
def test_chain_energy_histogram_3x3x2():
    """3x3x2 free-BC lattice (2^18 states): energy histogram against exact enumeration, chi = 1."""
    mdl, dims, bc, beta = model.MODEL_EA_PM, (3, 3, 2), (0, 0, 0), 0.7
    J, visits, energies, acc = _run_chain(mdl, dims, bc, beta, 1, 1500, seed=8)
    _, p, E = exact.boltzmann_lattice(mdl, J, beta, 2)
    levels = np.unique(np.round(E, 9))
    p_lev = np.array([p[np.isclose(E, e)].sum() for e in levels])
    emp = np.array([(np.isclose(energies, e)).mean() for e in levels])
    tau, _, _ = observables.tau_int(energies)
    n_eff = len(energies) / (2 * max(tau, 0.5))
    mean_exact = float((p_lev * levels).sum())
    sd_exact = float(np.sqrt((p_lev * (levels - mean_exact) ** 2).sum()))
    assert abs(energies.mean() - mean_exact) < 4.5 * sd_exact / np.sqrt(n_eff)
    assert 0.5 * np.abs(emp - p_lev).sum() < 0.12


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
