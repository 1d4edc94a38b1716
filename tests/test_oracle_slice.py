"""Pins of the oracle's slice network, sampler and energy against brute force.

At exact bond dimension the boundary-MPS conditionals equal the exact
conditionals of the slice (main text: exact Z(s_i, s_<i) gives exact sampling
and unit acceptance); at any chi the proposal is normalised by construction
(Eq. sm-proposal-distribution). Energies are checked against a full-lattice
recomputation, which shares nothing with the slice bookkeeping.
"""
import itertools

import numpy as np
import pytest

from oracle import bmps, exact, model, philox, update
from paper_2509_23945_gb300 import inputs

CASES = [
    # model, dims, bc, axis, k, fix_mode, beta
    (model.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 2, 1, model.FIX_R1, 1.0),
    (model.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 0, 2, model.FIX_R1, 1.25),
    (model.MODEL_EA_GAUSS, (4, 4, 4), (1, 1, 1), 1, 3, model.FIX_R1, 1.3),
    (model.MODEL_EA_PM, (3, 3, 3), (0, 0, 0), 2, 1, model.FIX_R1, 0.8),
    (model.MODEL_EA_PM, (4, 4, 3), (1, 1, 1), 0, 1, model.FIX_R2, 1.0),
    (model.MODEL_EA_GAUSS, (4, 3, 4), (0, 1, 1), 2, 0, model.FIX_R1, 1.6),
    (model.MODEL_POTTS, (3, 3, 3), (1, 1, 1), 2, 0, model.FIX_R1, 0.55),
    (model.MODEL_POTTS, (3, 4, 3), (0, 0, 0), 1, 0, model.FIX_R1, 0.55),
]


def _setup(case, seed=3, chi=64, env_beta=None):
    mdl, dims, bc, axis, k, fix, beta = case
    d = 3 if mdl == model.MODEL_POTTS else 2
    J = inputs.make_couplings(mdl, dims, bc, seed)
    spins = inputs.make_spins(1, dims, d, seed)[0]
    g = model.slice_geometry(dims, bc, axis, k, fix, 7, 5, 0)
    Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
    w = model.slice_weights(mdl, beta if env_beta is None else env_beta, g, Jh, Jv, hf)
    envs, logz = bmps.environments(w, g.ring, chi)
    return dict(mdl=mdl, dims=dims, bc=bc, d=d, J=J, spins=spins, g=g, Jh=Jh, Jv=Jv, hf=hf, w=w,
                envs=envs, logz=logz, beta=beta)


@pytest.mark.parametrize("case", CASES)
def test_logz_exact_chi_matches_enumeration(case):
    S = _setup(case)
    confs, logw = exact.slice_enumerate(S["mdl"], S["g"], S["Jh"], S["Jv"], S["hf"], S["beta"])
    assert abs((S["logz"] + S["w"].log_scale) - exact.log_sum_exp(logw)) < 1e-10 * max(1.0, abs(S["logz"]))


@pytest.mark.parametrize("case", CASES)
def test_conditionals_exact_chi_match_enumeration(case):
    S = _setup(case)
    confs, logw = exact.slice_enumerate(S["mdl"], S["g"], S["Jh"], S["Jv"], S["hf"], S["beta"])
    rng = np.random.default_rng(1)
    for _ in range(3):
        s = confs[rng.integers(len(confs))]
        probs = np.zeros(s.shape + (S["d"],))
        _, lq, ev = bmps.sample_slice(S["w"], S["envs"], S["g"].ring, forced=s, probs_out=probs)
        assert ev == 0
        P = exact.exact_conditionals(confs, logw, s)
        # the sampler floors every conditional by eps * sum (a fixed, stated rule)
        expect = (P + bmps.FLOOR_EPS) / (1 + S["d"] * bmps.FLOOR_EPS)
        np.testing.assert_allclose(probs, expect, rtol=1e-9, atol=1e-13)
        lq_expect = float(np.sum(np.log(np.take_along_axis(expect, s[..., None], axis=2))))
        assert abs(lq - lq_expect) < 1e-9
        # and the exact joint probability of the whole slice
        assert abs(lq - exact.exact_logq(confs, logw, s)) < np.sum(bmps.FLOOR_EPS / np.take_along_axis(P, s[..., None], 2)) * 1.01 + 1e-10


@pytest.mark.parametrize("chi", [1, 2])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[6]])
def test_truncated_proposal_is_normalised(case, chi):
    S = _setup(case, chi=chi)
    g, d = S["g"], S["d"]
    n = g.m * g.Lc
    if d ** n > 5000:
        pytest.skip("too many states for a full sum")
    total = 0.0
    for flat in itertools.product(range(d), repeat=n):
        s = np.array(flat).reshape(g.m, g.Lc)
        _, lq, _ = bmps.sample_slice(S["w"], S["envs"], g.ring, forced=s)
        total += np.exp(lq)
    assert abs(total - 1.0) < 1e-10


def test_truncation_changes_conditionals():
    """chi = 1 on a frustrated ring slice is a real approximation (guards against a no-op truncation)."""
    S1 = _setup(CASES[0], chi=1)
    S64 = _setup(CASES[0], chi=64)
    s = np.zeros((S1["g"].m, S1["g"].Lc), dtype=np.int64)
    _, lq1, _ = bmps.sample_slice(S1["w"], S1["envs"], S1["g"].ring, forced=s)
    _, lq64, _ = bmps.sample_slice(S64["w"], S64["envs"], S64["g"].ring, forced=s)
    assert abs(lq1 - lq64) > 1e-3


@pytest.mark.parametrize("case", CASES)
def test_sampled_logq_equals_forced_logq(case):
    S = _setup(case, chi=2)
    g = S["g"]
    u = np.random.default_rng(5).random((g.m, g.Lc))
    s, lq, _ = bmps.sample_slice(S["w"], S["envs"], g.ring, uniforms=u)
    _, lq2, _ = bmps.sample_slice(S["w"], S["envs"], g.ring, forced=s)
    assert abs(lq - lq2) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_slice_energy_difference_matches_full_lattice(case):
    S = _setup(case)
    g, dims = S["g"], S["dims"]
    rng = np.random.default_rng(9)
    s_old = model.active_spins(S["spins"], dims, g)
    for _ in range(5):
        s_new = rng.integers(0, S["d"], size=s_old.shape)
        de = model.slice_energy_int(S["mdl"], g, S["Jh"], S["Jv"], S["hf"], s_new) - \
            model.slice_energy_int(S["mdl"], g, S["Jh"], S["Jv"], S["hf"], s_old)
        lat = S["spins"].copy()
        model.write_active(lat, dims, g, s_new)
        assert de == model.full_energy_int(S["mdl"], lat, S["J"]) - model.full_energy_int(S["mdl"], S["spins"], S["J"])


def test_full_energy_single_bond():
    """A hand-computed energy: one +J bond between two aligned spins on an open 2x1x1 lattice."""
    J = np.zeros((3, 1, 1, 2), dtype=np.int32)
    J[0, 0, 0, 0] = 3 << model.J_FRAC_BITS
    s = np.zeros((1, 1, 2), dtype=np.int8)
    assert model.full_energy_int(model.MODEL_EA_PM, s, J) == -(3 << model.J_FRAC_BITS)
    s[0, 0, 1] = 1
    assert model.full_energy_int(model.MODEL_EA_PM, s, J) == (3 << model.J_FRAC_BITS)
    assert model.full_energy_int(model.MODEL_POTTS, s, J) == 0


def test_exact_chi_update_always_accepts():
    """At exact contraction q = P, so log A = 0 for every proposal (main text, TNMCMC paragraph)."""
    mdl, dims, bc = model.MODEL_EA_PM, (4, 4, 4), (1, 1, 1)
    J = inputs.make_couplings(mdl, dims, bc, 1)
    spins = inputs.make_spins(1, dims, 2, 1)[0]
    for t in range(3):
        for k in (0, 2, 1, 3):
            res = update.slice_update(mdl, dims, bc, spins, J, 1.0, 16, t % 3, k, 77, t * 4 + k % 2, 0)
            logA = (res.logq_old - res.logq_new) - 1.0 * res.dE * model.J_SCALE
            assert abs(logA) < 1e-6  # floor-limited; see the conditional test for the exact bound
            assert res.accept


def test_single_site_slice_is_heat_bath():
    """A 1 x 2 open slice of single sites: each conditional is the heat-bath probability."""
    mdl, dims, bc = model.MODEL_EA_PM, (2, 1, 3), (0, 0, 0)
    J = inputs.make_couplings(mdl, dims, bc, 4)
    spins = inputs.make_spins(1, dims, 2, 4)[0]
    g = model.slice_geometry(dims, bc, 2, 1, model.FIX_R1, 0, 0, 0)   # plane x (cols) by y (rows)
    Jh, Jv, hf = model.slice_terms(mdl, dims, spins, J, g)
    beta = 0.9
    w = model.slice_weights(mdl, beta, g, Jh, Jv, hf)
    envs, _ = bmps.environments(w, g.ring, 4)
    s = np.array([[0, 1]])
    probs = np.zeros((1, 2, 2))
    bmps.sample_slice(w, envs, g.ring, forced=s, probs_out=probs)
    # site 0 marginal: sum over site 1 of exp(beta (h0 s0 + h1 s1 + J s0 s1))
    h0 = (hf[0, 0, 0]) * model.J_SCALE
    h1 = (hf[0, 1, 0]) * model.J_SCALE
    j = Jh[0, 0] * model.J_SCALE
    z = {sv: sum(np.exp(beta * (h0 * sv + h1 * tv + j * sv * tv)) for tv in (1, -1)) for sv in (1, -1)}
    p_up = z[1] / (z[1] + z[-1])
    assert abs(probs[0, 0, 0] - (p_up + bmps.FLOOR_EPS) / (1 + 2 * bmps.FLOOR_EPS)) < 1e-12
    # site 1 given s0 = +1: heat bath in the field h1 + J
    q_up = 1 / (1 + np.exp(-2 * beta * (h1 + j)))
    assert abs(probs[0, 1, 0] - (q_up + bmps.FLOOR_EPS) / (1 + 2 * bmps.FLOOR_EPS)) < 1e-12


def test_fixed_line_is_a_state_independent_draw():
    g1 = model.slice_geometry((8, 8, 8), (1, 1, 1), 1, 3, model.FIX_R1, 5, 2, 9)
    y0 = min(int(philox.uniform(5, philox.PURPOSE_FIXED_ROW, 0, 3, 1, 2, 9) * 8), 7)
    assert g1.y0 == y0 and g1.m == 7 and g1.ring
    g2 = model.slice_geometry((8, 8, 8), (1, 1, 1), 1, 3, model.FIX_R2, 5, 2, 9)
    assert g2.x0 >= 0 and g2.Lc == 7 and not g2.ring
