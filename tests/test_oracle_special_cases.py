"""Special cases that fix the oracle's sampler by results known independently of it.

- A one-row slice (m = 1) needs no boundary MPS: its conditionals follow from
  transfer matrices, open or periodic (the row-MPO reading of SM I.A).
- An Ising ferromagnet without external field is symmetric under flipping
  every spin, so at exact bond dimension q(s) = q(-s) (Eq. sm-proposal-distribution
  with exact contraction gives q = P).
- The 2-state Potts model with coupling J_P is the Ising model with
  J_I = J_P / 2 (delta(v, w) = (1 + s_v s_w) / 2), so both give the same q on the
  same slice: this runs the d-generic code with d = 2 through both tables.
"""
import itertools

import numpy as np
import pytest

from oracle import bmps, model


def _floored(p):
    d = len(p)
    return (p + bmps.FLOOR_EPS) / (1.0 + d * bmps.FLOOR_EPS)


def _one_row_weights(rng, Lc, d, ring):
    phi = rng.uniform(0.2, 1.0, size=(1, Lc, d))
    psih = rng.uniform(0.2, 1.0, size=(1, Lc, d, d))
    if not ring:
        psih[0, Lc - 1] = 1.0
    psiv = np.ones((1, Lc, d, d))
    return model.SliceWeights(phi, psih, psiv, 0.0)


def _transfer_conditionals(w, s, ring):
    """P(s_x = v | s_<x) of a single row from products of transfer matrices."""
    phi, psih = w.phi[0], w.psih[0]
    Lc, d = phi.shape
    out = np.zeros((Lc, d))
    for x in range(Lc):
        # R[v, s0]: sum over s_{x+1..} of the weight to the right of site x (closing on s0 for a ring)
        if ring:
            R = psih[Lc - 1].copy()                       # psi_{L-1}(s_{L-1}, s_0)
            for y in range(Lc - 2, x - 1, -1):
                R = psih[y] @ (phi[y + 1][:, None] * R)
        else:
            R = np.ones((d, 1))
            for y in range(Lc - 2, x - 1, -1):
                R = psih[y] @ (phi[y + 1][:, None] * R)
        for v in range(d):
            left = phi[x, v] * (psih[x - 1, s[x - 1], v] if x > 0 else 1.0)
            if ring:
                right = R[v, v] if x == 0 else R[v, s[0]]
            else:
                right = R[v, 0] if x < Lc - 1 else 1.0
            out[x, v] = left * right
        out[x] /= out[x].sum()
    return out


@pytest.mark.parametrize("d,ring", [(2, False), (2, True), (3, False), (3, True)])
def test_one_row_slice_matches_transfer_matrices(d, ring):
    rng = np.random.default_rng(11 + d + 2 * ring)
    Lc = 6
    w = _one_row_weights(rng, Lc, d, ring)
    envs, _ = bmps.environments(w, ring, 8)
    for _ in range(4):
        s = rng.integers(0, d, size=(1, Lc))
        probs = np.zeros((1, Lc, d))
        bmps.sample_slice(w, envs, ring, forced=s, probs_out=probs)
        ref = _transfer_conditionals(w, s[0], ring)
        for x in range(Lc):
            np.testing.assert_allclose(probs[0, x], _floored(ref[x]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("ring", [False, True])
def test_zero_field_ferromagnet_is_flip_symmetric(ring):
    m, Lc, beta = 3, 4, 0.7
    t = np.array([[np.exp(beta), np.exp(-beta)], [np.exp(-beta), np.exp(beta)]]) / np.exp(beta)
    phi = np.ones((m, Lc, 2))
    psih = np.broadcast_to(t, (m, Lc, 2, 2)).copy()
    if not ring:
        psih[:, Lc - 1] = 1.0
    psiv = np.broadcast_to(t, (m, Lc, 2, 2)).copy()
    psiv[m - 1] = 1.0
    w = model.SliceWeights(phi, psih, psiv, 0.0)
    envs, _ = bmps.environments(w, ring, 2 ** Lc)          # exact bond dimension
    rng = np.random.default_rng(5)
    for _ in range(6):
        s = rng.integers(0, 2, size=(m, Lc))
        _, lq, _ = bmps.sample_slice(w, envs, ring, forced=s)
        _, lq_flip, _ = bmps.sample_slice(w, envs, ring, forced=1 - s)
        assert abs(lq - lq_flip) < 1e-12


def test_two_state_potts_equals_ising_at_half_coupling():
    rng = np.random.default_rng(8)
    g = model.slice_geometry((5, 4, 4), (1, 1, 1), 2, 1, model.FIX_R1, 3, 1, 0)
    m, Lc = g.m, g.Lc
    one = 1 << 20                                            # J = 1 in the fixed-point unit
    JP_h = rng.integers(1, 3, size=(m, Lc)) * 2 * one
    JP_v = rng.integers(1, 3, size=(m, Lc)) * 2 * one
    # held neighbour states sigma in {0, 1} (two per site) and their couplings
    sig = rng.integers(0, 2, size=(m, Lc, 2))
    Jn = rng.integers(1, 3, size=(m, Lc, 2)) * 2 * one
    spin = np.array([1, -1])                                 # Ising state v -> s_v
    hP = np.zeros((m, Lc, 2), dtype=np.int64)
    hI = np.zeros((m, Lc, 2), dtype=np.int64)
    for v in range(2):
        hP[:, :, v] = (Jn * (sig == v)).sum(axis=2)
        hI[:, :, v] = spin[v] * ((Jn // 2) * spin[sig]).sum(axis=2)
    beta = 0.6
    wP = model.slice_weights(model.MODEL_POTTS, beta, g, JP_h, JP_v, hP)
    wI = model.slice_weights(model.MODEL_EA_GAUSS, beta, g, JP_h // 2, JP_v // 2, hI)
    for chi in (2, 8):
        eP, _ = bmps.environments(wP, g.ring, chi)
        eI, _ = bmps.environments(wI, g.ring, chi)
        for _ in range(3):
            s = rng.integers(0, 2, size=(m, Lc))
            _, lqP, _ = bmps.sample_slice(wP, eP, g.ring, forced=s)
            _, lqI, _ = bmps.sample_slice(wI, eI, g.ring, forced=s)
            assert abs(lqP - lqI) < 1e-9 * max(1.0, abs(lqP))
