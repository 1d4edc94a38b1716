"""Pins of the oracle's masked-conv autoregressive proposal.

Finite differences pin the backward pass; perturbing later spins pins the
autoregressive masks; enumeration pins the normalisation of q_theta; a tiny
training run pins that Adam on the NLL moves q_theta towards its data.
"""
import itertools

import numpy as np
import pytest

from oracle import arnet


def _tiny(d=2, seed=0, m=3, L=4, ch=5, layers=4):
    P = arnet.init_params(d, channels=ch, layers=layers, seed=seed, scale=1.5)
    rng = np.random.default_rng(seed + 1)
    for k in P:
        if k.startswith("b"):
            P[k] = rng.standard_normal(P[k].shape) * 0.3
    cond = rng.standard_normal((arnet.n_cond(d), m, L))
    s = rng.integers(0, d, size=(m, L))
    return P, cond, s


@pytest.mark.parametrize("d", [2, 3])
def test_gradients_match_central_differences(d):
    P, cond, s = _tiny(d=d)
    rng = np.random.default_rng(7)
    conds = [cond, rng.standard_normal(cond.shape)]
    spins = [s, rng.integers(0, d, size=s.shape)]
    loss, G = arnet.loss_and_grads(P, conds, spins)
    h = 1e-6
    worst = 0.0
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            mk = arnet.mask("A") if k == "ws1" else (arnet.mask("B") if k.startswith("ws") else None)
            if mk is not None and mk.reshape(-1)[idx % 9] == 0:
                assert G[k].reshape(-1)[idx] == 0.0
                continue
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = arnet.loss_and_grads(P, conds, spins)
            flat[idx] = old - h
            lm, _ = arnet.loss_and_grads(P, conds, spins)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[k].reshape(-1)[idx]
            worst = max(worst, abs(fd - an) / max(1e-6, abs(fd) + abs(an)))
    assert worst < 1e-6, worst


def test_masks_make_logits_autoregressive():
    P, cond, s = _tiny(d=3, m=4, L=5)
    base, _ = arnet.forward(P, cond, s)
    n = s.size
    for i in range(n):
        s2 = s.copy().reshape(-1)
        s2[i:] = (s2[i:] + 1) % 3
        out, _ = arnet.forward(P, cond, s2.reshape(s.shape))
        r, x = divmod(i, s.shape[1])
        # every site at or before i in raster order sees no changed spin
        np.testing.assert_allclose(out.reshape(3, -1)[:, : i + 1], base.reshape(3, -1)[:, : i + 1], atol=1e-12)
    # and the mask is not vacuous: site 1 does depend on site 0
    s3 = s.copy()
    s3[0, 0] = (s3[0, 0] + 1) % 3
    out, _ = arnet.forward(P, cond, s3)
    assert np.abs(out[:, 0, 1] - base[:, 0, 1]).max() > 1e-6


def test_q_theta_is_normalised():
    P, cond, _ = _tiny(d=2, m=2, L=3)
    total = sum(np.exp(arnet.logq(P, cond, np.array(f).reshape(2, 3))) for f in itertools.product(range(2), repeat=6))
    assert abs(total - 1.0) < 1e-12


def test_sample_logq_matches_teacher_forced_logq():
    P, cond, _ = _tiny(d=3, m=3, L=3)
    u = np.random.default_rng(2).random((3, 3))
    s, lq = arnet.sample(P, cond, u)
    assert abs(lq - arnet.logq(P, cond, s)) < 1e-12


def test_cond_features_layout():
    phi = np.array([[[1.0, 0.5], [0.25, 1.0]]])      # m = 1, Lc = 2, d = 2
    Jh = np.array([[1 << 20, -(1 << 20)]])
    Jv = np.zeros((1, 2), dtype=np.int64)
    f = arnet.cond_features(phi, Jh, Jv, 0.5, True, 2.0 ** -20)
    assert np.allclose(f[0], [[0.0, np.log(0.25)]]) and np.allclose(f[1], [[np.log(0.5), 0.0]])
    assert np.allclose(f[2], [[0.5, -0.5]])          # right bonds (wrap on the ring)
    assert np.allclose(f[3], [[-0.5, 0.5]])          # left bonds
    assert np.allclose(f[4:], 0.0)


def test_adam_training_reduces_nll():
    P, cond, _ = _tiny(d=2, m=2, L=3, ch=6, layers=3)
    rng = np.random.default_rng(4)
    data = [np.array([[0, 0, 1], [1, 1, 0]])] * 6 + [rng.integers(0, 2, size=(2, 3)) for _ in range(2)]
    conds = [cond] * len(data)
    opt = arnet.Adam(P, lr=2e-2)
    first, _ = arnet.loss_and_grads(P, conds, data)
    for _ in range(60):
        loss, G = arnet.loss_and_grads(P, conds, data)
        opt.step(P, G)
    assert loss < 0.7 * first


def test_adam_two_steps_against_hand_computed_values():
    """Two Adam steps (Kingma & Ba 2015, Algorithm 1) worked out by hand for lr = 0.1, beta1 = 0.9,
    beta2 = 0.999, eps = 1e-8, theta_0 = (1, -2), gradients g_1 = (0.5, 3), g_2 = (-0.25, 1):
      t=1: m = 0.1 g_1 = (0.05, 0.3); v = 0.001 g_1^2 = (0.00025, 0.009);
           m^ = m / 0.1 = (0.5, 3); v^ = v / 0.001 = (0.25, 9);
           theta_1 = theta_0 - 0.1 m^ / (sqrt(v^) + eps) = (1 - 0.05/0.50000001, -2 - 0.3/3.00000001)
      t=2: m = 0.9 m + 0.1 g_2 = (0.02, 0.37); v = 0.999 v + 0.001 g_2^2 = (0.00031225, 0.009991);
           m^ = m / 0.19; v^ = v / 0.001999; theta_2 = theta_1 - 0.1 m^ / (sqrt(v^) + eps).
    The decimals below were evaluated from these expressions with 40-digit arithmetic. A missing bias
    correction, swapped betas or a dropped eps each move theta_1 by far more than the tolerance."""
    P = {"w": np.array([1.0, -2.0])}
    opt = arnet.Adam(P, lr=0.1, b1=0.9, b2=0.999, eps=1e-8)
    opt.step(P, {"w": np.array([0.5, 3.0])})
    np.testing.assert_allclose(P["w"], [0.90000000199999996000, -2.0999999996666666678], rtol=0, atol=1e-14)
    opt.step(P, {"w": np.array([-0.25, 1.0])})
    np.testing.assert_allclose(P["w"], [0.87336629870784616256, -2.1871063943494712565], rtol=0, atol=1e-14)
