"""Overlap, magnetisation and integrated autocorrelation time (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

* Overlap q = (1/N) sum_i s_i^(1) s_i^(2) of two replicas with the same
  couplings (main text, "Sampling 3D spin glasses").
* Autocorrelation rho_O(k) and tau_int,O = 1/2 + sum_{k>=1} rho_O(k) truncated
  at a window (SM III, "Integrated autocorrelation time"). The paper truncates
  "where rho ceases to be statistically significant"; the reading used here is
  Sokal's automatic window: the smallest W with W >= c * tau(W), c = 6.
"""
from __future__ import annotations

import numpy as np


def ising_values(spins: np.ndarray) -> np.ndarray:
    return 1 - 2 * spins.astype(np.int64)


def overlap(s1: np.ndarray, s2: np.ndarray) -> float:
    return float(np.mean(ising_values(s1) * ising_values(s2)))


def magnetisation(s: np.ndarray) -> float:
    return float(np.mean(ising_values(s)))


def autocorrelation(x: np.ndarray) -> np.ndarray:
    """rho(k) for k = 0..n-1 with the sample mean and variance (SM III definition)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    xc = x - x.mean()
    var = np.dot(xc, xc) / n
    if var == 0.0:
        out = np.zeros(n)
        out[0] = 1.0
        return out
    rho = np.array([np.dot(xc[: n - k], xc[k:]) / (n - k) for k in range(n)]) / var
    return rho


def tau_int(x: np.ndarray, c: float = 6.0):
    """(tau_int, window W, Madras-Sokal error estimate)."""
    rho = autocorrelation(x)
    n = len(rho)
    tau = 0.5
    W = n - 1
    for w in range(1, n):
        tau += rho[w]
        if w >= c * tau:
            W = w
            break
    err = tau * np.sqrt(2.0 * (2 * W + 1) / n)
    return float(tau), int(W), float(err)
