"""Chi-squared checks of sampled lattice states against an exact Boltzmann distribution (test helper).

The full state histogram of a 3x3x2 lattice has 2^18 bins, too many for a direct test at a feasible
sample size, so the states are lumped three ways, each a function of the state alone:
  * by energy level (exact energies of the enumeration),
  * into 16 bins of equal exact probability mass (states sorted by their exact probability),
  * into 16 bins of a fixed random partition of the state space.
Each lumped histogram is compared with its exact probabilities by Pearson's chi-squared statistic
scaled to the effective sample size n_eff = n / (2 tau_int) of the correlated chain samples; the
threshold is the 0.999 quantile of chi-squared with (bins - 1) degrees of freedom.
"""
import numpy as np
from scipy import stats


def state_index(spins):
    """Index of each lattice state in exact.boltzmann_lattice's enumeration (itertools.product order:
    the flattened [z, y, x] sites, first site most significant, base d)."""
    s = np.asarray(spins).reshape(len(spins), -1).astype(np.int64)
    n = s.shape[1]
    d = int(max(2, s.max() + 1))
    w = d ** np.arange(n - 1, -1, -1, dtype=np.int64)
    return s @ w


def _merge_small(p_bins, min_expected, n_eff):
    """Merge neighbouring bins (in the given order) until every bin expects >= min_expected counts."""
    groups, cur = [], []
    mass = 0.0
    for i, pi in enumerate(p_bins):
        cur.append(i)
        mass += pi
        if mass * n_eff >= min_expected:
            groups.append(cur)
            cur, mass = [], 0.0
    if cur:
        if groups:
            groups[-1].extend(cur)
        else:
            groups.append(cur)
    return groups


def lumped_chi2(indices, p, E, n_eff, seed=0, n_bins=16):
    """Returns {binning: (scaled chi2, threshold, dof)} for the visited state indices."""
    n = len(indices)
    counts = np.bincount(indices, minlength=len(p)).astype(np.float64)
    out = {}
    labels = {}
    levels, lev = np.unique(np.round(E, 9), return_inverse=True)
    labels["energy"] = lev
    order = np.argsort(p, kind="stable")
    cum = np.cumsum(p[order])
    q = np.minimum((cum * n_bins).astype(np.int64), n_bins - 1)
    lab = np.empty(len(p), dtype=np.int64)
    lab[order] = q
    labels["probability"] = lab
    labels["random"] = np.random.default_rng(seed).integers(0, n_bins, size=len(p))
    for name, lab in labels.items():
        k = int(lab.max()) + 1
        pb = np.bincount(lab, weights=p, minlength=k)
        ob = np.bincount(lab, weights=counts, minlength=k)
        groups = _merge_small(pb, 10.0, n_eff)
        P = np.array([pb[g].sum() for g in groups])
        O = np.array([ob[g].sum() for g in groups])
        chi2 = float(np.sum((O - n * P) ** 2 / (n * P))) * (n_eff / n)
        dof = len(groups) - 1
        out[name] = (chi2, float(stats.chi2.ppf(0.999, max(dof, 1))), dof)
    return out
