"""Chi-squared checks of sampled lattice states against an exact Boltzmann distribution (test helper).

The full state histogram of a 3x3x2 lattice has 2^18 bins, too many for a direct test at a feasible
sample size, so the states are lumped three ways, each a function of the state alone:
  * by energy level (exact energies of the enumeration),
  * into 16 bins of equal exact probability mass (states sorted by their exact probability),
  * into 16 bins of a fixed random partition of the state space.
Each lumped histogram is compared with its exact probabilities by Pearson's chi-squared statistic
scaled to the effective sample size n_eff = n / (2 tau) of the correlated chain samples, where tau is
the largest integrated autocorrelation time among the bin indicators of that lumping (pooled over
the chains, Sokal's window). A lumping that separates states of equal energy (the random partition,
ties inside a probability bin) sees slow modes such as a global flip that the energy does not. The
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


def pooled_tau(x):
    """Integrated autocorrelation time of x [T, chains] with the autocovariance pooled over chains and
    Sokal's window (smallest W with W >= 6 tau(W))."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[0]
    xc = x - x.mean()
    c0 = float((xc * xc).mean())
    if T < 4 or c0 <= 0.0:
        return 0.5
    tau = 0.5
    for w in range(1, T):
        tau += float((xc[: T - w] * xc[w:]).mean()) / c0
        if w >= 6 * tau:
            break
    return max(tau, 0.5)


def lumped_chi2(indices, p, E, seed=0, n_bins=16, flip_invariant=False):
    """indices: visited state indices [T, chains] (T samples of each chain, in order). Returns
    {binning: (scaled chi2, threshold, dof, tau)}.

    flip_invariant: for Ising states with a flip-symmetric distribution (p(s) = p(-s), no field), give
    s and -s the same label in the random and probability lumpings. The lumped distribution is then
    blind to the global flip, which a chain of local slice moves crosses slowly, and the test keeps
    its power for every other deviation."""
    indices = np.asarray(indices)
    T, nc = indices.shape
    flat = indices.reshape(-1)
    n = flat.size
    counts = np.bincount(flat, minlength=len(p)).astype(np.float64)
    out = {}
    labels = {}
    levels, lev = np.unique(np.round(E, 9), return_inverse=True)
    labels["energy"] = lev
    rep = np.arange(len(p))
    if flip_invariant:
        rep = np.minimum(rep, len(p) - 1 - rep)            # index of -s is the bitwise complement
    order = np.lexsort((rep, p))                           # by probability, ties by flip class
    cum = np.cumsum(p[order])
    q = np.minimum((cum * n_bins).astype(np.int64), n_bins - 1)
    lab = np.empty(len(p), dtype=np.int64)
    lab[order] = q
    if flip_invariant:
        lab = lab[rep]                                     # both members of a flip pair in one bin
    labels["probability"] = lab
    labels["random"] = np.random.default_rng(seed).integers(0, n_bins, size=len(p))[rep]
    for name, lab in labels.items():
        k = int(lab.max()) + 1
        pb = np.bincount(lab, weights=p, minlength=k)
        ob = np.bincount(lab, weights=counts, minlength=k)
        groups = _merge_small(pb, 10.0, n / 10.0)
        P = np.array([pb[g].sum() for g in groups])
        O = np.array([ob[g].sum() for g in groups])
        group_of = np.zeros(k, dtype=np.int64)
        for gi, g in enumerate(groups):
            group_of[g] = gi
        glab = group_of[lab[indices]]                       # [T, chains] group label of every sample
        tau = max(pooled_tau(glab == gi) for gi in range(len(groups)))
        n_eff = n / (2.0 * tau)
        chi2 = float(np.sum((O - n * P) ** 2 / (n * P))) * (n_eff / n)
        dof = len(groups) - 1
        out[name] = (chi2, float(stats.chi2.ppf(0.999, max(dof, 1))), dof, tau)
    return out
