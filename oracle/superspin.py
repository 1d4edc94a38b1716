"""TNMCMC-2: the update of one composite layer of superspins (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Follows SM II.B ("TNMCMC-2: coarse-graining with superspins") and the main
text's description of the two sampling schemes (Fig. 1(b)):
* two adjacent layers k and k + 1 along the slice normal form one composite
  layer; each site of it is a superspin whose state is the pair of the two
  spins, so an Ising superspin has 2 x 2 = 4 states;
* the couplings inside each of the two layers and the couplings between them
  are absorbed into the local tensors of a 2D network of superspins; the
  Markov blanket is layers k - 1 and k + 2, held fixed as a field;
* the composite layer is then sampled exactly as a TNMCMC-1 slice (boundary
  MPS contraction, raster-order conditionals, Algorithm 2) and accepted with
  Eq. (1) using the exact energy change.

Readings (the paper gives no more detail):
* superspin index v = a + 2 b, where a is the state index of the layer-k spin
  and b that of the layer-(k + 1) spin (index 0 is spin +1, as in SM I.C);
* the fixed line (R1) and column (R2) of a periodic in-plane axis are whole
  lines of superspins (both layers), drawn as for a TNMCMC-1 slice but with
  the Philox axis word axis | 16, so a composite update never reuses a draw
  of a single-slice update; every other draw (site uniforms, Metropolis) uses
  that axis word too;
* the network's bond tables are general d x d tables: the in-plane bond of
  two neighbouring superspins carries exp(beta (J_k e(a, a') + J_k+1 e(b, b'))),
  and the bond between the two layers at one site enters the site factor;
* schedule (the main text's pairs of contiguous layers separated by fixed
  layers): sweep t updates axis t mod 3 with composite offset o = (t div 3)
  mod 2; composites start at k = o, o + 2, ... (both layers inside the
  lattice on an open axis); composites j and j + 1 touch each other's blanket,
  so they are coloured like TNMCMC-1 slices: a ring of composites (periodic
  axis of even extent) or a path (otherwise), two colour classes, three for
  an odd ring; step word of colour c is 4 t + c.
Ising models only (a Potts superspin would have q^2 > 4 states).
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

from . import bmps, model, philox, update

KIND_SUPER = 1
D_SUPER = 4


def rng_axis(axis: int) -> int:
    """Philox axis word of TNMCMC-2 draws."""
    return axis | (KIND_SUPER << 4)


def comp(v: int, layer: int) -> int:
    """State index of the spin of ``layer`` (0 = k, 1 = k + 1) in superspin v."""
    return (v >> layer) & 1


def geometry(dims, bc, axis: int, k: int, fix_mode: int, seed: int, step: int, chain: int) -> model.SliceGeom:
    n = int(dims[axis])
    if not bc[axis] and k + 1 >= n:
        raise ValueError("composite layer leaves the lattice on an open axis")
    return model.slice_geometry(dims, bc, axis, k, fix_mode, seed, step, chain, kind=KIND_SUPER)


def layer_coord(dims, g: model.SliceGeom, r: int, x: int, layer: int):
    c = list(g.coord(r, x))
    c[g.axis] = (g.k + layer) % int(dims[g.axis])
    return tuple(c)


def _idx(c):
    return c[2], c[1], c[0]


def terms(mdl: int, dims, spins: np.ndarray, J: np.ndarray, g: model.SliceGeom):
    """Integer energy tables of the composite layer (units of 2**-20).

    Returns (eh, ev, hf):
      eh[r-1, x, v, w]  sum of J e over the in-plane bonds (r, x) -> (r, x+1) of both layers
                        (wrap at x = Lc-1 on rings), superspins v at (r, x) and w at its neighbour
      ev[r-1, x, u, v]  the same for the bonds (r, x) -> (r+1, x), r < m
      hf[r-1, x, v]     every other bond touching the superspin at (r, x): the bonds between its
                        two spins, the held layers k-1 and k+2, the fixed line / column, and the
                        (zero-valued) wraps of open axes
    Every bond record of the lattice with at least one end in the composite layer is visited once.
    """
    if mdl == model.MODEL_POTTS:
        raise ValueError("superspins are built for Ising models")
    m, Lc, D = g.m, g.Lc, D_SUPER
    eh = np.zeros((m, Lc, D, D), dtype=np.int64)
    ev = np.zeros((m, Lc, D, D), dtype=np.int64)
    hf = np.zeros((m, Lc, D), dtype=np.int64)
    active = {}
    for r in range(1, m + 1):
        for x in range(Lc):
            for layer in (0, 1):
                active[layer_coord(dims, g, r, x, layer)] = (r, x, layer)
    hor, ver = model.tn_bonds(g)
    carried = {}
    for (r, x, _) in hor:
        for layer in (0, 1):
            carried[(layer_coord(dims, g, r, x, layer), g.ca)] = (eh, r, x)
    for (r, x) in ver:
        for layer in (0, 1):
            carried[(layer_coord(dims, g, r, x, layer), g.ra)] = (ev, r, x)
    records = set()
    for pos in active:
        for a in range(3):
            records.add((pos, a))
            records.add((model._step(dims, pos, a, -1), a))
    for (p, a) in sorted(records):
        q = model._step(dims, p, a, +1)
        jv = int(J[(a,) + _idx(p)])
        pa, qa = active.get(p), active.get(q)
        if (p, a) in carried:
            tab, r, x = carried[(p, a)]
            layer = pa[2]
            for v in range(D):
                for w in range(D):
                    tab[r - 1, x, v, w] += jv * model.pair_e(mdl, comp(v, layer), comp(w, layer))
        elif pa is not None and qa is not None:
            if pa[:2] == qa[:2] and pa[2] != qa[2]:
                # bond between the two spins of one superspin
                r, x = pa[0], pa[1]
                for v in range(D):
                    hf[r - 1, x, v] += jv * model.pair_e(mdl, comp(v, pa[2]), comp(v, qa[2]))
            elif jv != 0:
                raise AssertionError("uncarried bond between two superspins")
        elif pa is not None:
            r, x, layer = pa
            sv = int(spins[_idx(q)])
            for v in range(D):
                hf[r - 1, x, v] += jv * model.pair_e(mdl, comp(v, layer), sv)
        elif qa is not None:
            r, x, layer = qa
            sv = int(spins[_idx(p)])
            for v in range(D):
                hf[r - 1, x, v] += jv * model.pair_e(mdl, comp(v, layer), sv)
    return eh, ev, hf


def active_superspins(spins: np.ndarray, dims, g: model.SliceGeom) -> np.ndarray:
    out = np.zeros((g.m, g.Lc), dtype=np.int64)
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            a = int(spins[_idx(layer_coord(dims, g, r, x, 0))])
            b = int(spins[_idx(layer_coord(dims, g, r, x, 1))])
            out[r - 1, x] = a + 2 * b
    return out


def write_superspins(spins: np.ndarray, dims, g: model.SliceGeom, s: np.ndarray) -> None:
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            v = int(s[r - 1, x])
            spins[_idx(layer_coord(dims, g, r, x, 0))] = comp(v, 0)
            spins[_idx(layer_coord(dims, g, r, x, 1))] = comp(v, 1)


def energy_int(g: model.SliceGeom, eh, ev, hf, s: np.ndarray) -> int:
    """Energy of every bond touching the composite layer for superspins s [m, Lc] (exact integer)."""
    e = 0
    for r in range(g.m):
        for x in range(g.Lc):
            v = int(s[r, x])
            e -= int(hf[r, x, v])
            if x + 1 < g.Lc:
                e -= int(eh[r, x, v, int(s[r, x + 1])])
            elif g.ring:
                e -= int(eh[r, x, v, int(s[r, 0])])
            if r + 1 < g.m:
                e -= int(ev[r, x, v, int(s[r + 1, x])])
    return e


def weights(beta: float, g: model.SliceGeom, eh, ev, hf) -> model.SliceWeights:
    """Boltzmann factors of the superspin network, each normalised to a maximum of 1."""
    m, Lc, D = hf.shape
    b = beta * model.J_SCALE
    hmax = hf.max(axis=2, keepdims=True)
    phi = np.exp(b * (hf - hmax).astype(np.float64))
    log_scale = float(b * hmax.astype(np.float64).sum())
    psih = np.ones((m, Lc, D, D))
    psiv = np.ones((m, Lc, D, D))
    for r in range(m):
        for x in range(Lc):
            if x + 1 < Lc or g.ring:
                mx = eh[r, x].max()
                psih[r, x] = np.exp(b * (eh[r, x] - mx).astype(np.float64))
                log_scale += b * float(mx)
            if r + 1 < m:
                mx = ev[r, x].max()
                psiv[r, x] = np.exp(b * (ev[r, x] - mx).astype(np.float64))
                log_scale += b * float(mx)
    return model.SliceWeights(phi, psih, psiv, log_scale)


def site_uniforms(seed, g: model.SliceGeom, chain: int, step: int) -> np.ndarray:
    u = np.zeros((g.m, g.Lc))
    for r in range(1, g.m + 1):
        for x in range(g.Lc):
            u[r - 1, x] = philox.uniform(seed, philox.PURPOSE_SITE, (r - 1) * g.Lc + x, g.k, rng_axis(g.axis),
                                         step, chain)
    return u


def composite_update(mdl: int, dims, bc, spins: np.ndarray, J: np.ndarray, beta: float, chi: int,
                     axis: int, k: int, seed: int, step: int, chain: int,
                     fix_mode: int = model.FIX_R1, env_beta: Optional[float] = None,
                     write_back: bool = True) -> update.UpdateResult:
    """TNMCMC-2 update of the composite layer (k, k+1) normal to ``axis``; updates ``spins`` in place.

    s_old / s_new of the result are superspin indices [m, Lc]."""
    g = geometry(dims, bc, axis, k, fix_mode, seed, step, chain)
    eh, ev, hf = terms(mdl, dims, spins, J, g)
    s_old = active_superspins(spins, dims, g)
    w = weights(beta if env_beta is None else env_beta, g, eh, ev, hf)
    envs, logz = bmps.environments(w, g.ring, chi)
    u = site_uniforms(seed, g, chain, step)
    s_new, lq_new, ev1 = bmps.sample_slice(w, envs, g.ring, uniforms=u)
    _, lq_old, ev2 = bmps.sample_slice(w, envs, g.ring, forced=s_old)
    dE = energy_int(g, eh, ev, hf, s_new) - energy_int(g, eh, ev, hf, s_old)
    logA = (lq_old - lq_new) - beta * dE * model.J_SCALE
    u_mh = philox.uniform(seed, philox.PURPOSE_MH, 0, k, rng_axis(axis), step, chain)
    accept = bool(u_mh < np.exp(min(0.0, logA)))
    if accept and write_back:
        write_superspins(spins, dims, g, s_new)
    return update.UpdateResult(s_old, s_new, lq_new, lq_old, dE, accept, g.y0, g.x0, ev1 + ev2,
                               logz + w.log_scale)


def composite_classes(n: int, periodic: bool, offset: int) -> List[List[int]]:
    """Start layers of the composites of one axis and offset, grouped into colour classes."""
    if periodic:
        nc, ring = n // 2, n % 2 == 0
    else:
        nc, ring = (n - offset) // 2, False
    if nc <= 0:
        return []
    return [[(offset + 2 * j) % n for j in cls] for cls in update.colour_classes(nc, ring)]


def sweep(mdl: int, dims, bc, spins: np.ndarray, J_of_chain, betas, chi: int, t: int, seed: int,
          fix_mode: int = model.FIX_R1, env_beta_factor: Optional[float] = None):
    """One TNMCMC-2 sweep t of every chain. Returns (accepted, proposed)."""
    axis = t % 3
    offset = (t // 3) % 2
    n = int(dims[axis])
    acc = tot = 0
    for colour, ks in enumerate(composite_classes(n, bool(bc[axis]), offset)):
        step = t * 4 + colour
        for c in range(spins.shape[0]):
            beta = float(betas[c])
            eb = None if env_beta_factor is None else beta * env_beta_factor
            for k in ks:
                res = composite_update(mdl, dims, bc, spins[c], J_of_chain(c), beta, chi, axis, k, seed, step, c,
                                       fix_mode=fix_mode, env_beta=eb)
                acc += int(res.accept)
                tot += 1
    return acc, tot
