"""Boundary-MPS contraction of one slice and its conditional sampler (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

The slice weight of active rows r = 1..m is
    W(s) = prod_r [ prod_x phi_r,x(s_r,x) prod_x psih_r,x(s_r,x, s_r,x+1) ]
           * prod_{r<m} prod_x psiv_r,x(s_r,x, s_r+1,x).
Environments E_r(s_r) = sum over rows r+1..m of the weight below row r (with
E_m = 1) obey E_{r-1}(u) = sum_s prod_x psiv_{r-1,x}(u_x, s_x) * rowweight_r(s)
* E_r(s): a row MPO applied to the boundary MPS E_r and truncated back to bond
dimension chi (SM I.B: "a row of the MPO is applied to the boundary MPS, and
the resulting MPS is then truncated back to the bond dimension chi").

Truncation reading (the paper names only SVD truncation to chi, SM I.B and the
retained-largest-singular-values rule of SM I.B): bring the applied MPS to
right-canonical form by LQ decompositions from right to left, then sweep left
to right, taking a thin SVD at each bond and keeping exactly
k = min(chi, rows, cols) singular vectors in descending order.

Sampling follows SM I.C / Eq. (sm-proposal-distribution) and Algorithm 2:
spins are drawn in raster order (row 1 first, column 0 first); the conditional
of each spin is the ratio of network contractions with the earlier spins
projected onto their basis vectors; a uniform u picks the smallest state v with
u < CDF(v), which for d = 2 is the rule "random() < q(+1) -> +1".
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

FLOOR_EPS = 1e-12


def row_mpo(psih_row: np.ndarray, ring: bool) -> List[np.ndarray]:
    """Diagonal MPO of prod_x psih(s_x, s_x+1) for one row: tensors W[i, j, v].

    Open row: the bond carries the previous spin (dimension d).
    Ring: the bond carries (first spin s_0, previous spin) (dimension d^2) and
    the last site closes the wrapping bond psih_{L-1}(s_{L-1}, s_0).
    """
    Lc, d = psih_row.shape[0], psih_row.shape[1]
    Ws = []
    if not ring:
        for x in range(Lc):
            Dl = 1 if x == 0 else d
            Dr = 1 if x == Lc - 1 else d
            W = np.zeros((Dl, Dr, d))
            for v in range(d):
                for i in range(Dl):
                    left = 1.0 if x == 0 else psih_row[x - 1, i, v]
                    if x == Lc - 1:
                        W[i, 0, v] = left
                    else:
                        W[i, v, v] = left
            Ws.append(W)
        return Ws
    D = d * d
    for x in range(Lc):
        Dl = 1 if x == 0 else D
        Dr = 1 if x == Lc - 1 else D
        W = np.zeros((Dl, Dr, d))
        for v in range(d):
            if x == 0:
                if Lc == 1:
                    W[0, 0, v] = psih_row[0, v, v]
                else:
                    W[0, v * d + v, v] = 1.0
                continue
            for c in range(d):
                for t in range(d):
                    i = c * d + t
                    val = psih_row[x - 1, t, v]
                    if x == Lc - 1:
                        W[i, 0, v] = val * psih_row[Lc - 1, v, c]
                    else:
                        W[i, c * d + v, v] = val
        Ws.append(W)
    return Ws


def apply_row(E: List[np.ndarray], Ws: List[np.ndarray], phi_row: np.ndarray, psiv_row) -> List[np.ndarray]:
    """B_x[(a,i), u, (b,j)] = sum_v psiv(u, v) phi(v) E_x[a, v, b] W_x[i, j, v].

    ``psiv_row`` is [Lc, du, d]; du = 1 with all ones closes the network (log Z).
    """
    out = []
    for x in range(len(E)):
        A, W = E[x], Ws[x]
        B = np.einsum("uv,v,avb,ijv->aiubj", psiv_row[x], phi_row[x], A, W)
        a, i, u, b, j = B.shape
        out.append(B.reshape(a * i, u, b * j))
    return out


def compress(B: List[np.ndarray], chi: int) -> Tuple[List[np.ndarray], float]:
    """Right-canonicalise by LQ, then truncate left to right by SVD keeping min(chi, ...) values.

    Returns the left-canonical truncated MPS (last tensor carries unit norm) and
    the log of the norm divided out along the way.
    """
    B = [t.copy() for t in B]
    L = len(B)
    lognorm = 0.0
    for x in range(L - 1, 0, -1):
        Dl, d, Dr = B[x].shape
        M = B[x].reshape(Dl, d * Dr)
        Q, R = np.linalg.qr(M.T)          # M = R^T Q^T
        k = Q.shape[1]
        B[x] = Q.T.reshape(k, d, Dr)
        Lm = R.T
        nrm = np.linalg.norm(Lm)
        if nrm == 0.0:
            raise FloatingPointError("zero environment")
        lognorm += np.log(nrm)
        B[x - 1] = np.einsum("adb,bk->adk", B[x - 1], Lm / nrm)
    out = []
    G = None
    for x in range(L):
        C = B[x] if G is None else np.einsum("ka,adb->kdb", G, B[x])
        kl, d, Dr = C.shape
        if x == L - 1:
            nrm = np.linalg.norm(C)
            lognorm += np.log(nrm)
            out.append(C / nrm)
            break
        U, S, Vt = np.linalg.svd(C.reshape(kl * d, Dr), full_matrices=False)
        k = min(chi, kl * d, Dr)
        G = S[:k, None] * Vt[:k]
        nrm = np.linalg.norm(G)
        lognorm += np.log(nrm)
        G = G / nrm
        out.append(U[:, :k].reshape(kl, d, k))
    return out, lognorm


def environments(w, ring: bool, chi: int) -> Tuple[List[List[np.ndarray]], float]:
    """E_1 .. E_m for the slice weights ``w`` (oracle.model.SliceWeights).

    Returns (envs, logz) where envs[r-1] is E_r and logz is log Z of the slice
    network relative to the normalised weights (exact when chi is exact).
    """
    m, Lc, d = w.phi.shape
    ones = [np.ones((1, d, 1)) for _ in range(Lc)]
    envs = [None] * m
    envs[m - 1] = ones
    E = ones
    logz = 0.0
    for r in range(m, 1, -1):               # build E_{r-1} from row r
        Ws = row_mpo(w.psih[r - 1], ring)
        B = apply_row(E, Ws, w.phi[r - 1], w.psiv[r - 2])
        E, ln = compress(B, chi)
        logz += ln
        envs[r - 2] = E
    # close with row 1: no row above, physical index summed
    Ws = row_mpo(w.psih[0], ring)
    B = apply_row(E, Ws, w.phi[0], np.ones((Lc, 1, d)))
    vec = B[0].reshape(B[0].shape[0] * B[0].shape[1], -1)
    for x in range(1, Lc):
        vec = vec @ B[x].reshape(B[x].shape[0], -1)
        nrm = np.max(np.abs(vec))
        logz += float(np.log(nrm))
        vec = vec / nrm
    logz += float(np.log(vec.reshape(-1)[0]))
    return envs, logz


def _floor_probs(pt: np.ndarray):
    pos = np.maximum(pt, 0.0)
    s = pos.sum()
    if not np.isfinite(s) or s <= 0.0:
        return np.full(pt.shape, 1.0 / pt.size), True
    p = pos + FLOOR_EPS * s
    return p / p.sum(), False


def sample_slice(w, envs, ring: bool, uniforms=None, forced=None, probs_out=None):
    """Draw (or evaluate) an active configuration row by row.

    ``uniforms[r-1, x]`` drives the draws; with ``forced`` [m, Lc] the choices
    are forced (teacher forcing) and no uniform is used. Returns
    (s [m, Lc], log q, number of floor/uniform fallback events). If
    ``probs_out`` is an array [m, Lc, d] it receives every conditional.
    """
    m, Lc, d = w.phi.shape
    s = np.zeros((m, Lc), dtype=np.int64)
    logq = 0.0
    events = 0
    for r in range(1, m + 1):
        E = envs[r - 1]
        Ws = row_mpo(w.psih[r - 1], ring)
        a = w.phi[r - 1].copy()
        if r >= 2:
            for x in range(Lc):
                a[x] = a[x] * w.psiv[r - 2, x, s[r - 2, x], :]
        T = []
        for x in range(Lc):
            t = np.einsum("avb,ijv,v->aivbj", E[x], Ws[x], a[x])
            al, i, _, b, j = t.shape
            T.append(t.reshape(al * i, d, b * j))
        R = [None] * (Lc + 1)
        R[Lc] = np.ones(1)
        for x in range(Lc - 1, -1, -1):
            vec = np.einsum("avb,b->a", T[x], R[x + 1])
            R[x] = vec / np.max(np.abs(vec))
        ell = np.ones(1)
        for x in range(Lc):
            pt = np.einsum("a,avb,b->v", ell, T[x], R[x + 1])
            p, ev = _floor_probs(pt)
            events += int(ev)
            if probs_out is not None:
                probs_out[r - 1, x] = p
            if forced is not None:
                v = int(forced[r - 1, x])
            else:
                u = uniforms[r - 1, x]
                cdf = 0.0
                v = d - 1
                for cand in range(d):
                    cdf += p[cand]
                    if u < cdf:
                        v = cand
                        break
            s[r - 1, x] = v
            logq += float(np.log(p[v]))
            ell = ell @ T[x][:, v, :]
            ell = ell / np.max(np.abs(ell))
    return s, logq, events
