"""How well a density-matrix cut can match the oracle's SVD cut in FP64 (CPU).

The GPU path truncates each bond from the eigenvectors of the reduced density
matrix rho = C N C^T, where N is the Gram matrix of the part of the applied
row MPS to the right of the bond (the cut of SM I.B, reached without
canonicalisation). rho squares singular values, so directions below sqrt(eps)
of the largest are not resolved. This test takes the oracle's environment pass
(oracle.bmps), replaces its LQ + SVD compression with that density-matrix cut
written in numpy FP64, adds symmetric noise of one ulp of max|rho_ii| to rho
(any rounding of rho can do as much), and measures how far the forced log q of
the current slice moves. On typical slices (the seeded start advanced by oracle
sweeps) the shift stays far below the 1e-4 per-slice bound that the GPU parity
tests apply to the FP64 path; the numbers are printed.
"""
import numpy as np
import pytest

from oracle import bmps, model, update
from paper_2509_23945_gb300 import inputs

pytestmark = pytest.mark.slow


def _compress_density_matrix(rng, noise):
    def compress(B, chi):
        B = [t.astype(np.float64) for t in B]
        L = len(B)
        N = [None] * L
        Dl, d, Dr = B[L - 1].shape
        M = B[L - 1].reshape(Dl, d * Dr)
        N[L - 1] = M @ M.T
        N[L - 1] /= np.max(np.diag(N[L - 1]))
        for x in range(L - 2, -1, -1):
            acc = sum(B[x][:, v, :] @ N[x + 1] @ B[x][:, v, :].T for v in range(B[x].shape[1]))
            N[x] = acc / np.max(np.diag(acc))
        out, G = [], None
        for x in range(L):
            C = B[x] if G is None else np.einsum("ka,adb->kdb", G, B[x])
            kl, d, Dr = C.shape
            if x == L - 1:
                out.append(C / np.linalg.norm(C))
                break
            Cm = C.reshape(kl * d, Dr)
            rho = Cm @ N[x + 1] @ Cm.T
            rho = 0.5 * (rho + rho.T)
            if noise:
                E = rng.standard_normal(rho.shape)
                rho = rho + noise * np.max(np.abs(np.diag(rho))) * 0.5 * (E + E.T)
            _, U = np.linalg.eigh(rho)
            k = min(chi, kl * d, Dr)
            Uk = U[:, ::-1][:, :k]
            G = Uk.T @ Cm
            G = G / np.linalg.norm(G)
            out.append(Uk.reshape(kl, d, k))
        return out, 0.0
    return compress


def test_density_matrix_cut_on_typical_slices(monkeypatch):
    mdl, dims, bc, chi = inputs.MODEL_EA_GAUSS, (10, 10, 10), (1, 1, 1), 24
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[1.0], n_inst=1, n_rep=2, seed=5)
    spins = wl.initial_spins()
    for t in range(2):
        update.sweep(mdl, dims, bc, spins, lambda c: wl.couplings[0], wl.chain_beta(), chi, t, 2025)
    rng = np.random.default_rng(0)
    shifts = []
    for c in range(wl.n_chains):
        for k in update.colour_classes(dims[1], True)[c % 2]:
            g = model.slice_geometry(dims, bc, 1, k, model.FIX_R1, 2024, 11, c)
            w = model.slice_weights(mdl, 1.0, g, *model.slice_terms(mdl, dims, spins[c], wl.couplings[0], g))
            s_old = model.active_spins(spins[c], dims, g)
            envs, _ = bmps.environments(w, g.ring, chi)
            ref = bmps.sample_slice(w, envs, g.ring, forced=s_old)[1]
            for noise in (0.0, 1e-16, 1e-16):
                with monkeypatch.context() as mp:
                    mp.setattr(bmps, "compress", _compress_density_matrix(rng, noise))
                    envs_dm, _ = bmps.environments(w, g.ring, chi)
                shifts.append(abs(bmps.sample_slice(w, envs_dm, g.ring, forced=s_old)[1] - ref))
    shifts = np.array(shifts)
    print(f"density-matrix cut vs SVD cut, FP64, L=10 chi=24 typical slices: median {np.median(shifts):.2e} "
          f"max {shifts.max():.2e}")
    assert shifts.max() < 1e-4
