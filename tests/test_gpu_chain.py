"""Chain-level GPU tests: exact Boltzmann sampling, determinism of the batched
schedule (graph replay, uneven lattice groups in one launch) and checkpointing.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import boltzmann_check  # noqa: E402
from oracle import exact, model, observables  # noqa: E402
from paper_2509_23945_gb300 import inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _tv_against_exact(mdl, J, beta, visits, energies):
    states, p, _ = exact.boltzmann_lattice(mdl, J, beta, 2)
    index = {s.tobytes(): i for i, s in enumerate(states)}
    counts = np.zeros(len(states))
    for v in visits:
        counts[index[v.tobytes()]] += 1
    emp = counts / counts.sum()
    tv = 0.5 * np.abs(emp - p).sum()
    # tau from every chain's energy series (pooled), which is far less noisy than one chain's
    taus = [observables.tau_int(e)[0] for e in energies]
    tau = float(np.mean(taus))
    n_eff = max(int(len(visits) / (2 * max(tau, 0.5))), 1)
    rng = np.random.default_rng(0)
    null = [0.5 * np.abs(rng.multinomial(n_eff, p) / n_eff - p).sum() for _ in range(200)]
    return tv, float(np.quantile(null, 0.999))


@pytest.mark.parametrize("prec,chi,factor", [(tnmc.PREC_F64, 1, 1.0), (tnmc.PREC_F32, 4, 1.0),
                                             (tnmc.PREC_F64, 1, 0.7)])
def test_gpu_chain_samples_exact_boltzmann(prec, chi, factor):
    """2x2x2 free-BC lattice (256 states): the GPU chain's state histogram matches exact
    enumeration at a truncating chi, at exact chi and with a deliberately mismatched proposal."""
    mdl, dims, bc, beta = inputs.MODEL_EA_PM, (2, 2, 2), (0, 0, 0), 0.8
    n_chains = 16
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=n_chains, seed=11)
    J = wl.couplings[0]
    ctx = tnmc.Context([wl], precision=prec)
    ctx.set_spins(0, wl.initial_spins())
    if factor != 1.0:
        ctx.set_proposal_beta_factor(factor)
    visits, energies = [], [[] for _ in range(n_chains)]
    for t in range(1000):
        ctx.sweep(1, 3, use_graph=True)
        if t >= 10:
            s = ctx.get_spins(0)
            for c in range(n_chains):
                visits.append(s[c].copy())
                energies[c].append(model.full_energy_int(mdl, s[c], J) * model.J_SCALE)
    ctx.close()
    tv, bound = _tv_against_exact(mdl, J, beta, visits, [np.array(e) for e in energies])
    assert tv < bound, (tv, bound)


_EXACT = {}


@pytest.mark.parametrize("bc,prec,chi,factor", [((0, 0, 0), tnmc.PREC_F64, 1, 1.0),
                                                ((0, 0, 0), tnmc.PREC_F32, 4, 1.0),
                                                ((0, 0, 0), tnmc.PREC_F64, 1, 0.7),
                                                ((1, 1, 0), tnmc.PREC_F32, 4, 1.0),
                                                ((1, 1, 0), tnmc.PREC_F64, 1, 1.0)])
def test_gpu_chain_3x3x2_state_histogram(bc, prec, chi, factor):
    """3x3x2 lattice (2^18 states), 256 chains of the GPU sweep: the visited states, lumped by energy,
    by exact probability and by a random partition (flip pairs s, -s share a bin), match exact
    enumeration (chi-squared at the 0.999 level). Free BC at a truncating chi (1), exact chi (4) and a proposal built at 0.7 beta; x and y
    periodic, which runs R1 fixed lines, ring rows and three colour classes per odd periodic axis."""
    mdl, dims, beta, n_chains = inputs.MODEL_EA_PM, (3, 3, 2), 0.7, 256
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=n_chains, seed=13)
    J = wl.couplings[0]
    key = (bc, J.tobytes())
    if key not in _EXACT:
        _EXACT[key] = exact.boltzmann_lattice(mdl, J, beta, 2)
    _, p, E = _EXACT[key]
    ctx = tnmc.Context([wl], precision=prec)
    ctx.set_spins(0, wl.initial_spins())
    if factor != 1.0:
        ctx.set_proposal_beta_factor(factor)
    acc = torch.zeros(n_chains, dtype=torch.int32, device="cuda")
    ctx.sweep(20, 3, use_graph=True)
    snaps, n_sweeps = [], 300
    for t in range(n_sweeps):
        ctx.sweep(1, 3, use_graph=True, accept_counter=acc)
        snaps.append(ctx.get_spins(0))
    ctx.close()
    snaps = np.array(snaps)                                    # [T, chains, 2, 3, 3]
    idx = boltzmann_check.state_index(snaps.reshape(-1, *dims[::-1])).reshape(n_sweeps, n_chains)
    res = boltzmann_check.lumped_chi2(idx, p, E, flip_invariant=True)
    rate = acc.sum().item() / (n_sweeps * n_chains * sum(dims) / 3)
    print(f"3x3x2 bc={bc} prec={prec} chi={chi} factor={factor}: acceptance {rate:.4f} {res}")
    for name, (chi2, thr, dof, tau) in res.items():
        assert chi2 < thr, (name, chi2, thr, dof, tau)


@pytest.mark.parametrize("bc,chi", [((1, 1, 0), 4), ((1, 1, 0), 1), ((0, 0, 0), 1), ((1, 1, 1), 2)])
def test_gpu_chain_trajectory_equals_oracle_chain(bc, chi):
    """The GPU sweep (graph-replayed, all chains and colour classes in single launches) and the oracle's
    sweep (one slice at a time) follow the same trajectory in FP64: after every sweep the lattices of
    every chain are equal. Covers odd periodic axes (three colour classes), R1 fixed lines, rings of
    three sites and a periodic axis of length 2 (two bonds joining one pair of sites)."""
    from oracle import update
    mdl, dims, beta, n_chains, seed = inputs.MODEL_EA_PM, (3, 3, 2), 0.7, 6, 3
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=n_chains, seed=21)
    J = wl.couplings[0]
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64)
    ctx.set_spins(0, spins)
    lat = spins.copy()
    for t in range(24):
        ctx.sweep(1, seed, use_graph=True)
        update.sweep(mdl, dims, bc, lat, lambda c: J, wl.chain_beta(), chi, t, seed)
        assert np.array_equal(ctx.get_spins(0), lat), t
    ctx.close()


def test_graph_replay_equals_direct_launches():
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(6, 6, 6), bc=(1, 1, 1), chi=6, betas=[0.7, 1.2], n_inst=2,
                         n_rep=2, seed=2)
    out = []
    for graph in (False, True):
        ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
        ctx.set_spins(0, wl.initial_spins())
        ctx.sweep(7, 99, use_graph=graph)
        out.append(ctx.get_spins(0))
        ctx.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", [tnmc.PREC_F64, tnmc.PREC_F32])
def test_batched_slices_equal_one_call_per_slice(prec):
    """All same-parity slices of several chains in one launch give bitwise the results of updating
    each slice in a call of its own (each slice sees the spins as they stood before its phase)."""
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(6, 6, 6), bc=(1, 1, 1), chi=6, betas=[0.8, 1.3],
                         n_inst=1, n_rep=2, seed=4)
    spins = wl.initial_spins()
    chains, slices = [], []
    for c in range(wl.n_chains):
        for k in tnmc.colour_classes(6, True)[c % 2]:
            chains.append(c)
            slices.append(k)
    ctx = tnmc.Context([wl], precision=prec)
    ctx.set_spins(0, spins)
    batch = {k: v.cpu().numpy() for k, v in ctx.slice_update(0, 2, chains, slices, 31, 5).items()}
    lat_batch = ctx.get_spins(0)
    ctx.close()
    ctx = tnmc.Context([wl], precision=prec)
    ctx.set_spins(0, spins)
    for i, (c, k) in enumerate(zip(chains, slices)):
        one = {key: v.cpu().numpy() for key, v in ctx.slice_update(0, 2, [c], [k], 31, 5).items()}
        for key in batch:
            assert np.array_equal(one[key][0], batch[key][i]), (key, i)
    assert np.array_equal(ctx.get_spins(0), lat_batch)
    ctx.close()


def test_uneven_lattices_in_one_launch_equal_separate_runs():
    """Groups of different L share every launch. The first group's chains evolve exactly as in a
    context of their own; the second group's (global chain ids 2, 3) match direct launches."""
    wa = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=8, betas=[1.0], n_inst=1,
                         n_rep=2, seed=4)
    wb = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(6, 6, 6), bc=(1, 1, 1), chi=8, betas=[1.0], n_inst=1,
                         n_rep=2, seed=5)
    sa, sb = wa.initial_spins(), wb.initial_spins()
    both = tnmc.Context([wa, wb], precision=tnmc.PREC_F64)
    both.set_spins(0, sa)
    both.set_spins(1, sb)
    both.sweep(6, 21, use_graph=True)
    ga, gb = both.get_spins(0), both.get_spins(1)
    both.close()
    alone = tnmc.Context([wa], precision=tnmc.PREC_F64)
    alone.set_spins(0, sa)
    alone.sweep(6, 21)
    assert np.array_equal(alone.get_spins(0), ga)
    alone.close()
    pair = tnmc.Context([wa, wb], precision=tnmc.PREC_F64)
    pair.set_spins(0, sa)
    pair.set_spins(1, sb)
    pair.sweep(6, 21, use_graph=False)
    assert np.array_equal(pair.get_spins(1), gb)
    pair.close()


def test_checkpoint_resume_is_bitwise(tmp_path):
    wl = inputs.Workload(model=inputs.MODEL_POTTS, dims=(5, 4, 6), bc=(1, 1, 1), chi=6, betas=[0.55], n_inst=1,
                         n_rep=2, seed=8)
    ref = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ref.set_spins(0, wl.initial_spins())
    ref.sweep(8, 1234)
    want = ref.get_spins(0)
    ref.close()
    a = tnmc.Context([wl], precision=tnmc.PREC_F32)
    a.set_spins(0, wl.initial_spins())
    a.sweep(5, 1234)
    path = str(tmp_path / "ckpt.bin")
    a.save(path)
    a.close()
    b = tnmc.Context([wl], precision=tnmc.PREC_F32)
    b.load(path)
    assert b.sweep_counter == 5
    b.sweep(3, 1234)
    assert np.array_equal(b.get_spins(0), want)
    b.close()


def test_observables_match_host_computation():
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(5, 6, 4), bc=(1, 0, 1), chi=4, betas=[1.0], n_inst=1,
                         n_rep=4, seed=6)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl])
    ctx.set_spins(0, spins)
    obs = ctx.observables(0)
    ctx.sync()
    obs = obs.cpu().numpy()
    N = spins[0].size
    for c in range(wl.n_chains):
        e = model.full_energy_int(wl.model, spins[c], wl.couplings[0]) * model.J_SCALE / N
        assert abs(obs[c, 0] - e) < 1e-12
        assert abs(obs[c, 1] - observables.magnetisation(spins[c])) < 1e-12
        assert abs(obs[c, 2] - observables.overlap(spins[c], spins[c ^ 1])) < 1e-12
    ctx.close()


@pytest.mark.parametrize("n_prop", [2, 4])
def test_k_proposals_per_environment_match_oracle(n_prop):
    """K proposals from one environment build: the GPU slice updates equal the oracle's (final slice,
    number of accepted proposals, dE) and the chain trajectory is the oracle's."""
    from oracle import update
    mdl, dims, bc, beta, chi, seed = inputs.MODEL_EA_GAUSS, (6, 6, 6), (1, 1, 1), 1.0, 6, 5
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=2, seed=8)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64)
    ctx.set_spins(0, spins)
    ctx.set_proposals_per_env(n_prop)
    chains, slices = [0, 0, 1, 1], [0, 3, 1, 4]
    out = {k: v.cpu().numpy() for k, v in ctx.slice_update(0, 2, chains, slices, seed, 9).items()}
    lat = spins.copy()
    for i, (c, k) in enumerate(zip(chains, slices)):
        r = update.slice_update_k(mdl, dims, bc, lat[c], wl.couplings[0], beta, chi, 2, k, seed, 9, c, n_prop)
        g = model.slice_geometry(dims, bc, 2, k, model.FIX_R1, seed, 9, c)
        assert np.array_equal(out["new_spins"][i][: g.m, : g.Lc], r.s_final)
        assert int(out["accept"][i]) == r.accepted and int(out["dE"][i]) == r.dE
        assert abs(out["logq_old"][i] - r.logq_old) < 1e-6 and abs(out["logq_new"][i] - r.logq_final) < 1e-6
    assert np.array_equal(ctx.get_spins(0), lat)
    for t in range(6):
        ctx.sweep(1, seed, use_graph=True)
        update.sweep(mdl, dims, bc, lat, lambda c: wl.couplings[0], wl.chain_beta(), chi, t, seed, n_prop=n_prop)
        assert np.array_equal(ctx.get_spins(0), lat), t
    ctx.close()


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_gpu_metropolis_equals_oracle_metropolis(bc):
    """Checkerboard single-spin Metropolis: the GPU sweeps equal the oracle's bit for bit (same Philox
    draws), on open and on even periodic lattices, and a periodic axis of odd extent is refused."""
    from oracle import metropolis
    dims = (4, 6, 4)
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=dims, bc=bc, chi=4, betas=[0.9, 1.4], n_inst=2,
                         n_rep=2, seed=6)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64)
    ctx.set_spins(0, spins)
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    lat = spins.copy()
    inst, betas = wl.chain_instance(), wl.chain_beta()
    flips = np.zeros(wl.n_chains, dtype=np.int64)
    for t in range(5):
        ctx.metropolis_sweep(1, 17, accept_counter=acc)
        for c in range(wl.n_chains):
            flips[c] += metropolis.sweep(lat[c], wl.couplings[inst[c]], float(betas[c]), 17, t, c)
        assert np.array_equal(ctx.get_spins(0), lat), t
    assert np.array_equal(acc.cpu().numpy(), flips)
    ctx.close()
    odd = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(3, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                          n_rep=1)
    c2 = tnmc.Context([odd])
    with pytest.raises(tnmc.TnmcError):
        c2.metropolis_sweep(1, 1)
    c2.close()


def test_first_passage_harness_runs():
    """The tau_fp harness starts every chain at M = 1 and records the first sweep with M <= 0."""
    from paper_2509_23945_gb300 import first_passage
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(0, 0, 0), chi=4, betas=[0.6], n_inst=2,
                         n_rep=2, seed=3)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    for method in ("tnmcmc", "metropolis"):
        fp, dt = first_passage.run_method(ctx, method, 5, 400)
        s = first_passage.summary(fp)
        assert s["chains"] == 4 and s["censored"] == 0 and s["mean_sweeps"] >= 1, (method, s)
    ctx.close()
