"""GPU parity of proposals from the environment cache (the Conclusions' cache of typical fields) against
the CPU oracle, through the C ABI.

The cache is built from one lattice state on both sides (same fixed-line draws), the lattice is then
moved to another state, and a batch of cached updates is compared element by element: sampled spins
(bit-exact unless a uniform lies within the stated tolerance of a CDF boundary), log q of the proposal
and of the current slice, the integer dE, the accept decision and the lattice afterwards. Sweeps that
mix cached and fresh updates must follow the oracle's trajectory bit for bit in FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bmps, cache, model, philox, update  # noqa: E402
from paper_2509_23945_gb300 import inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {tnmc.PREC_F64: 1e-6, tnmc.PREC_F32: 1e-4}
NEAR = {tnmc.PREC_F64: 1e-9, tnmc.PREC_F32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = {
    # name: (model, dims, bc, chi, fix, betas, axis)
    "L4_R1": (inputs.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 8, tnmc.FIX_R1, [1.0], 1),
    "L6_gauss_R1": (inputs.MODEL_EA_GAUSS, (6, 6, 6), (1, 1, 1), 6, tnmc.FIX_R1, [0.8, 1.4], 2),
    "L5_R2": (inputs.MODEL_EA_PM, (5, 5, 5), (1, 1, 1), 5, tnmc.FIX_R2, [1.1], 0),
    "open": (inputs.MODEL_EA_GAUSS, (5, 4, 3), (0, 0, 0), 4, tnmc.FIX_R1, [0.9], 2),
    "potts": (inputs.MODEL_POTTS, (4, 4, 4), (1, 1, 1), 6, tnmc.FIX_R1, [0.55], 0),
}

BUILD_SEED, BUILD_STEP = 31, 5


def _run(name, prec, seed=13, step=21):
    mdl, dims, bc, chi, fix, betas, axis = CASES[name]
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=betas, n_inst=1, n_rep=2, seed=4)
    d = wl.d
    built_from = wl.initial_spins()
    now = inputs.make_spins(wl.n_chains, dims, d, 999)      # the state the cached proposals meet
    ctx = tnmc.Context([wl], precision=prec, fix_mode=fix)
    ctx.set_spins(0, built_from)
    ctx.cache_build(BUILD_SEED, BUILD_STEP)
    ctx.set_spins(0, now)
    n = dims[axis]
    chains, slices = [], []
    for c in range(wl.n_chains):
        for k in tnmc.colour_classes(n, bool(bc[axis]))[c % 2]:
            chains.append(c)
            slices.append(k)
    out = ctx.slice_update(0, axis, chains, slices, seed, step, proposal=tnmc.PROPOSAL_CACHE)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    lat_gpu = ctx.get_spins(0)
    ctx.close()
    lat = now.copy()
    J_c = [wl.couplings[i] for i in wl.chain_instance()]
    beta_c = wl.chain_beta()
    diverged = set()
    for i, (c, k) in enumerate(zip(chains, slices)):
        e = cache.build_entry(mdl, dims, bc, built_from[c], J_c[c], float(beta_c[c]), chi, axis, k, fix,
                              BUILD_SEED, BUILD_STEP, c)
        before = lat[c].copy()
        res = cache.cached_update(mdl, dims, lat[c], J_c[c], float(beta_c[c]), e, seed, step, c)
        g = e.g
        s_gpu = out["new_spins"][i][: g.m, : g.Lc].astype(np.int64)
        assert abs(out["logq_old"][i] - res.logq_old) < TOL[prec], (name, i, out["logq_old"][i], res.logq_old)
        if not np.array_equal(s_gpu, res.s_new):
            Jh, Jv, hf = model.slice_terms(mdl, dims, before, J_c[c], g)
            w = model.slice_weights(mdl, float(beta_c[c]), g, Jh, Jv, hf)
            probs = np.zeros((g.m, g.Lc, d))
            bmps.sample_slice(w, e.envs, g.ring, forced=res.s_new, probs_out=probs)
            j = int(np.argmax(s_gpu.reshape(-1) != res.s_new.reshape(-1)))
            r, x = divmod(j, g.Lc)
            u = update.site_uniforms(seed, g, c, step)[r, x]
            assert float(np.min(np.abs(np.cumsum(probs[r, x])[:-1] - u))) < NEAR[prec], (name, i)
            diverged.add(c)
            continue
        assert abs(out["logq_new"][i] - res.logq_new) < TOL[prec], (name, i)
        assert int(out["dE"][i]) == res.dE
        if bool(out["accept"][i]) != res.accept:
            logA = (res.logq_old - res.logq_new) - float(beta_c[c]) * res.dE * model.J_SCALE
            u_mh = philox.uniform(seed, philox.PURPOSE_MH, 0, k, axis, step, c)
            assert abs(u_mh - np.exp(min(0.0, logA))) < 2 * TOL[prec], (name, i)
            diverged.add(c)
    for c in range(wl.n_chains):
        if c not in diverged:
            assert np.array_equal(lat_gpu[c], lat[c]), (name, c)
    return len(diverged)


@pytest.mark.parametrize("name", list(CASES))
def test_cached_update_parity_f64(name):
    assert _run(name, tnmc.PREC_F64) == 0


@pytest.mark.parametrize("name", ["L4_R1", "L6_gauss_R1", "L5_R2"])
def test_cached_update_parity_f32(name):
    _run(name, tnmc.PREC_F32)


def test_cache_of_current_state_equals_fresh_update():
    """Open plane (no fixed-line draw): a cache built from the current spins gives the fresh update bit for
    bit, in the same launch shape."""
    mdl, dims, bc, chi, fix, betas, axis = CASES["open"]
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=betas, n_inst=1, n_rep=2, seed=4)
    outs = []
    for proposal in (tnmc.PROPOSAL_TN, tnmc.PROPOSAL_CACHE):
        ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
        ctx.set_spins(0, wl.initial_spins())
        ctx.cache_build(1, 2)
        o = ctx.slice_update(0, axis, [0, 1], [0, 1], 7, 3, proposal=proposal)
        outs.append({k: v.cpu().numpy() for k, v in o.items()})
        ctx.close()
    for key in outs[0]:
        assert np.array_equal(outs[0][key], outs[1][key]), key


SWEEP_CASES = [
    (inputs.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 4, tnmc.FIX_R1, 3),
    (inputs.MODEL_EA_GAUSS, (3, 4, 5), (0, 0, 0), 3, tnmc.FIX_R1, 0),
    (inputs.MODEL_EA_PM, (4, 3, 4), (1, 1, 1), 4, tnmc.FIX_R2, 2),
]


@pytest.mark.parametrize("case", SWEEP_CASES)
@pytest.mark.parametrize("use_graph", [False, True])
def test_cached_sweeps_follow_oracle_trajectory(case, use_graph):
    """Six sweeps of four chains mixing cached and fresh updates (fresh on t % k == k - 1) equal the
    oracle's sweeps bit for bit after every sweep (FP64)."""
    mdl, dims, bc, chi, fix, every = case
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[0.8, 1.2], n_inst=1, n_rep=2, seed=9)
    spins = wl.initial_spins()
    J_c = [wl.couplings[i] for i in wl.chain_instance()]
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, fix_mode=fix)
    ctx.set_spins(0, spins)
    ctx.cache_build(41, 0)
    ctx.set_cache_mix(True, every)
    C = cache.build(mdl, dims, bc, spins, lambda c: J_c[c], wl.chain_beta(), chi, fix, 41, 0)
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    total = 0
    for t in range(6):
        ctx.sweep(1, 55, use_graph=use_graph, accept_counter=acc)
        a, _ = cache.sweep(mdl, dims, bc, spins, lambda c: J_c[c], wl.chain_beta(), chi, t, 55, C, every, fix_mode=fix)
        total += a
        assert np.array_equal(ctx.get_spins(0), spins), t
    assert int(acc.sum().item()) == total
    ctx.close()


def test_cache_state_errors():
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=2, betas=[1.0], n_inst=1,
                         n_rep=1, seed=1)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64)
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.slice_update(0, 0, [0], [0], 1, 0, proposal=tnmc.PROPOSAL_CACHE)
    assert e.value.code == 7
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.set_cache_mix(True, 2)
    assert e.value.code == 7
    ctx.close()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, layers=2)
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.cache_build(1, 0)
    assert e.value.code == 1
    ctx.close()
