"""GPU parity of the TNMCMC-2 composite-layer update (SM II.B) against the CPU oracle, through the C ABI.

A batch of composite layers (two adjacent layers of Ising spins merged into superspins of 4 states)
runs in one launch; the oracle runs the same updates with the same inputs and Philox draws. Compared
element by element: every sampled superspin (bit-exact unless the uniform lies within the stated
tolerance of a CDF boundary), log q of the proposal and of the current layer, the integer energy
change of both layers (bit-exact), the accept decision and the lattice afterwards. Whole TNMCMC-2
sweeps (both composite offsets, all three axes) must reproduce the oracle's trajectory bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bmps, model, superspin  # noqa: E402
from paper_2509_23945_gb300 import inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu

# log q bars per composite layer, as for TNMCMC-1 slices: FP64 1e-6, FP32 1e-4
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
    "open_L5_exact": (inputs.MODEL_EA_PM, (4, 3, 5), (0, 0, 0), 16, tnmc.FIX_R1, [1.0], 2),
    "L4_R1_chi8": (inputs.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 8, tnmc.FIX_R1, [0.9], 0),
    "L6_gauss_R1_chi6": (inputs.MODEL_EA_GAUSS, (6, 6, 6), (1, 1, 1), 6, tnmc.FIX_R1, [0.7, 1.3], 1),
    "L5_R2_chi5": (inputs.MODEL_EA_PM, (5, 5, 5), (1, 1, 1), 5, tnmc.FIX_R2, [1.1], 2),
    "extent2_periodic": (inputs.MODEL_EA_GAUSS, (2, 4, 3), (1, 0, 1), 8, tnmc.FIX_R1, [1.2], 0),
    "extent3_periodic": (inputs.MODEL_EA_PM, (4, 3, 4), (1, 1, 1), 6, tnmc.FIX_R1, [1.0], 1),
}


def _first_divergence_is_near(w, envs, ring, s_gpu, s_orc, u, tol_near):
    """The first site where the GPU draw differs from the oracle's must have its uniform within tol_near
    of a CDF boundary of the oracle's conditional there (both sides agree on every earlier site)."""
    probs = np.zeros(s_orc.shape + (4,))
    bmps.sample_slice(w, envs, ring, forced=s_orc, probs_out=probs)
    j = int(np.argmax(s_gpu.reshape(-1) != s_orc.reshape(-1)))
    r, x = divmod(j, s_orc.shape[1])
    cdf = np.cumsum(probs[r, x])
    return float(np.min(np.abs(cdf[:-1] - u[r, x]))) < tol_near


def _run_case(name, prec, seed=77, step=9):
    mdl, dims, bc, chi, fix, betas, axis = CASES[name]
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=betas, n_inst=1, n_rep=2, seed=3)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=prec, fix_mode=fix, layers=2)
    ctx.set_spins(0, spins)
    n = dims[axis]
    chains, slices = [], []
    for c in range(wl.n_chains):
        classes = tnmc.composite_classes(n, bool(bc[axis]), c % 2)
        for k in classes[0]:
            chains.append(c)
            slices.append(k)
    out = ctx.slice_update(0, axis, chains, slices, seed, step)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    lat_gpu = ctx.get_spins(0)
    ctx.close()
    lat = spins.copy()
    J_c = [wl.couplings[i] for i in wl.chain_instance()]
    beta_c = wl.chain_beta()
    diverged = set()
    worst = 0.0
    for i, (c, k) in enumerate(zip(chains, slices)):
        before = lat[c].copy()
        res = superspin.composite_update(mdl, dims, bc, lat[c], J_c[c], float(beta_c[c]), chi, axis, k, seed, step, c,
                                         fix_mode=fix)
        g = superspin.geometry(dims, bc, axis, k, fix, seed, step, c)
        s_gpu = out["new_spins"][i][: g.m, : g.Lc].astype(np.int64)
        assert abs(out["logq_old"][i] - res.logq_old) < TOL[prec], (name, i, out["logq_old"][i], res.logq_old)
        worst = max(worst, abs(out["logq_old"][i] - res.logq_old))
        if not np.array_equal(s_gpu, res.s_new):
            eh, ev, hf = superspin.terms(mdl, dims, before, J_c[c], g)
            w = superspin.weights(float(beta_c[c]), g, eh, ev, hf)
            envs, _ = bmps.environments(w, g.ring, chi)
            u = superspin.site_uniforms(seed, g, c, step)
            assert _first_divergence_is_near(w, envs, g.ring, s_gpu, res.s_new, u, NEAR[prec]), (name, i)
            diverged.add(c)
            continue
        assert abs(out["logq_new"][i] - res.logq_new) < TOL[prec], (name, i, out["logq_new"][i], res.logq_new)
        worst = max(worst, abs(out["logq_new"][i] - res.logq_new))
        assert int(out["dE"][i]) == res.dE
        if bool(out["accept"][i]) != res.accept:
            # only a Metropolis uniform within the log q differences of its threshold may flip
            import oracle.philox as ph
            logA = (res.logq_old - res.logq_new) - float(beta_c[c]) * res.dE * model.J_SCALE
            u_mh = ph.uniform(seed, ph.PURPOSE_MH, 0, k, superspin.rng_axis(axis), step, c)
            assert abs(u_mh - np.exp(min(0.0, logA))) < 2 * TOL[prec], (name, i)
            diverged.add(c)
    for c in range(wl.n_chains):
        if c not in diverged:
            assert np.array_equal(lat_gpu[c], lat[c]), (name, c)
    return worst, len(diverged)


@pytest.mark.parametrize("name", list(CASES))
def test_composite_update_parity_f64(name):
    worst, nd = _run_case(name, tnmc.PREC_F64)
    assert nd == 0, name


@pytest.mark.parametrize("name", ["L4_R1_chi8", "L6_gauss_R1_chi6", "L5_R2_chi5"])
def test_composite_update_parity_f32(name):
    _run_case(name, tnmc.PREC_F32)


def test_composite_logz_hook_exact_chi():
    """tnmc_slice_logz of a composite layer at exact chi equals the oracle's log Z (which equals
    enumeration, tests/test_oracle_superspin.py)."""
    mdl, dims, bc, chi, fix, betas, axis = CASES["open_L5_exact"]
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=betas, n_inst=1, n_rep=1, seed=3)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, fix_mode=fix, layers=2)
    ctx.set_spins(0, spins)
    for k in range(dims[axis] - 1):
        lz = ctx.slice_logz(0, 0, axis, k, 5, 3)
        res = superspin.composite_update(mdl, dims, bc, spins[0].copy(), wl.couplings[0], betas[0], chi, axis, k,
                                         5, 3, 0, fix_mode=fix, write_back=False)
        assert abs(lz - res.logz) < 1e-9 * abs(res.logz), (k, lz, res.logz)
    ctx.close()


SWEEP_CASES = [
    # model, dims, bc, chi, fix
    (inputs.MODEL_EA_PM, (4, 4, 4), (1, 1, 1), 4, tnmc.FIX_R1),
    (inputs.MODEL_EA_GAUSS, (3, 4, 5), (0, 0, 0), 3, tnmc.FIX_R1),
    (inputs.MODEL_EA_PM, (6, 3, 4), (1, 0, 1), 4, tnmc.FIX_R2),
]


@pytest.mark.parametrize("case", SWEEP_CASES)
@pytest.mark.parametrize("use_graph", [False, True])
def test_composite_sweeps_follow_oracle_trajectory(case, use_graph):
    """Six TNMCMC-2 sweeps (three axes x two composite offsets, every colour class in one launch) of four
    chains equal the oracle's sweeps bit for bit after every sweep (FP64)."""
    mdl, dims, bc, chi, fix = case
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[0.8, 1.2], n_inst=1, n_rep=2, seed=9)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, fix_mode=fix, layers=2)
    ctx.set_spins(0, spins)
    J_c = [wl.couplings[i] for i in wl.chain_instance()]
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    total_acc = 0
    for t in range(6):
        ctx.sweep(1, 123, use_graph=use_graph, accept_counter=acc)
        a, _ = superspin.sweep(mdl, dims, bc, spins, lambda c: J_c[c], wl.chain_beta(), chi, t, 123, fix_mode=fix)
        total_acc += a
        assert np.array_equal(ctx.get_spins(0), spins), t
    assert int(acc.sum().item()) == total_acc
    ctx.close()


def test_composite_batch_rules():
    """Composites of one chain closer than 3 layers, or leaving an open axis, are refused by the host."""
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(6, 4, 5), bc=(1, 0, 0), chi=2, betas=[1.0], n_inst=1,
                         n_rep=1, seed=1)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, layers=2)
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.slice_update(0, 0, [0, 0], [0, 4], 1, 0)         # periodic extent 6: 4 -> 0 is 2 layers
    assert e.value.code == 2
    ctx.slice_update(0, 0, [0, 0], [0, 3], 1, 0)             # 3 apart both ways: allowed
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.slice_update(0, 2, [0], [4], 1, 0)               # open extent 5: layers 4, 5 do not exist
    assert e.value.code == 1
    with pytest.raises(tnmc.TnmcError):
        ctx.net_init(channels=8, layers=3, seed=1, buffer_slots=4)
    ctx.close()
    with pytest.raises(tnmc.TnmcError):
        tnmc.Context([inputs.Workload(model=inputs.MODEL_POTTS, dims=(4, 4, 4), bc=(1, 1, 1), chi=2, betas=[0.5],
                                      n_inst=1, n_rep=1)], layers=2)
