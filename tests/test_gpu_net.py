"""GPU parity of the learned slice proposal against the FP64 oracle, through the C ABI.

The network's parameters are set from the oracle's initialisation, so both
sides evaluate the same function: teacher-forced logits and log q, the
gradient of the training loss, and the sampled proposal with the same Philox
uniforms inside the exact Metropolis-Hastings step. A training run on slices
accepted by the tensor-network sampler must raise the network's acceptance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import arnet, model, philox  # noqa: E402
from paper_2509_23945_gb300 import inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def flatten(P):
    nl = arnet.n_layers(P)
    return np.concatenate([np.concatenate([P[f"ws{l}"].ravel(), P[f"wc{l}"].ravel(), P[f"b{l}"].ravel()])
                           for l in range(1, nl + 1)]).astype(np.float64)


def _setup(mdl=inputs.MODEL_EA_GAUSS, dims=(6, 6, 6), bc=(1, 1, 1), H=8, layers=4, seed=2):
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=4, betas=[1.1], n_inst=1, n_rep=2, seed=seed)
    spins = wl.initial_spins()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ctx.set_spins(0, spins)
    ctx.net_init(channels=H, layers=layers, seed=1, buffer_slots=64)
    P = arnet.init_params(wl.d, channels=H, layers=layers, seed=3, scale=1.0)
    rng = np.random.default_rng(4)
    for k in P:
        if k.startswith("b"):
            P[k] = rng.standard_normal(P[k].shape) * 0.2
    P = {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}   # exactly representable on both sides
    ctx.net_set_params(flatten(P))
    return wl, spins, ctx, P


def _oracle_slice(wl, spins, chain, axis, k, seed, step):
    g = model.slice_geometry(wl.dims, wl.bc, axis, k, model.FIX_R1, seed, step, chain)
    Jh, Jv, hf = model.slice_terms(wl.model, wl.dims, spins[chain], wl.couplings[0], g)
    beta = float(wl.chain_beta()[chain])
    w = model.slice_weights(wl.model, beta, g, Jh, Jv, hf)
    cond = arnet.cond_features(w.phi, Jh, Jv, beta, g.ring, model.J_SCALE)
    s_old = model.active_spins(spins[chain], wl.dims, g)
    return g, Jh, Jv, hf, cond, s_old


def test_forward_logits_and_logq_match_oracle():
    wl, spins, ctx, P = _setup()
    chains, slices, axis, seed, step = [0, 1, 0], [0, 3, 2], 1, 9, 4
    out = ctx.net_eval(0, axis, chains, slices, seed, step)
    logits = out["logits"].cpu().numpy()
    lq = out["logq"].cpu().numpy()
    for i, (c, k) in enumerate(zip(chains, slices)):
        g, _, _, _, cond, s_old = _oracle_slice(wl, spins, c, axis, k, seed, step)
        ref, _ = arnet.forward(P, cond, s_old)
        got = logits[i][:, : g.m * g.Lc].reshape(wl.d, g.m, g.Lc)
        np.testing.assert_allclose(got, ref, rtol=1e-4, atol=2e-4)
        assert abs(lq[i] - arnet.logq(P, cond, s_old)) < 2e-3
    ctx.close()


def test_gradient_matches_oracle():
    wl, spins, ctx, P = _setup(mdl=inputs.MODEL_POTTS, dims=(5, 4, 5), bc=(0, 0, 0))
    chains, slices, axis, seed, step = [0, 1, 1], [1, 0, 2], 2, 5, 1
    out = ctx.net_eval(0, axis, chains, slices, seed, step, logits=False, grad=True)
    got = out["grad"].cpu().numpy().astype(np.float64)
    conds, ss = [], []
    for c, k in zip(chains, slices):
        g, _, _, _, cond, s_old = _oracle_slice(wl, spins, c, axis, k, seed, step)
        conds.append(cond)
        ss.append(s_old)
    loss, G = arnet.loss_and_grads(P, conds, ss)
    ref = flatten(G)
    # element by element: FP32 forward/backward against FP64, relative 1e-4 plus an absolute floor of
    # 1e-6 of the largest entry (entries that cancel to near zero carry FP32 rounding of their terms)
    err = np.abs(got - ref)
    bound = 1e-4 * np.abs(ref) + 1e-6 * np.abs(ref).max()
    worst = int(np.argmax(err / bound))
    print(f"gradient: max |err| {err.max():.3e}, worst ratio {err[worst] / bound[worst]:.3f} at {worst}")
    assert np.all(err <= bound), (worst, got[worst], ref[worst])
    ctx.close()


def test_gpu_adam_step_matches_oracle_adam():
    """Two GPU Adam steps (the update tnmc_net_train applies) with given gradients equal the oracle's
    Adam (Kingma & Ba; pinned by a hand-computed example) on every parameter, in FP32."""
    wl, spins, ctx, P = _setup()
    n = ctx.net_param_count()
    rng = np.random.default_rng(8)
    w0 = ctx.net_get_params().astype(np.float64)
    grads = [rng.standard_normal(n).astype(np.float32) * 0.1, rng.standard_normal(n).astype(np.float32) * 0.01]
    Po = {"w": w0.copy()}
    opt = arnet.Adam(Po, lr=3e-3)
    for g in grads:
        ctx.net_adam_step(g, 3e-3)
        opt.step(Po, {"w": g.astype(np.float64)})
    got = ctx.net_get_params().astype(np.float64)
    np.testing.assert_allclose(got, Po["w"], rtol=0, atol=2e-6 * max(1.0, np.abs(w0).max()))
    assert np.abs(got - w0).max() > 1e-3        # the steps moved the parameters
    ctx.close()


def test_checkpoint_carries_the_network(tmp_path):
    """tnmc_save/tnmc_load carry weights, Adam moments and step, the replay buffer and the schedule: a
    resumed training and proposal run is bitwise identical to an uninterrupted one."""
    def make():
        wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(6, 6, 6), bc=(1, 1, 1), chi=6, betas=[0.6], n_inst=1,
                             n_rep=4, seed=3)
        ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
        ctx.set_spins(0, wl.initial_spins())
        ctx.net_init(channels=8, layers=3, seed=7, buffer_slots=256)
        return ctx

    def phase2(ctx):
        ctx.net_train(5, 16, 3e-3, 11)
        ctx.set_proposal_mix(2, True)
        ctx.sweep(4, 13)
        return ctx.get_spins(0), ctx.net_get_params()

    ref = make()
    ref.set_proposal_mix(0, True)
    ref.sweep(6, 13)
    ref.net_train(5, 16, 3e-3, 9)
    want_s, want_w = phase2(ref)
    ref.close()
    a = make()
    a.set_proposal_mix(0, True)
    a.sweep(6, 13)
    a.net_train(5, 16, 3e-3, 9)
    path = str(tmp_path / "net.ckpt")
    a.save(path)
    a.close()
    b = make()
    b.load(path)
    got_s, got_w = phase2(b)
    assert np.array_equal(got_s, want_s)
    assert np.array_equal(got_w, want_w)
    b.close()


def test_net_proposal_matches_oracle():
    wl, spins, ctx, P = _setup()
    axis, seed, step = 0, 31, 6
    chains = [0, 0, 0, 1, 1, 1]
    slices = [0, 2, 4, 1, 3, 5]
    out = ctx.slice_update(0, axis, chains, slices, seed, step, proposal=tnmc.PROPOSAL_NET)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    lat = spins.copy()
    near = 0
    for i, (c, k) in enumerate(zip(chains, slices)):
        g, Jh, Jv, hf, cond, s_old = _oracle_slice(wl, spins, c, axis, k, seed, step)
        u = np.array([[philox.uniform(seed, philox.PURPOSE_NET_SITE, r * g.Lc + x, k, axis, step, c)
                       for x in range(g.Lc)] for r in range(g.m)])
        s_new, lq_new = arnet.sample(P, cond, u)
        got = out["new_spins"][i][: g.m, : g.Lc]
        lq_old = arnet.logq(P, cond, s_old)
        assert abs(out["logq_old"][i] - lq_old) < 2e-3
        if not np.array_equal(got, s_new):
            near += 1   # allowed only at a CDF boundary: check the first differing site
            j = int(np.argmax(got.reshape(-1) != s_new.reshape(-1)))
            logits, _ = arnet.forward(P, cond, s_new)
            p = np.exp(arnet.log_softmax(logits))[:, j // g.Lc, j % g.Lc]
            assert np.min(np.abs(np.cumsum(p) - u.reshape(-1)[j])) < 1e-4
            continue
        assert abs(out["logq_new"][i] - lq_new) < 2e-3
        dE = model.slice_energy_int(wl.model, g, Jh, Jv, hf, s_new) - model.slice_energy_int(wl.model, g, Jh, Jv, hf, s_old)
        assert int(out["dE"][i]) == dE
        logA = (lq_old - lq_new) - float(wl.chain_beta()[c]) * dE * model.J_SCALE
        u_mh = philox.uniform(seed, philox.PURPOSE_MH, 0, k, axis, step, c)
        if bool(out["accept"][i]) != (u_mh < np.exp(min(0.0, logA))):
            assert abs(u_mh - np.exp(min(0.0, logA))) < 1e-2
    assert near <= 1
    ctx.close()


def test_training_on_tn_accepted_slices_raises_acceptance():
    """The gain of the learned proposal: after training on slices the tensor network accepted,
    the network's own proposals are accepted far more often, at a fraction of the TN cost."""
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(6, 6, 6), bc=(1, 1, 1), chi=8, betas=[0.6], n_inst=2,
                         n_rep=4, seed=3)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ctx.set_spins(0, wl.initial_spins())
    ctx.net_init(channels=32, layers=4, seed=7, buffer_slots=2048)
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")

    def net_acceptance(n=6):
        ctx.set_proposal_mix(1, False)       # every sweep uses the network
        acc.zero_()
        ctx.sweep(n, 11, accept_counter=acc)
        torch.cuda.synchronize()
        return acc.sum().item() / (n * wl.n_chains * 6)

    ctx.set_proposal_mix(0, True)            # tensor network only, record accepted slices
    ctx.sweep(30, 5)
    torch.cuda.synchronize()
    assert ctx.net_buffer_count() > 200
    before = net_acceptance()
    losses = ctx.net_train(300, 64, 3e-3, 9)
    after = net_acceptance()
    print(f"net acceptance before {before:.3f} after {after:.3f}; loss {losses[0]:.3f} -> {losses[-1]:.3f}")
    assert losses[-20:].mean() < 0.8 * losses[:20].mean()
    assert after > before + 0.05
    ctx.close()


def test_trained_net_accepted_slices_per_second_vs_tensor_network():
    """What the trained network buys: accepted slices per second of its own sweeps against
    tensor-network sweeps of the same chains (L=8, chi=32, where contraction is costly)."""
    import time
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(8, 8, 8), bc=(1, 1, 1), chi=32, betas=[0.7], n_inst=2,
                         n_rep=8, seed=12)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ctx.set_spins(0, wl.initial_spins())
    ctx.net_init(channels=32, layers=5, seed=3, buffer_slots=4096)
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    slices_per_sweep = wl.n_chains * 8

    def timed(mix, n):
        ctx.set_proposal_mix(mix, mix == 0)
        ctx.sweep(3, 23, use_graph=True)         # captures the graphs of the three axes
        acc.zero_()
        ctx.sync()
        t0 = time.perf_counter()
        ctx.sweep(n, 19, use_graph=True, accept_counter=acc)
        ctx.sync()
        return acc.sum().item() / (n * slices_per_sweep), (time.perf_counter() - t0) / n

    acc_tn, t_tn = timed(0, 12)                  # tensor network, recording accepted slices
    before, _ = timed(1, 3)
    ctx.net_train(400, 64, 3e-3, 5)
    after, t_net = timed(1, 6)
    rate_tn = acc_tn * slices_per_sweep / t_tn
    rate_net = after * slices_per_sweep / t_net
    print(f"L=8 chi=32: TN acceptance {acc_tn:.3f} at {t_tn * 1e3:.1f} ms/sweep -> {rate_tn:.0f} accepted slices/s; "
          f"network acceptance {before:.3f} -> {after:.3f} at {t_net * 1e3:.1f} ms/sweep -> {rate_net:.0f}/s "
          f"(ratio {rate_net / max(rate_tn, 1e-9):.2f})")
    assert after > before
    ctx.close()
