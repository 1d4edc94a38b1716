"""GPU parity at the benchmark's size: 3D EA Gaussian glass, L = 32 periodic, chi = 64, R1.

Four slice updates of two chains run on the GPU in FP32 and FP64 and in the oracle with the same
seeded inputs and Philox draws, twice:
  1. from the seeded hot start (the benchmark's own start): the current slices are uniformly random;
  2. with the oracle's sampled slice written into each slice, so the current slices are typical
     draws of q (the state of a chain after its first update).
Compared: the fixed line, sampled spins (bit-exact unless a uniform lies at a CDF boundary), log q
of the sampled slice and of the current slice (bars per slice: FP32 1e-4, FP64 1e-6; the log q of a
uniformly random current slice, about -2000 here, is held per active site: 5e-5 in FP32, 1e-8 in
FP64), the integer dE and the accept decision. The oracle needs about 25 s per slice update on one core.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bmps, model, philox, update  # noqa: E402
from paper_2509_23945_gb300 import inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu

L, CHI, BETA = 32, 64, 1.1
ITEMS = [(0, 0), (0, 16), (1, 5), (1, 21)]
SEED, STEP, AXIS = 77, 3, 1
TOL = {tnmc.PREC_F32: 1e-4, tnmc.PREC_F64: 1e-6}
HOT_OLD_PER_SITE = {tnmc.PREC_F32: 5e-5, tnmc.PREC_F64: 1e-8}
NEAR = {tnmc.PREC_F32: 1e-5, tnmc.PREC_F64: 1e-9}


def _oracle(wl, spins, step):
    res = []
    for c, k in ITEMS:
        lat = spins[c].copy()
        res.append(update.slice_update(wl.model, wl.dims, wl.bc, lat, wl.couplings[0], BETA, CHI, AXIS, k, SEED, step,
                                       c, write_back=False))
    return res


@pytest.fixture(scope="module")
def oracle_results():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(L, L, L), bc=(1, 1, 1), chi=CHI, betas=[BETA],
                         n_inst=1, n_rep=2, seed=19)
    hot = wl.initial_spins()
    res_hot = _oracle(wl, hot, STEP)
    typical = hot.copy()
    for (c, k), r in zip(ITEMS, res_hot):
        g = model.slice_geometry(wl.dims, wl.bc, AXIS, k, model.FIX_R1, SEED, STEP, c)
        model.write_active(typical[c], wl.dims, g, r.s_new)
    res_typ = _oracle(wl, typical, STEP + 1)
    return wl, {"hot": (hot, STEP, res_hot), "typical": (typical, STEP + 1, res_typ)}


@pytest.mark.parametrize("start", ["typical", "hot"])
@pytest.mark.parametrize("prec", [tnmc.PREC_F32, tnmc.PREC_F64])
def test_parity_L32_chi64(oracle_results, prec, start):
    wl, runs = oracle_results
    spins, step, res = runs[start]
    ctx = tnmc.Context([wl], precision=prec)
    ctx.set_spins(0, spins)
    chains = [c for c, _ in ITEMS]
    slices = [k for _, k in ITEMS]
    out = {k: v.cpu().numpy() for k, v in ctx.slice_update(0, AXIS, chains, slices, SEED, step, write_back=False).items()}
    ctx.close()
    T = TOL[prec]
    worst_new = worst_old = 0.0
    for i, ((c, k), r) in enumerate(zip(ITEMS, res)):
        g = model.slice_geometry(wl.dims, wl.bc, AXIS, k, model.FIX_R1, SEED, step, c)
        assert g.y0 == r.y0
        T_old = T if (start == "typical" or HOT_OLD_PER_SITE[prec] is None) else HOT_OLD_PER_SITE[prec] * g.m * g.Lc
        s_gpu = out["new_spins"][i][: g.m, : g.Lc].astype(np.int64)
        worst_old = max(worst_old, abs(out["logq_old"][i] - r.logq_old))
        assert abs(out["logq_old"][i] - r.logq_old) < T_old, (prec, start, i, out["logq_old"][i], r.logq_old)
        if not np.array_equal(s_gpu, r.s_new):
            j = int(np.argmax(s_gpu.reshape(-1) != r.s_new.reshape(-1)))
            rr, x = divmod(j, g.Lc)
            Jh, Jv, hf = model.slice_terms(wl.model, wl.dims, spins[c], wl.couplings[0], g)
            w = model.slice_weights(wl.model, BETA, g, Jh, Jv, hf)
            envs, _ = bmps.environments(w, g.ring, CHI)
            probs = np.zeros((g.m, g.Lc, 2))
            bmps.sample_slice(w, envs, g.ring, forced=r.s_new, probs_out=probs)
            u = philox.uniform(SEED, philox.PURPOSE_SITE, j, k, AXIS, step, c)
            assert np.min(np.abs(np.cumsum(probs[rr, x]) - u)) < NEAR[prec], (prec, start, i, j)
            continue
        worst_new = max(worst_new, abs(out["logq_new"][i] - r.logq_new))
        assert abs(out["logq_new"][i] - r.logq_new) < T, (prec, start, i, out["logq_new"][i], r.logq_new)
        assert int(out["dE"][i]) == r.dE
        if bool(out["accept"][i]) != r.accept:
            logA = (r.logq_old - r.logq_new) - BETA * r.dE * model.J_SCALE
            u_mh = philox.uniform(SEED, philox.PURPOSE_MH, 0, k, AXIS, step, c)
            slack = abs(out["logq_old"][i] - r.logq_old) + abs(out["logq_new"][i] - r.logq_new) + 1e-12
            assert abs(u_mh - np.exp(min(0.0, logA))) < slack
    print(f"L=32 chi=64 prec={prec} {start}: worst |d log q_new| {worst_new:.3e}, |d log q_old| {worst_old:.3e}")


@pytest.mark.parametrize("tile", [1, 2])
def test_gemm_tiles_bitwise_at_L32_chi64(oracle_results, tile):
    """The GEMM tile variants of the FP32 kernel give the default tile's outputs bit for bit at the
    benchmark's size (bond 256: every GEMM spans several tiles of each shape)."""
    wl, runs = oracle_results
    spins, step, _ = runs["typical"]
    outs = []
    for t in (0, tile):
        ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
        ctx.set_tuning(gemm_tile=t)
        ctx.set_spins(0, spins)
        o = ctx.slice_update(0, AXIS, [c for c, _ in ITEMS], [k for _, k in ITEMS], SEED, step, write_back=False)
        outs.append({k: v.cpu().numpy() for k, v in o.items()})
        ctx.close()
    for key in outs[0]:
        assert np.array_equal(outs[0][key], outs[1][key]), key
