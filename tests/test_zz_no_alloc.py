"""The allocation-free log Z entry point gives the same result as the context-based one.

tnmc_slice_logz_noalloc serves callers that may not allocate device memory
(hosts that own the device memory pool). It keeps its scratch in a fixed device
array of the library, so two calls in a row must not leak state into each
other. This file runs last (pytest collects files in name order), so a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_23945_gb300 import inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    # model, dims, bc, chi, beta, axis, slice, fix
    (inputs.MODEL_EA_PM, (6, 6, 6), (1, 1, 1), 8, 1.0, 2, 3, tnmc.FIX_R1),
    (inputs.MODEL_EA_GAUSS, (5, 7, 4), (0, 1, 0), 16, 1.3, 0, 2, tnmc.FIX_R2),
]


def _reference(mdl, dims, bc, chi, beta, axis, k, fix, spins, seed, step):
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=1, seed=7)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, fix_mode=fix)
    ctx.set_spins(0, spins[None])
    v = ctx.slice_logz(0, 0, axis, k, seed, step)
    ctx.close()
    return wl, v


def test_noalloc_logz_matches_context_logz_twice():
    results = []
    for (mdl, dims, bc, chi, beta, axis, k, fix) in CASES:
        wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=1, seed=7)
        spins = wl.initial_spins()[0]
        _, ref = _reference(mdl, dims, bc, chi, beta, axis, k, fix, spins, 5, 9)
        d_spins = torch.from_numpy(spins).cuda()
        d_J = torch.from_numpy(np.ascontiguousarray(wl.couplings[0])).cuda()
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        got = []
        for _ in range(2):            # two calls in a row share the scratch array
            tnmc.slice_logz_noalloc(d_spins, d_J, dims, bc, mdl, beta, chi, axis, k, 5, 9, fix, out=out)
            torch.cuda.synchronize()
            got.append(float(out.item()))
        for g in got:
            assert abs(g - ref) < 1e-9 * max(1.0, abs(ref)), (g, ref)
        results.append(got)
    assert results[0][0] != results[1][0]


def test_noalloc_rejects_sizes_beyond_its_limit():
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(17, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                         n_rep=1, seed=1)
    d_spins = torch.from_numpy(wl.initial_spins()[0]).cuda()
    d_J = torch.from_numpy(np.ascontiguousarray(wl.couplings[0])).cuda()
    with pytest.raises(tnmc.TnmcError) as e:
        tnmc.slice_logz_noalloc(d_spins, d_J, (17, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 4, 0, 0, 1, 1)
    assert e.value.code == 1
    with pytest.raises(tnmc.TnmcError):
        tnmc.slice_logz_noalloc(d_spins, d_J, (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 32, 0, 0, 1, 1)
