"""The allocation-free log Z entry point gives the same result as the context-based one.

tnmc_slice_logz_noalloc serves callers that may not allocate device memory
(hosts that own the device memory pool). It keeps its scratch in a fixed device
array of the library, so consecutive calls must not leak state into each other:
the cases alternate between a large and a small lattice (A, B, A), and the
largest case fills the scratch to its size limit (extents 16, chi 16). This
file runs last (pytest collects files in name order), so a run that stops at
the first failure has already run every other test.
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


CASES = {
    # name: model, dims, bc, chi, beta, axis, slice, fix
    "limit": (inputs.MODEL_EA_PM, (16, 16, 16), (1, 1, 1), 16, 1.0, 2, 3, tnmc.FIX_R1),
    "small": (inputs.MODEL_EA_GAUSS, (5, 7, 4), (0, 1, 0), 16, 1.3, 0, 2, tnmc.FIX_R2),
    "chi16_mid": (inputs.MODEL_EA_GAUSS, (12, 9, 10), (1, 1, 1), 16, 0.8, 1, 4, tnmc.FIX_R1),
    "chi8": (inputs.MODEL_EA_PM, (6, 6, 6), (1, 1, 1), 8, 1.0, 2, 3, tnmc.FIX_R1),
}


def _inputs(name):
    mdl, dims, bc, chi, beta, axis, k, fix = CASES[name]
    wl = inputs.Workload(model=mdl, dims=dims, bc=bc, chi=chi, betas=[beta], n_inst=1, n_rep=1, seed=7)
    return wl, wl.initial_spins()[0]


def _reference(name):
    mdl, dims, bc, chi, beta, axis, k, fix = CASES[name]
    wl, spins = _inputs(name)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, fix_mode=fix)
    ctx.set_spins(0, spins[None])
    v = ctx.slice_logz(0, 0, axis, k, 5, 9)
    ctx.close()
    return v


def _noalloc(name, out):
    mdl, dims, bc, chi, beta, axis, k, fix = CASES[name]
    wl, spins = _inputs(name)
    d_spins = torch.from_numpy(spins).cuda()
    d_J = torch.from_numpy(np.ascontiguousarray(wl.couplings[0])).cuda()
    tnmc.slice_logz_noalloc(d_spins, d_J, dims, bc, mdl, beta, chi, axis, k, 5, 9, fix, out=out)
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_logz_matches_context_logz_on_alternating_calls():
    refs = {name: _reference(name) for name in CASES}
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    order = ["limit", "small", "limit", "chi16_mid", "chi8", "chi16_mid", "small"]
    for name in order:          # every call follows a call of another size on the same scratch
        got = _noalloc(name, out)
        ref = refs[name]
        assert abs(got - ref) < 1e-9 * max(1.0, abs(ref)), (name, got, ref)
    assert len({round(v, 6) for v in refs.values()}) == len(refs)


def test_noalloc_rejects_sizes_beyond_its_limit():
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(17, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                         n_rep=1, seed=1)
    d_spins = torch.from_numpy(wl.initial_spins()[0]).cuda()
    d_J = torch.from_numpy(np.ascontiguousarray(wl.couplings[0])).cuda()
    with pytest.raises(tnmc.TnmcError) as e:
        tnmc.slice_logz_noalloc(d_spins, d_J, (17, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 4, 0, 0, 1, 1)
    assert e.value.code == 1
    wl4 = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                          n_rep=1, seed=1)
    s4 = torch.from_numpy(wl4.initial_spins()[0]).cuda()
    J4 = torch.from_numpy(np.ascontiguousarray(wl4.couplings[0])).cuda()
    with pytest.raises(tnmc.TnmcError):       # chi above 16
        tnmc.slice_logz_noalloc(s4, J4, (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 32, 0, 0, 1, 1)
    with pytest.raises(tnmc.TnmcError):       # non-finite beta
        tnmc.slice_logz_noalloc(s4, J4, (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, float("inf"), 4, 0, 0, 1, 1)


def test_noalloc_binding_rejects_mis_shaped_tensors():
    wl4 = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                          n_rep=1, seed=1)
    s4 = torch.from_numpy(wl4.initial_spins()[0]).cuda()
    J4 = torch.from_numpy(np.ascontiguousarray(wl4.couplings[0])).cuda()
    with pytest.raises(ValueError):           # couplings of the wrong shape
        tnmc.slice_logz_noalloc(s4, J4[:2], (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 4, 0, 0, 1, 1)
    with pytest.raises(ValueError):           # int64 couplings
        tnmc.slice_logz_noalloc(s4, J4.long(), (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 4, 0, 0, 1, 1)
    with pytest.raises(ValueError):           # non-contiguous spins
        tnmc.slice_logz_noalloc(s4.transpose(0, 2), J4, (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 4, 0, 0, 1, 1)
    with pytest.raises(ValueError):           # output of the wrong dtype
        tnmc.slice_logz_noalloc(s4, J4, (4, 4, 4), (1, 1, 1), inputs.MODEL_EA_PM, 1.0, 4, 0, 0, 1, 1,
                                out=torch.empty(1, dtype=torch.float32, device="cuda"))
