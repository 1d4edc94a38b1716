"""Failure detection of the boundary, made on the host (no GPU fault): inputs that cannot be turned into
finite weights are refused or latched, and the context stays usable.

* A non-finite or negative beta is refused by tnmc_create (TNMC_ERR_ARG).
* A proposal beta factor of +inf (a test hook) makes every proposal weight non-finite: the kernels
  fall back to the uniform conditional (so q stays normalised and the chain exact), count the
  fallback sites, latch TNMC_ERR_NONFINITE in the device status word, and the next synchronising
  call returns it once. The lattice stays a valid configuration and later calls succeed.
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


@pytest.mark.parametrize("beta", [float("nan"), float("inf"), -1.0])
def test_create_refuses_non_finite_or_negative_beta(beta):
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=4, betas=[beta], n_inst=1,
                         n_rep=1)
    with pytest.raises(tnmc.TnmcError) as e:
        tnmc.Context([wl])
    assert e.value.code == 1


def test_non_finite_weights_are_latched_and_reported_once():
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(6, 6, 6), bc=(1, 1, 1), chi=6, betas=[0.9], n_inst=1,
                         n_rep=2, seed=4)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ctx.set_spins(0, wl.initial_spins())
    assert ctx.events() == 0
    ctx.set_proposal_beta_factor(float("inf"))
    out = ctx.slice_update(0, 1, [0, 0, 1], [0, 2, 3], 5, 1)
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.sync()
    assert e.value.code == 6                     # TNMC_ERR_NONFINITE, returned once
    ctx.sync()                                   # cleared: the next call succeeds
    assert ctx.events() > 0
    assert torch.isfinite(out["logq_new"]).all() and torch.isfinite(out["logq_old"]).all()
    s = ctx.get_spins(0)
    assert s.min() >= 0 and s.max() <= 1
    ctx.set_proposal_beta_factor(1.0)           # back to normal: no new status
    ctx.slice_update(0, 1, [0, 0, 1], [0, 2, 3], 5, 2)
    ctx.sync()
    ctx.close()


def test_sweep_status_is_returned_by_get_spins():
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                         n_rep=2, seed=2)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64)
    ctx.set_spins(0, wl.initial_spins())
    ctx.set_proposal_beta_factor(float("inf"))
    ctx.sweep(1, 3)
    with pytest.raises(tnmc.TnmcError) as e:
        ctx.get_spins(0)
    assert e.value.code == 6
    assert ctx.get_spins(0).shape == (2, 4, 4, 4)
    ctx.close()
