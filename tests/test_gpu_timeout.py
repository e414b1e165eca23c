"""The timeout path of the persistent Risbo sweep, without a GPU fault: one
block leaves before a plane without publishing it (MW_DEBUG_STALL_PLANE), the
neighbour waits are limited to a few thousand polls (MW_DEBUG_POLLS), the
waiting blocks give up and leave, mw_plan_sync reports MW_ETIMEOUT, and the
same plan then computes a correct transform once the knobs are cleared."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def mw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6298_gb300 import build
    build.build()
    from paper_1110_6298_gb300 import mw as m
    m.lib()
    return m


@pytest.mark.parametrize("prec,delta", [("fp64", None), ("mixed", "risbo")])
def test_stalled_block_times_out_and_plan_recovers(mw, monkeypatch, prec, delta):
    L, spins = 96, [0, 2]
    g = wl.rng(900)
    flm = np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])
    plan = mw.Plan(L, spins, precision=prec, delta=delta)
    x = torch.from_numpy(flm).cuda()
    monkeypatch.setenv("MW_DEBUG_STALL_PLANE", "40")
    monkeypatch.setenv("MW_DEBUG_POLLS", "4096")
    plan.inverse(x)
    with pytest.raises(mw.MWError) as ei:
        plan.sync()
    assert ei.value.status == mw.MW_ETIMEOUT
    monkeypatch.delenv("MW_DEBUG_STALL_PLANE")
    monkeypatch.delenv("MW_DEBUG_POLLS")
    plan.sync()  # the flag was cleared by the report
    got = plan.inverse(x)
    plan.sync()
    for b, s in enumerate(spins):
        ref = oracle.inverse(flm[b], L, s)
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert np.max(np.abs(got[b].cpu().numpy() - ref)) / np.max(np.abs(ref)) < tol
    plan.close()
