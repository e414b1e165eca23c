"""Calls on page-locked host buffers: the copies run in pieces on a second
stream, overlapping the phi / theta stages (forward: per group of maps in,
per chunk of Wigner planes out; inverse: per group of maps out).  The results
must be bitwise those of the same calls on device buffers, for every mix of
host and device input and output, at batch sizes that give one-map groups
(B <= 8) and ragged groups (B = 11: groups of 2 and a last group of 1), and on
the FP64 path (64-plane chunks, many row copies) as well as the mixed one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,spins", [(130, [0, 2, 0, -1, 2]), (97, [0, 1, 2, 0, 0, 1, 2, -2, 0, 3, 1])])
def test_pinned_matches_device(mw, prec, L, spins):
    g = wl.rng(5150 + L)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins]))
    x = torch.from_numpy(np.stack([wl.gaussian_map(g, L) for _ in spins]))
    plan = mw.Plan(L, spins, precision=prec, graph=True)
    ref_map = plan.inverse(flm.cuda()).cpu()
    ref_flm = plan.forward(x.cuda()).cpu()
    flm_p, x_p = flm.pin_memory(), x.pin_memory()
    for _ in range(2):  # second round: the plan's copy stream and events are reused
        map_p = torch.empty_like(x).pin_memory()
        out_p = torch.empty_like(flm).pin_memory()
        plan.inverse(flm_p, out=map_p)
        assert torch.equal(map_p, ref_map)
        plan.forward(x_p, out=out_p)
        assert torch.equal(out_p, ref_flm)
    # host in, device out and device in, host out
    map_d = torch.empty(x.shape, dtype=torch.complex128, device="cuda")
    plan.inverse(flm_p, out=map_d)
    torch.cuda.synchronize()
    assert torch.equal(map_d.cpu(), ref_map)
    out_p = torch.empty_like(flm).pin_memory()
    plan.forward(x.cuda(), out=out_p)
    assert torch.equal(out_p, ref_flm)
    # pageable host buffers keep the staged path
    assert torch.equal(plan.inverse(flm), ref_map)
    plan.close()
