"""Ragged batches (maps of different band limit and spin in one plan, one
shared Wigner-Delta sweep) and whole-call CUDA graphs.

Workload: 64 maps, L uniform on {64,128,256,384,512}, s uniform on
{0,+1,-1,+2,-2}, E|f_lm|^2 = 1/(l+1)^2 (zero for l < |s|), mixed precision.
The ragged result must equal, bit for bit, the per-band-limit plans (the planes
do not depend on L, the chunk boundaries coincide), and sampled maps must match
the FP64 oracle within the mixed-path bar."""
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


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def test_ragged_inverse_forward_matches_uniform_plans_and_oracle(mw):
    w = wl.workload_ragged()
    Ls, spins, flms = w["Ls"], w["spins"], w["flm"]
    plan = mw.RaggedPlan(Ls, spins, precision="mixed")
    flat = torch.from_numpy(np.concatenate(flms)).cuda()
    maps = plan.inverse(flat)
    back = plan.forward(maps)
    plan.sync()
    maps_np, back_np = maps.cpu().numpy(), back.cpu().numpy()
    mo, fo = plan.map_offsets, plan.flm_offsets
    # bitwise equality with one uniform plan per band limit
    for L in sorted(set(Ls)):
        idx = [b for b, x in enumerate(Ls) if x == L]
        up = mw.Plan(L, [spins[b] for b in idx], precision="mixed")
        um = up.inverse(torch.from_numpy(np.stack([flms[b] for b in idx])).cuda()).cpu().numpy()
        ub = up.forward(torch.from_numpy(um).cuda()).cpu().numpy()
        for k, b in enumerate(idx):
            assert np.array_equal(maps_np[mo[b]:mo[b] + mw.map_size(L)], um[k])
            assert np.array_equal(back_np[fo[b]:fo[b] + L * L], ub[k])
    # oracle on one map of every band limit
    seen = set()
    for b, (L, s) in enumerate(zip(Ls, spins)):
        if L in seen:
            continue
        seen.add(L)
        ref = oracle.inverse(flms[b], L, s)
        assert relmax(maps_np[mo[b]:mo[b] + mw.map_size(L)], ref) < 1e-6
        assert np.max(np.abs(back_np[fo[b]:fo[b] + L * L] - flms[b])) / np.max(np.abs(flms[b])) < 1e-6


def test_ragged_fp64_small(mw):
    Ls, spins = [9, 33, 17, 33, 65], [0, 2, -1, -3, 1]
    g = wl.rng(123)
    flms = [wl.gaussian_flm(g, L, s, wl.cl_red) for L, s in zip(Ls, spins)]
    plan = mw.RaggedPlan(Ls, spins, precision="fp64")
    maps = plan.inverse(torch.from_numpy(np.concatenate(flms)).cuda()).cpu().numpy()
    for b, (L, s) in enumerate(zip(Ls, spins)):
        ref = oracle.inverse(flms[b], L, s)
        assert relmax(maps[plan.map_offsets[b]:plan.map_offsets[b] + mw.map_size(L)], ref) < 1e-12
    x = [wl.gaussian_map(g, L) for L in Ls]
    fwd = plan.forward(torch.from_numpy(np.concatenate(x)).cuda()).cpu().numpy()
    for b, (L, s) in enumerate(zip(Ls, spins)):
        ref = oracle.forward(x[b], L, s)
        assert relmax(fwd[plan.flm_offsets[b]:plan.flm_offsets[b] + L * L], ref) < 1e-12


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_replay_matches_direct(mw, prec):
    L, spins = 96, [0, 2, -1]
    g = wl.rng(7)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])).cuda()
    direct = mw.Plan(L, spins, precision=prec)
    graphed = mw.Plan(L, spins, precision=prec, graph=True)
    a = direct.inverse(flm)
    out = torch.empty_like(a)
    for _ in range(3):  # capture, then replays
        graphed.inverse(flm, out=out)
    graphed.sync()
    assert graphed.last_launches == 1  # replayed as one graph launch
    assert torch.equal(a, out)
    b1 = direct.forward(a)
    b2 = torch.empty_like(b1)
    for _ in range(2):
        graphed.forward(a, out=b2)
    assert graphed.last_launches == 1
    assert torch.equal(b1, b2)


def test_graph_replay_on_a_side_stream(mw):
    L, spins = 64, [0, 1]
    g = wl.rng(8)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])).cuda()
    ref = mw.Plan(L, spins, precision="mixed").inverse(flm)
    graphed = mw.Plan(L, spins, precision="mixed", graph=True)
    out = torch.empty_like(ref)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            graphed.inverse(flm, out=out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    assert graphed.last_launches == 1
    assert torch.equal(out, ref)


def test_plan_layout_queries(mw):
    """The layout the C ABI reports for a plan (mw_plan_batch / band_limit /
    spin / map_offset / flm_offset) equals the host-only mw_layout_ragged
    prefix sums for a ragged plan, b * N_MW and b * L^2 for uniform and real
    plans, and -1 past the last map."""
    w = wl.workload_ragged()
    Ls, spins = w["Ls"], w["spins"]
    plan = mw.RaggedPlan(Ls, spins, precision="mixed")
    mo, fo = mw.layout_ragged(Ls)
    lay = plan.layout()
    assert [x[0] for x in lay] == Ls and [x[1] for x in lay] == spins
    assert [x[2] for x in lay] == mo[:-1] and [x[3] for x in lay] == fo[:-1]
    assert mo[-1] == plan._nmap and fo[-1] == plan._nflm
    assert mw.lib().mw_plan_map_offset(plan.handle, len(Ls)) == -1
    up = mw.Plan(40, [0, 2, -1], precision="fp64")
    assert up.layout() == [(40, s, b * mw.map_size(40), b * 1600) for b, s in enumerate([0, 2, -1])]
    rp = mw.RealPlan(17, 3, precision="mixed")
    assert rp.layout() == [(17, 0, b * mw.map_size(17), b * 289) for b in range(3)]
