"""GPU parity of plans whose Wigner planes come from the Trapani-Navaza
recursion (MW_FLAG_DELTA_TN; Sec. V-B cites it as the alternative to Risbo's),
through the C ABI, against the oracle and against Risbo plans.

Tolerance 1e-6 relative (the mixed precisions).  Sizes span several 256-column
blocks with ragged tails (L = 257, 300), the degenerate cases (L = 1, 2,
|s| = L-1), mixed-spin batches, fused, ragged, real-signal and graph-replayed
calls, and the full L = 2048 x 16 workload on sampled outputs, where the start
values of the recursion reach 2^-2047.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402

TOL = 1e-6


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
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def by_spin(fn, x, L, spins):
    out = [None] * len(spins)
    for s in sorted(set(spins)):
        idx = [b for b, t in enumerate(spins) if t == s]
        r = fn(x[idx], L, s)
        for k, b in enumerate(idx):
            out[b] = r[k]
    return np.stack(out)


CASES = [(1, [0]), (2, [1, 0, -1]), (7, [-3, 0]), (65, [2, -1, 0]), (257, [0, 3]), (300, [1, -2])]


@pytest.mark.parametrize("prec", ["mixed", "mixed_tf32"])
@pytest.mark.parametrize("L,spins", CASES)
def test_inverse_and_forward(mw, prec, L, spins):
    g = wl.rng(4000 + L)
    flm = np.stack([wl.gaussian_flm(g, L, s, wl.cl_white) for s in spins])
    maps = np.stack([wl.gaussian_map(g, L) for _ in spins])
    plan = mw.Plan(L, spins, precision=prec, delta="tn")
    f = plan.inverse(torch.from_numpy(flm).cuda())
    c = plan.forward(torch.from_numpy(maps).cuda())
    plan.sync()
    ref_f = by_spin(oracle.inverse, flm, L, spins)
    ref_c = by_spin(oracle.forward, maps, L, spins)
    for b in range(len(spins)):
        assert relmax(f[b].cpu().numpy(), ref_f[b]) < TOL, ("inverse", b)
        assert relmax(c[b].cpu().numpy(), ref_c[b]) < TOL, ("forward", b)


def test_agrees_with_risbo_plans(mw):
    L, spins = 400, [0, 2, -5]
    g = wl.rng(4100)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_white) for s in spins])).cuda()
    a = mw.Plan(L, spins, precision="mixed", delta="tn")
    b = mw.Plan(L, spins, precision="mixed")
    fa, fb = a.inverse(flm), b.inverse(flm)
    ca, cb = a.forward(fa), b.forward(fa)
    a.sync()
    b.sync()
    assert relmax(fa.cpu().numpy(), fb.cpu().numpy()) < TOL
    assert relmax(ca.cpu().numpy(), cb.cpu().numpy()) < TOL


def test_fused_ragged_real_graph(mw):
    L, spins = 96, [0, 1, 0]
    g = wl.rng(4200)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_white) for s in spins])).cuda()
    maps = torch.from_numpy(np.stack([wl.gaussian_map(g, L) for _ in spins])).cuda()
    plan = mw.Plan(L, spins, precision="mixed", graph=True, delta="tn")
    f_sep, m_sep = plan.forward(maps), plan.inverse(flm)
    f_fu, m_fu = plan.forward_inverse(maps, flm)
    f_g, m_g = plan.forward_inverse(maps, flm)  # graph replay
    plan.sync()
    assert torch.equal(f_fu, f_sep) and torch.equal(m_fu, m_sep)
    assert torch.equal(f_g, f_sep) and torch.equal(m_g, m_sep)
    assert plan.last_launches == 1
    # ragged: maps of several band limits, one recursion to the largest
    Ls, rs = [64, 160, 64, 130], [0, -1, 2, 1]
    rp = mw.RaggedPlan(Ls, rs, precision="mixed", delta="tn")
    fl = [wl.gaussian_flm(g, Lb, s, wl.cl_white) for Lb, s in zip(Ls, rs)]
    out = rp.inverse(torch.from_numpy(np.concatenate(fl)).cuda()).cpu().numpy()
    rp.sync()
    for k, (Lb, s) in enumerate(zip(Ls, rs)):
        o = rp.map_offsets[k]
        assert relmax(out[o:o + wl.map_size(Lb)], oracle.inverse(fl[k], Lb, s)) < TOL
    # real signals
    c = np.stack([wl.uniform_flm_real(wl.rng(4300 + b), L) for b in range(3)])
    real = mw.RealPlan(L, 3, precision="mixed", delta="tn")
    x = real.inverse(torch.from_numpy(c).cuda()).cpu().numpy()
    real.sync()
    ref = oracle.inverse_real(c, L)
    for b in range(3):
        assert relmax(x[b], ref[b]) < TOL


def test_fp64_rejected(mw):
    with pytest.raises(mw.MWError) as ei:
        mw.Plan(16, [0], precision="fp64", delta="tn")
    assert ei.value.status == mw.MW_EUNSUPPORTED


def test_full_size_l2048_b16_sampled(mw):
    """The benchmarked workload (L = 2048, 16 maps: 8 of spin 0, 8 of spin 2)
    on a Trapani-Navaza plan: three rings of the inverse against the oracle's
    ring synthesis, eight m columns of the forward of the GPU maps against the
    oracle's forward restricted to those m, and the round trip."""
    w = wl.workload_l2048_b16()
    L, spins = w["L"], w["spins"]
    flm = np.stack(w["flm"])
    plan = mw.Plan(L, spins, precision="mixed", delta="tn")
    f_gpu = plan.inverse(torch.from_numpy(flm).cuda())
    back = plan.forward(f_gpu).cpu().numpy()
    plan.sync()
    f_np = f_gpu.cpu().numpy()
    M = 2 * L - 1
    rings = [0, 1023, L - 2]
    ms = [-2047, -1000, -3, 0, 2, 517, 1999, 2047]
    ell = wl.ell_of_index(L)
    sel = np.isin(np.arange(L * L) - ell * ell - ell, ms)
    for s, idx in ((0, [0, 7]), (2, [8, 15])):
        ref_r = oracle.inverse_rings(flm[idx], L, s, rings)
        ref_f = oracle.forward(f_np[idx], L, s, m_list=ms)
        for k, b in enumerate(idx):
            got_r = np.stack([f_np[b][t * M:(t + 1) * M] for t in rings])
            assert relmax(got_r, ref_r[k]) < TOL
            assert relmax(back[b][sel], ref_f[k][sel]) < TOL
            assert np.max(np.abs(back[b] - flm[b])) / np.max(np.abs(flm[b])) < TOL
