"""Fused forward+inverse (one shared Wigner-Delta recursion) against the two
separate calls: the results must be bitwise equal, because the planes do not
depend on the direction and every kernel runs in a fixed order.  Covers both
precisions, uniform and ragged plans, host buffers and graph replay, plus the
oracle at one small size.
"""
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


def inputs(mw, L, spins, seed):
    g = wl.rng(9000 + seed)
    flm = np.stack([wl.gaussian_flm(g, L, s, wl.cl_white) for s in spins])
    maps = np.stack([wl.gaussian_map(g, L) for _ in spins])
    return torch.from_numpy(maps).cuda(), torch.from_numpy(flm).cuda()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tf32"])
@pytest.mark.parametrize("L,spins", [(1, [0]), (7, [0, -2]), (130, [1, 0, 2]), (300, [0] * 9 + [2])])
def test_fused_equals_separate_calls(mw, precision, L, spins):
    maps, flm = inputs(mw, L, spins, L)
    plan = mw.Plan(L, spins, precision=precision)
    f_sep = plan.forward(maps)
    m_sep = plan.inverse(flm)
    f_fu, m_fu = plan.forward_inverse(maps, flm)
    plan.sync()
    assert torch.equal(f_fu, f_sep)
    assert torch.equal(m_fu, m_sep)
    # and a second fused call on the same plan (twin workspace reused)
    f2, m2 = plan.forward_inverse(maps, flm)
    plan.sync()
    assert torch.equal(f2, f_sep) and torch.equal(m2, m_sep)


def test_fused_against_oracle(mw):
    L, spins = 24, [0, 1]
    maps, flm = inputs(mw, L, spins, 5)
    plan = mw.Plan(L, spins, precision="fp64")
    f, m = plan.forward_inverse(maps, flm)
    plan.sync()
    for b, s in enumerate(spins):
        fo = oracle.forward(maps[b].cpu().numpy(), L, s)
        mo = oracle.inverse(flm[b].cpu().numpy(), L, s)
        assert np.max(np.abs(f[b].cpu().numpy() - fo)) / np.max(np.abs(fo)) < 1e-12
        assert np.max(np.abs(m[b].cpu().numpy() - mo)) / np.max(np.abs(mo)) < 1e-12


def test_fused_ragged_equals_separate(mw):
    Ls, spins = [64, 128, 64, 200], [0, -1, 2, 1]
    plan = mw.RaggedPlan(Ls, spins, precision="mixed")
    g = wl.rng(77)
    flm = torch.from_numpy(np.concatenate([wl.gaussian_flm(g, L, s, wl.cl_white) for L, s in zip(Ls, spins)])).cuda()
    maps = torch.from_numpy(np.concatenate([wl.gaussian_map(g, L) for L in Ls])).cuda()
    f_sep, m_sep = plan.forward(maps), plan.inverse(flm)
    f_fu, m_fu = plan.forward_inverse(maps, flm)
    plan.sync()
    assert torch.equal(f_fu, f_sep) and torch.equal(m_fu, m_sep)


def test_fused_host_buffers_and_graph(mw):
    L, spins = 96, [0, 2, 0]
    maps, flm = inputs(mw, L, spins, 3)
    ref = mw.Plan(L, spins, precision="mixed")
    f_ref, m_ref = ref.forward_inverse(maps, flm)
    ref.sync()
    # host (pinned and pageable) buffers through the C ABI
    hm, hf = maps.cpu().pin_memory(), flm.cpu()
    f_h, m_h = ref.forward_inverse(hm, hf)
    assert torch.equal(f_h, f_ref.cpu()) and torch.equal(m_h, m_ref.cpu())
    # graph capture: first call captures, the second replays as one launch
    gp = mw.Plan(L, spins, precision="mixed", graph=True)
    fo = torch.empty_like(f_ref)
    mo = torch.empty_like(m_ref)
    gp.forward_inverse(maps, flm, fo, mo)
    gp.forward_inverse(maps, flm, fo, mo)
    gp.sync()
    assert gp.last_launches == 1
    assert torch.equal(fo, f_ref) and torch.equal(mo, m_ref)
