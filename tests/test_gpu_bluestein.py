"""GPU parity of the length-(2L-1) DFTs run by Bluestein's chirp-z convolution.

2L-1 is the number of phi samples per ring and of theta nodes after the
periodic extension (Sec. IV-C).  Where its prime factors are large (2L-1 = 127
at L = 64, 599 at L = 300 and 4093 at L = 2047 are prime; 767 = 13 * 59 at
L = 384) the plan runs those DFTs as a convolution of power-of-two length
instead of mixed-radix stages.  These tests compare every transform of such
plans with the FP64 oracle (1e-12 FP64, 1e-6 mixed), force the Bluestein route
(MW_FFT_BLUESTEIN=1, read at plan creation) on small and smooth lengths
including the degenerate L = 1 and 2, force the mixed-radix route at prime
lengths, and check the full-size prime case L = 2047 on sampled outputs.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402

TOL = {"fp64": 1e-12, "mixed": 1e-6}


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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def plan_with(mw, L, spins, prec, route=None, **kw):
    """A plan built with MW_FFT_BLUESTEIN set to `route` ("0", "1" or None for
    the plan's own choice) during its creation only."""
    old = os.environ.pop("MW_FFT_BLUESTEIN", None)
    try:
        if route is not None:
            os.environ["MW_FFT_BLUESTEIN"] = route
        return mw.Plan(L, spins, precision=prec, **kw)
    finally:
        os.environ.pop("MW_FFT_BLUESTEIN", None)
        if old is not None:
            os.environ["MW_FFT_BLUESTEIN"] = old


def by_spin(fn, x, L, spins):
    out = [None] * len(spins)
    for s in sorted(set(spins)):
        idx = [b for b, t in enumerate(spins) if t == s]
        r = fn(x[idx], L, s)
        for k, b in enumerate(idx):
            out[b] = r[k]
    return np.stack(out)


def check_all(mw, plan, L, spins, prec, seed):
    """inverse, forward of a non-band-limited map and both adjoints against the oracle"""
    g = wl.rng(4100 + seed)
    flm = np.stack([wl.gaussian_flm(g, L, s, wl.cl_white) for s in spins])
    x = np.stack([wl.gaussian_map(g, L) for _ in spins])
    tol = TOL[prec]
    got = plan.inverse(torch.from_numpy(flm).cuda()).cpu().numpy()
    assert relmax(got, by_spin(oracle.inverse, flm, L, spins)) < tol
    got = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(got, by_spin(oracle.forward, x, L, spins)) < tol
    got = plan.forward_adjoint(torch.from_numpy(flm).cuda()).cpu().numpy()
    assert relmax(got, by_spin(oracle.forward_adjoint, flm, L, spins)) < tol
    got = plan.inverse_adjoint(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(got, by_spin(oracle.inverse_adjoint, x, L, spins)) < tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,spins", [(64, [0, 2]), (300, [1, -2]), (384, [0])])
def test_prime_lengths_choose_bluestein(mw, prec, L, spins):
    """2L-1 = 127, 599 (prime) and 767 = 13 * 59: the plan's own choice is
    Bluestein, and every transform matches the oracle."""
    plan = plan_with(mw, L, spins, prec)
    assert plan.fft_bluestein
    check_all(mw, plan, L, spins, prec, L)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,spins", [(1, [0]), (2, [1, 0]), (3, [0, -2]), (7, [3]), (32, [0]), (65, [2, -1])])
def test_forced_bluestein_any_length(mw, prec, L, spins):
    """Bluestein at smooth and tiny lengths (2L-1 = 1, 3, 5, 13, 63, 129)."""
    plan = plan_with(mw, L, spins, prec, route="1")
    assert plan.fft_bluestein
    check_all(mw, plan, L, spins, prec, 7 * L)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_forced_mixed_radix_at_prime_length(mw, prec):
    """The mixed-radix route (one 599-term dot-product stage) still matches."""
    L, spins = 300, [0, 2]
    plan = plan_with(mw, L, spins, prec, route="0")
    assert not plan.fft_bluestein
    check_all(mw, plan, L, spins, prec, 3)
    plan.close()


def test_smooth_length_keeps_mixed_radix(mw):
    """2L-1 = 4095 = 3^2 5 7 13 (the benchmarked band limit) stays mixed radix."""
    plan = plan_with(mw, 2048, [0], "mixed")
    assert not plan.fft_bluestein
    plan.close()


def test_ragged_and_real_plans(mw):
    """Ragged plans pick the route per band limit; real-signal plans use it too."""
    old = os.environ.pop("MW_FFT_BLUESTEIN", None)
    try:
        Ls, ss = [64, 65, 300], [0, 1, -2]
        rp = mw.RaggedPlan(Ls, ss, precision="mixed")
        assert rp.fft_bluestein
        g = wl.rng(4242)
        fl = [wl.gaussian_flm(g, L, s, wl.cl_white) for L, s in zip(Ls, ss)]
        out = rp.inverse(torch.from_numpy(np.concatenate(fl)).cuda()).cpu().numpy()
        for k, (L, s) in enumerate(zip(Ls, ss)):
            o = rp.map_offsets[k]
            assert relmax(out[o:o + wl.map_size(L)], oracle.inverse(fl[k], L, s)) < TOL["mixed"]
        rp.close()
        L = 300
        real = mw.RealPlan(L, 3, precision="mixed")
        assert real.fft_bluestein
        c = np.stack([wl.uniform_flm_real(wl.rng(4300 + b), L) for b in range(3)])
        got = real.inverse(torch.from_numpy(c).cuda()).cpu().numpy()
        assert relmax(got, oracle.inverse_real(c, L)) < TOL["mixed"]
        back = real.forward(torch.from_numpy(got).cuda()).cpu().numpy()
        assert relmax(back, c) < 1e-6
        real.close()
    finally:
        if old is not None:
            os.environ["MW_FFT_BLUESTEIN"] = old


RINGS_2047 = [0, 1, 1023, 2045]
MS_2047 = [-2046, -2045, -1, 0, 1, 1500, 2046]
_REF = {}


def _ref_2047(mw):
    """Oracle references at L = 2047, computed once for both precisions: the
    workload's coefficients, the oracle's sampled rings of the spin-0 map, the
    FP64 plan's inverse (band-limited input of the forward checks) and the
    oracle forward of its spin-0 map on sampled m columns."""
    if not _REF:
        L, spins = 2047, [0, 2]
        g = wl.rng(2047)
        flm = np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])
        _REF["flm"] = flm
        _REF["rings"] = oracle.inverse_rings(flm[:1], L, 0, RINGS_2047 + [L - 1])[0]
        p64 = plan_with(mw, L, spins, "fp64")
        _REF["maps64"] = p64.inverse(torch.from_numpy(flm).cuda()).cpu().numpy()
        p64.close()
        _REF["fwd"] = oracle.forward(_REF["maps64"][:1], L, 0, m_list=MS_2047)[0]
    return _REF


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_prime_l2047(mw, prec):
    """L = 2047 (2L-1 = 4093 prime), one map of spin 0 and one of spin 2: the
    inverse on sampled rings and the pole and the forward on sampled m columns
    against the oracle (spin 0), the Bluestein plan against a plan forced onto
    the 4093-term dot-product stages (spin 2, every output), and the round
    trip."""
    L, spins = 2047, [0, 2]
    ref = _ref_2047(mw)
    flm, x64 = ref["flm"], ref["maps64"]
    plan = plan_with(mw, L, spins, prec)
    assert plan.fft_bluestein
    f_gpu = plan.inverse(torch.from_numpy(flm).cuda())
    back = plan.forward(f_gpu).cpu().numpy()
    f_np = f_gpu.cpu().numpy()
    del f_gpu
    tol = TOL[prec]
    M = 2 * L - 1
    ref_r = ref["rings"]
    got_r = np.stack([f_np[0][t * M:(t + 1) * M] for t in RINGS_2047])
    assert relmax(got_r, ref_r[:-1]) < tol
    assert abs(f_np[0][(L - 1) * M] - ref_r[-1][0]) / np.max(np.abs(ref_r)) < tol
    ell = wl.ell_of_index(L)
    sel = np.isin(np.arange(L * L) - ell ** 2 - ell, MS_2047)
    fx = plan.forward(torch.from_numpy(x64).cuda()).cpu().numpy()
    assert relmax(fx[0][sel], ref["fwd"][sel]) < tol
    for b in range(2):
        assert np.max(np.abs(back[b] - flm[b])) / np.max(np.abs(flm[b])) < (1e-11 if prec == "fp64" else 1e-6)
    direct = plan_with(mw, L, spins, prec, route="0")
    assert not direct.fft_bluestein
    f_d = direct.inverse(torch.from_numpy(flm).cuda()).cpu().numpy()
    assert relmax(f_d[1], f_np[1]) < 2 * tol
    b_d = direct.forward(torch.from_numpy(x64).cuda()).cpu().numpy()
    assert relmax(b_d[1], fx[1]) < 2 * tol
    direct.close()
    plan.close()
