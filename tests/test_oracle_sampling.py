"""Pins of the sampling layer of the oracle (Sec. IV-C, Sec. V-A) and of the
quadrature weights (Sec. IV-D) against the paper's printed values and against
numerical integration."""
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_sample_counts_golden():
    for L, nmw, ngl, ndh in _rows("sample_counts.txt"):
        L = int(L)
        assert oracle.sample_count(L) == int(nmw)
        assert L * (2 * L - 1) == int(ngl)
        assert 2 * L * (2 * L - 1) == int(ndh)


def test_l2_bound_reached_only_for_l1_l2():
    # Sec. V-A: N_MW reaches the L^2 degrees of freedom only for L in {1, 2}
    hits = [L for L in range(1, 200) if oracle.sample_count(L) == L * L]
    assert hits == [1, 2]
    assert all(oracle.sample_count(L) >= L * L for L in range(1, 200))


def test_mri_example_golden():
    (bls, gl, mw, pct), = _rows("mri_shells.txt")
    Ls = [int(x) for x in bls.split(",")]
    tot_gl = sum(L * (2 * L - 1) for L in Ls)
    tot_mw = sum(oracle.sample_count(L) for L in Ls)
    assert (tot_gl, tot_mw) == (int(gl), int(mw))
    assert round(100 * (tot_gl - tot_mw) / tot_gl) == int(pct)
    # the reading: N_GL - N_MW = 2(L-1)
    assert all(L * (2 * L - 1) - oracle.sample_count(L) == 2 * (L - 1) for L in range(1, 50))


def test_nodes():
    for L in (1, 2, 3, 8, 33):
        th = oracle.theta_nodes(L)
        the = oracle.theta_nodes(L, extended=True)
        ph = oracle.phi_nodes(L)
        M = 2 * L - 1
        assert len(th) == L and len(ph) == M and len(the) == M
        assert np.isclose(th[-1], np.pi)              # last ring is the south pole
        assert th[0] > 0                              # no sample at the north pole
        # symmetric about pi: theta_{2L-2-t} = 2 pi - theta_t
        assert np.allclose(the[2 * L - 2 - np.arange(M)], 2 * np.pi - the)
        assert np.allclose(np.diff(ph), 2 * np.pi / M) and ph[0] == 0


def test_weights_golden_and_quadrature():
    for k, re, im in _rows("weights.txt"):
        w = oracle.weight(np.array([int(k)]))[0]
        assert abs(w - (float(re) + 1j * float(im))) < 1e-15
    for k in range(-25, 26):
        cr, _ = integrate.quad(lambda t: np.sin(t) * np.cos(k * t), 0, np.pi, limit=200, epsabs=1e-14)
        ci, _ = integrate.quad(lambda t: np.sin(t) * np.sin(k * t), 0, np.pi, limit=200, epsabs=1e-14)
        w = oracle.weight(np.array([k]))[0]
        assert abs(w - (cr + 1j * ci)) < 1e-12, k


@pytest.mark.parametrize("L", [1, 2, 5, 16, 64])
def test_weight_convolution_direct_vs_paper_fft(L):
    # Eq. (Gmm_convolution) written out vs the zero-padded FFT route of Sec. IV-D
    g = np.random.default_rng(L)
    M = 2 * L - 1
    F = g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))
    a = oracle.weight_convolution(F, L)
    for N in (4 * L - 3, 4 * L + 7, 2 * (4 * L - 3)):
        b = oracle.weight_convolution_fft(F, L, N)
        assert np.max(np.abs(a - b)) < 1e-11 * max(1, np.max(np.abs(a)))
    with pytest.raises(ValueError):
        oracle.weight_convolution_fft(F, L, 4 * L - 4)
