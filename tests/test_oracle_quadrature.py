"""Pins of the oracle's MW quadrature rule (Sec. IV-F, Eq. quadrature).

- the sample count L(L-1)+1 stated in Sec. IV-F;
- v(theta_t) equals the band-limited samples of sin(theta) on [0, pi), zero on
  [pi, 2pi) (the statement after the weights' definition), with Fourier
  coefficients computed here by numerical integration, not by the closed form
  of w(k);
- exactness: every spin-0 harmonic Y_lm with l < L, evaluated by Wigner's
  explicit sum, integrates to sqrt(4 pi) delta_{l0} delta_{m0};
- spin s != 0: the rule reproduces 2 pi int_0^pi sY_l0 sin(theta) dtheta
  (numerical integration of the explicit harmonic) and 0 for m != 0;
- planted mistakes (the pole fold without the Kronecker delta, the (-1)^s
  factor dropped) are caught by these checks.
"""
import mpmath as mp
import numpy as np
import pytest
from scipy import integrate

import oracle
from exact_wigner import d_sum, spin_sh

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def q_grid_values(fun, L):
    """Samples of fun(theta, phi) in the quadrature layout (L-1 rings of L, pole)."""
    th = oracle.theta_nodes(L)
    ph = oracle.quadrature_phi_nodes(L)
    out = [fun(th[t], ph[p]) for t in range(L - 1) for p in range(L)]
    out.append(fun(np.pi, 0.0))
    return np.array(out, dtype=np.complex128)


@pytest.mark.parametrize("L,n", [(1, 1), (2, 3), (4, 13), (64, 4033)])
def test_sample_count(L, n):
    assert oracle.quadrature_sample_count(L) == n


@pytest.mark.parametrize("L", [4, 16])
def test_v_is_band_limited_half_sine(L):
    # Fourier coefficients of g = sin(theta) on [0, pi), 0 on [pi, 2 pi), by quadrature
    M = 2 * L - 1
    ks = np.arange(-(L - 1), L)
    gk = []
    for k in ks:
        re = integrate.quad(lambda x: np.sin(x) * np.cos(k * x), 0, np.pi, epsabs=1e-14)[0]
        im = integrate.quad(lambda x: -np.sin(x) * np.sin(k * x), 0, np.pi, epsabs=1e-14)[0]
        gk.append(re + 1j * im)
    th = oracle.theta_nodes(L, extended=True)
    g_L = (np.array(gk)[None, :] * np.exp(1j * np.outer(th, ks))).sum(axis=1) / (2 * np.pi)
    v = oracle.quadrature_v(L)
    assert np.max(np.abs(v - (2 * np.pi / M) * g_L.real)) < 1e-13
    assert np.max(np.abs(g_L.imag)) < 1e-13


@pytest.mark.parametrize("L", [1, 3, 5])
def test_exact_on_spin0_harmonics(L):
    for l in range(L):
        for m in range(-l, l + 1):
            f = q_grid_values(lambda t, p: spin_sh(l, m, 0, t, p), L)
            got = oracle.quadrature_integrate(f, L, 0)
            want = np.sqrt(4 * np.pi) if l == 0 else 0.0
            assert abs(got - want) < 1e-13, (L, l, m, got)


def _theta_integral(l, s):
    """2 pi int_0^pi sY_l0(theta) sin(theta) dtheta of the explicit harmonic."""
    f = lambda x: float((-1) ** s * np.sqrt((2 * l + 1) / (4 * np.pi))
                        * float(d_sum(2 * l, 0, -2 * s, mp.mpf(x))) * np.sin(x))
    return 2 * np.pi * integrate.quad(f, 0, np.pi, epsabs=1e-14, limit=200)[0]


@pytest.mark.parametrize("s", [1, -2])
def test_spin_integrals(s):
    L = 5
    for l in range(abs(s), L):
        for m in (-1, 0, 2):
            if abs(m) > l:
                continue
            f = q_grid_values(lambda t, p: spin_sh(l, m, s, t, p), L)
            got = oracle.quadrature_integrate(f, L, s)
            want = _theta_integral(l, s) if m == 0 else 0.0
            assert abs(got - want) < 1e-12, (s, l, m, got, want)


def test_samples_helper_matches_explicit_synthesis():
    L, s = 4, 1
    rng = np.random.default_rng(3)
    flm = np.zeros(L * L, dtype=np.complex128)
    for l in range(abs(s), L):
        for m in range(-l, l + 1):
            flm[l * l + l + m] = rng.normal() + 1j * rng.normal()
    fun = lambda t, p: sum(flm[l * l + l + m] * spin_sh(l, m, s, t, p)
                           for l in range(abs(s), L) for m in range(-l, l + 1))
    assert np.max(np.abs(oracle.quadrature_samples(flm, L, s) - q_grid_values(fun, L))) < 1e-12


def test_planted_mistakes_are_caught(monkeypatch):
    L = 4
    ones = q_grid_values(lambda t, p: spin_sh(0, 0, 0, t, p), L)
    good = oracle.quadrature_weights
    # pole folded twice (Kronecker delta dropped)
    def no_delta(L_, s_=0):
        v = oracle.quadrature_v(L_)
        t = np.arange(L_)
        sg = -1.0 if (s_ % 2) else 1.0
        return 2 * np.pi / L_ * (v[:L_] + sg * v[2 * L_ - 2 - t])
    monkeypatch.setattr(oracle.mw_oracle, "quadrature_weights", no_delta)
    assert abs(oracle.quadrature_integrate(ones, L, 0) - np.sqrt(4 * np.pi)) > 1e-3
    # (-1)^s dropped: the spin-1 integral of 1Y_10 changes
    def no_sign(L_, s_=0):
        return good(L_, 0)
    monkeypatch.setattr(oracle.mw_oracle, "quadrature_weights", no_sign)
    f = q_grid_values(lambda t, p: spin_sh(1, 0, 1, t, p), 5)
    assert abs(oracle.quadrature_integrate(f, 5, 1) - _theta_integral(1, 1)) > 1e-3
