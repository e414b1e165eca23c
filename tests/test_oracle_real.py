"""Pins of the oracle's real-signal transforms (Sec. IV-G).

- closed forms: Re(Y_lm) sampled from Wigner's explicit d sum has coefficients
  1/2 at (l, m) and (-1)^m / 2 at (l, -m) (1 at (l, 0)), both directions;
- the half-m forward agrees with the full complex forward on real maps, and the
  complex forward of a real map obeys the reality condition the half-m route
  relies on (f_{l,-m} = (-1)^m conj(f_lm));
- the displayed symmetry F_{-m,-m'} = conj(F_mm') of the theta-DFT output for
  a real spin-0 map;
- inverse_real equals the real part of the full complex inverse for any
  coefficients (not only those of a real signal);
- exact round trip on real band-limited maps;
- planted mistakes (the (-1)^m of the reality condition dropped, the conjugate
  dropped) are caught;
- the general reality condition for spin signals: conj of a spin-s signal is a
  spin -s signal with coefficients (-1)^(s+m) conj(f_{l,-m}), through both
  transforms of the complex path at s = 1, 2, -3, 4.
"""
import numpy as np
import pytest

import oracle
from exact_wigner import spin_sh
from paper_1110_6298_gb300 import workloads as wl


def grid_values(fun, L):
    th = oracle.theta_nodes(L)
    ph = oracle.phi_nodes(L)
    vals = [fun(th[t], ph[p]) for t in range(L - 1) for p in range(2 * L - 1)]
    vals.append(fun(np.pi, 0.0))
    return np.array(vals)


@pytest.mark.parametrize("l,m", [(0, 0), (1, 0), (1, 1), (2, 1), (3, 2), (3, 3), (4, 0)])
def test_real_part_of_harmonic(l, m):
    L = 5
    f = grid_values(lambda t, p: spin_sh(l, m, 0, t, p).real, L)
    want = np.zeros(L * L, dtype=np.complex128)
    if m == 0:
        want[l * l + l] = 1.0
    else:
        want[l * l + l + m] = 0.5
        want[l * l + l - m] = 0.5 * (-1) ** m
    got = oracle.forward_real(f, L)
    assert np.max(np.abs(got - want)) < 1e-14
    back = oracle.inverse_real(want, L)
    assert back.dtype == np.float64 and np.max(np.abs(back - f)) < 1e-14


@pytest.mark.parametrize("L", [1, 2, 5, 16])
def test_half_m_forward_matches_complex_forward(L):
    g = wl.rng(700 + L)
    f = np.stack([wl.gaussian_real_map(g, L) for _ in range(3)])
    full = oracle.forward(f.astype(np.complex128), L, 0)
    half = oracle.forward_real(f, L)
    assert np.max(np.abs(full - half)) < 1e-13 * max(1.0, np.max(np.abs(full)))


@pytest.mark.parametrize("L", [3, 8])
def test_reality_condition_of_complex_forward(L):
    f = wl.gaussian_real_map(wl.rng(710 + L), L)
    flm = oracle.forward(f.astype(np.complex128), L, 0)
    for l in range(L):
        for m in range(1, l + 1):
            a, b = flm[l * l + l + m], flm[l * l + l - m]
            assert abs(b - (-1) ** m * np.conj(a)) < 1e-13
        assert abs(flm[l * l + l].imag) < 1e-13


@pytest.mark.parametrize("L", [4, 9])
def test_F_symmetry(L):
    f = wl.gaussian_real_map(wl.rng(720 + L), L)
    F = oracle.theta_dft(oracle.theta_extend(oracle.phi_dft(f.astype(np.complex128), L, 0), L, 0), L)
    # F[i, j] at (m, m') = (i - L + 1, j - L + 1); (-m, -m') sits at (M-1-i, M-1-j)
    assert np.max(np.abs(F[::-1, ::-1] - np.conj(F))) < 1e-14


@pytest.mark.parametrize("L", [1, 2, 6, 13])
def test_inverse_real_is_real_part_of_inverse(L):
    g = wl.rng(730 + L)
    flm = np.stack([wl.uniform_flm(g, L, 0) for _ in range(2)])
    a = oracle.inverse_real(flm, L)
    b = oracle.inverse(flm, L, 0).real
    assert a.shape == b.shape and np.max(np.abs(a - b)) < 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("L", [2, 7, 32])
def test_round_trip(L):
    flm = wl.uniform_flm_real(wl.rng(740 + L), L)
    f = oracle.inverse_real(flm, L)
    assert np.max(np.abs(oracle.forward_real(f, L) - flm)) < 1e-12
    assert np.max(np.abs(oracle.hermitian_part(flm, L) - flm)) == 0.0


def test_planted_mistakes_are_caught(monkeypatch):
    L, l, m = 5, 3, 1
    f = grid_values(lambda t, p: spin_sh(l, m, 0, t, p).real, L)
    want = np.zeros(L * L, dtype=np.complex128)
    want[l * l + l + m] = 0.5
    want[l * l + l - m] = -0.5
    assert np.max(np.abs(oracle.forward_real(f, L) - want)) < 1e-14
    # (-1)^m dropped
    monkeypatch.setattr(oracle.mw_oracle, "_neg_m_sign", lambda L_: np.ones(L_ * L_))
    assert np.max(np.abs(oracle.forward_real(f, L) - want)) > 0.5
    monkeypatch.undo()
    # conjugate dropped in the Hermitian part: the inverse of i Y_11 + c.c. breaks
    c = np.zeros(L * L, dtype=np.complex128)
    c[1 * 1 + 1 + 1] = 0.5j
    c[1 * 1 + 1 - 1] = 0.5j  # (-1)^1 conj(0.5 i)
    good = oracle.inverse_real(c, L)
    monkeypatch.setattr(oracle.mw_oracle, "hermitian_part",
                        lambda x, L_: 0.5 * (x + oracle.mw_oracle._neg_m_sign(L_) * x[..., oracle.mw_oracle._mirror_index(L_)]))
    assert np.max(np.abs(oracle.inverse_real(c, L) - good)) > 0.1


@pytest.mark.parametrize("L,s", [(4, 1), (6, 2), (7, -3), (5, 4)])
def test_spin_reality_condition(L, s):
    # Sec. IV-G: for a spin-s signal f, conj(f) is a spin -s signal with
    # coefficients (-1)^(s+m) conj(f_{l,-m}); checked through both transforms
    flm = wl.uniform_flm(wl.rng(750 + L), L, s)
    f = oracle.inverse(flm, L, s)
    g = oracle.forward(np.conj(f), L, -s)
    ell = wl.ell_of_index(L)
    m = np.arange(L * L) - ell * ell - ell
    mirror = ell * ell + ell - m
    want = np.where((s + m) % 2 == 0, 1.0, -1.0) * np.conj(flm[mirror])
    assert np.max(np.abs(g - want)) < 1e-12
    # and the synthesis side: inverse of those coefficients with spin -s is conj(f)
    assert np.max(np.abs(oracle.inverse(want, L, -s) - np.conj(f))) < 1e-12
