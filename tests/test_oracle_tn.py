"""Pins of the oracle's Trapani-Navaza planes (Sec. V-B, the alternative Delta
recursion) and of the top row it starts from.

- the top row against d^l_{l,m}(pi/2) from Jacobi's form (exact Wigner
  module) for small l, and against the closed form evaluated in 50-digit
  arithmetic for l up to 2047, where 2^-l leaves the double range;
- quarter planes against Jacobi's form (l <= 16) and against Risbo's
  recursion (l up to 511);
- the transpose symmetry Delta_{m',m} = (-1)^(m-m') Delta_{m,m'} (Eq.
  wignerd_sym3 with d(-b) = d(b)^T), which the column recursion does not
  impose: each triangle is computed from different start values;
- spot values at l = 2047 (and of Risbo's planes at l = 511) against Wigner's
  explicit sum evaluated exactly in integers (inside, on and outside the
  circle m^2 + m'^2 = l^2, and at 2^-2047);
- planted mistakes (the sign of the 2m term, a dropped factor of the
  recursion, an exponent off by one in the start values) are caught.
"""
import mpmath as mp
import numpy as np
import pytest

import oracle
from exact_wigner import delta_exact, delta_half_pi_exact


@pytest.mark.parametrize("l", [0, 1, 2, 5, 12])
def test_top_row_vs_jacobi(l):
    mant, expo = oracle.delta_top_row(l)
    got = np.ldexp(mant, expo)
    want = delta_exact(l)[2 * l, l:]
    assert np.max(np.abs(got - want)) < 1e-15


@pytest.mark.parametrize("l,ms", [(300, [0, 150, 300]), (2047, [0, 1, 1000, 1447, 2046, 2047])])
def test_top_row_far_below_double_range(l, ms):
    mp.mp.dps = 50
    mant, expo = oracle.delta_top_row(l)
    for m in ms:
        want = (-1) ** (l - m) * mp.sqrt(mp.binomial(2 * l, l + m)) * mp.mpf(2) ** (-l)
        got = mp.mpf(float(mant[m])) * mp.mpf(2) ** int(expo[m])
        assert abs(got / want - 1) < 2e-16, (l, m)


@pytest.mark.parametrize("l", [0, 1, 3, 8, 16])
def test_quarter_vs_jacobi(l):
    assert np.max(np.abs(oracle.delta_plane_tn(l) - delta_exact(l)[l:, l:])) < 1e-14


@pytest.mark.parametrize("l", [40, 200, 511])
def test_quarter_vs_risbo(l):
    D = oracle.delta_plane(l)[l:, l:]
    assert np.max(np.abs(oracle.delta_plane_tn(l) - D)) < 5e-15


@pytest.mark.parametrize("l", [9, 100, 333])
def test_transpose_symmetry(l):
    Q = oracle.delta_plane_tn(l)
    idx = np.arange(l + 1)
    sign = np.where((idx[None, :] - idx[:, None]) % 2 == 0, 1.0, -1.0)
    assert np.max(np.abs(Q - sign * Q.T)) < 5e-15


def test_planted_mistakes_are_caught(monkeypatch):
    l = 16
    ref = delta_exact(l)[l:, l:]
    good_top = oracle.delta_top_row
    # exponent off by one in the start values
    monkeypatch.setattr(oracle.mw_oracle, "delta_top_row", lambda l_: (good_top(l_)[0], good_top(l_)[1] + 1))
    assert np.max(np.abs(oracle.delta_plane_tn(l) - ref)) > 1e-3
    monkeypatch.undo()
    # sign of the 2m term flipped, or the sqrt((l-m')(l+m'+1)) factor dropped:
    # rebuild the recursion with each mistake from the oracle's own start values
    mant, expo = oracle.delta_top_row(l)
    top = np.ldexp(mant, expo)
    for mistake in ("sign", "factor"):
        m = np.arange(l + 1, dtype=np.float64)
        cur, prev = top.copy(), np.zeros(l + 1)
        out = np.zeros((l + 1, l + 1))
        out[l] = cur
        for mp_ in range(l, 0, -1):
            a = np.sqrt(float((l - mp_) * (l + mp_ + 1))) if mistake != "factor" else 1.0
            b = np.sqrt(float((l + mp_) * (l - mp_ + 1)))
            s1 = -1.0 if mistake == "sign" else 1.0
            prev, cur = cur, (s1 * 2.0 * m * cur - a * prev) / b
            out[mp_ - 1] = cur
        assert np.max(np.abs(out - ref)) > 1e-3, mistake


SPOTS = [(1, 0), (0, 1), (1000, 500), (500, 1000), (1447, 1447), (2047, 0), (2047, 2047), (1800, 300),
         (2046, 500), (100, 1999), (0, 0)]


def recursion_bound(l, D):
    """Worst-case rounding of a recursion of up to 2l dependent steps, each
    rounding at most one unit in the last place of the plane's largest
    entries: 2 l eps max|Delta| (observed errors sit 10 to 50 times below)."""
    return 2 * l * np.finfo(np.float64).eps * np.max(np.abs(D))


def test_spot_values_at_l2047():
    l = 2047
    Q = oracle.delta_plane_tn(l)
    tol = recursion_bound(l, Q)
    for a, b in SPOTS:
        assert abs(Q[a, b] - float(delta_half_pi_exact(l, a, b))) < tol, (a, b)


def test_risbo_spot_values_at_l511():
    l = 511
    D = oracle.delta_plane(l)
    tol = recursion_bound(l, D)
    for a, b in [(0, 1), (300, 200), (361, 361), (511, 0), (510, 100), (20, 499), (-7, 400), (250, -250)]:
        assert abs(D[a + l, b + l] - float(delta_half_pi_exact(l, a, b))) < tol, (a, b)
