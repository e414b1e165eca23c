"""Pins of the oracle's Risbo recursion against the paper's explicit Wigner
d-function (Eq. wignerd_b) and the identities of Sec. III-C."""
import mpmath as mp
import numpy as np
import pytest

import oracle
from exact_wigner import d_jacobi, d_sum, delta_exact


@pytest.mark.parametrize("beta", [0.3, 1.1, np.pi / 2, 2.9])
def test_risbo_vs_jacobi_form_half_and_integer_j(beta):
    for two_j in range(0, 21):
        D = oracle.wigner_plane(two_j, beta)
        P = two_j + 1
        E = np.array([[float(d_jacobi(two_j, 2 * i - two_j, 2 * k - two_j, beta)) for k in range(P)]
                      for i in range(P)])
        assert np.max(np.abs(D - E)) < 2e-15, two_j


def test_delta_planes_vs_jacobi_to_l16():
    for l in (0, 1, 2, 5, 9, 16):
        assert np.max(np.abs(oracle.delta_plane(l) - delta_exact(l))) < 1e-14, l


@pytest.mark.parametrize("l", [1, 7, 64, 300])
def test_delta_orthogonal(l):
    D = oracle.delta_plane(l)
    assert np.max(np.abs(D.T @ D - np.eye(2 * l + 1))) < 1e-13 * max(1, l / 16)


@pytest.mark.parametrize("l", [3, 10, 41])
def test_symmetries(l):
    b = 0.77
    D = oracle.wigner_plane(2 * l, b)
    Dpi = oracle.wigner_plane(2 * l, np.pi - b)
    Dneg = oracle.wigner_plane(2 * l, -b)
    m = np.arange(-l, l + 1)
    sgn = (-1.0) ** ((m[:, None] - m[None, :]) % 2)
    # Eq. (wignerd_sym1): d_mn = (-1)^(m-n) d_{-m,-n}
    assert np.allclose(D, sgn * D[::-1, ::-1], atol=1e-14)
    # Eq. (wignerd_sym2): d_mn(pi - b) = (-1)^(l-n) d_{-m,n}(b)
    assert np.allclose(Dpi, ((-1.0) ** ((l - m) % 2))[None, :] * D[::-1, :], atol=1e-13)
    # Eq. (wignerd_sym3): d_mn(-b) = (-1)^(m-n) d_mn(b)
    assert np.allclose(Dneg, sgn * D, atol=1e-14)
    # transpose: d_mn = (-1)^(m-n) d_nm (from sym3 and d(-b) = d(b)^T)
    assert np.allclose(D, sgn * D.T, atol=1e-14)


@pytest.mark.parametrize("l", [2, 6, 25])
def test_fourier_relation(l):
    # Eq. (wigner_sum_reln): d_mn(b) = i^(n-m) sum_m' Delta_{m'm} Delta_{m'n} e^{i m' b}
    b = 1.234
    Dl = oracle.delta_plane(l)
    m = np.arange(-l, l + 1)
    ex = np.exp(1j * m * b)
    lhs = oracle.wigner_plane(2 * l, b)
    rhs = (1j ** ((m[None, :] - m[:, None]) % 4)) * np.einsum("pm,pn,p->mn", Dl, Dl, ex)
    assert np.max(np.abs(rhs.imag)) < 1e-13
    assert np.max(np.abs(lhs - rhs.real)) < 1e-13
    if l <= 6:
        for mm in range(-l, l + 1, 3):
            for nn in range(-l, l + 1, 2):
                assert abs(lhs[mm + l, nn + l] - float(d_jacobi(2 * l, 2 * mm, 2 * nn, mp.mpf(b)))) < 1e-14


def test_explicit_sum_equals_jacobi_form():
    # the explicit Wigner sum used by the brute-force synthesis agrees with the
    # paper's Jacobi form (Eq. wignerd_b) away from beta in {0, pi}
    for two_j in range(0, 13):
        for two_m in range(-two_j, two_j + 1, 2):
            for two_n in range(-two_j, two_j + 1, 2):
                for b in (0.4, 2.0):
                    assert abs(d_sum(two_j, two_m, two_n, b) - d_jacobi(two_j, two_m, two_n, b)) < 1e-28
