"""Explicit (non-recursive) formulas used to pin the oracle.

Independent of the oracle's Risbo recursion: Wigner d-functions from the
Jacobi-polynomial form printed in the paper (Eq. wignerd_b, Sec. III-C),
evaluated in mpmath at 30+ digits; spin spherical harmonics from Eq.
(ssh_wigner) and Eq. (d_decomp); and the textbook scalar harmonics with the
Condon-Shortley phase (Sec. III-A).
"""
from functools import lru_cache

import mpmath as mp
import numpy as np

mp.mp.dps = 34


def gbinom(r, k):
    """Generalised binomial coefficient r(r-1)...(r-k+1)/k! (any integer r, k >= 0)."""
    if k < 0:
        return mp.mpf(0)
    num = mp.mpf(1)
    for i in range(k):
        num *= (r - i)
    return num / mp.factorial(k)


def jacobi_poly(deg, a, b, x):
    """Jacobi polynomial P_deg^(a,b)(x) by its finite sum
    sum_s C(deg+a, deg-s) C(deg+b, s) ((x-1)/2)^s ((x+1)/2)^(deg-s),
    a polynomial identity that holds for negative integer a, b as well."""
    x = mp.mpf(x)
    return mp.fsum(gbinom(deg + a, deg - s) * gbinom(deg + b, s) * ((x - 1) / 2) ** s *
                   ((x + 1) / 2) ** (deg - s) for s in range(deg + 1))


def d_jacobi(two_j, two_m, two_n, beta):
    """d^j_{mn}(beta) by Eq. (wignerd_b); arguments in twice-units so that
    half-integer j are allowed."""
    j, m, n = mp.mpf(two_j) / 2, mp.mpf(two_m) / 2, mp.mpf(two_n) / 2
    beta = mp.mpf(beta)
    pref = mp.sqrt(mp.factorial(j + n) * mp.factorial(j - n) / (mp.factorial(j + m) * mp.factorial(j - m)))
    # j-n, n-m and n+m are integers even for half-integer j
    deg, a, b = (two_j - two_n) // 2, (two_n - two_m) // 2, (two_n + two_m) // 2
    return pref * mp.sin(beta / 2) ** a * mp.cos(beta / 2) ** b * jacobi_poly(deg, a, b, mp.cos(beta))


def d_sum(two_j, two_m, two_n, beta):
    """d^j_{mn}(beta) by Wigner's explicit finite sum (all exponents are
    non-negative, so it is exact at beta = 0 and pi too):
      sum_k (-1)^(k-n+m) sqrt((j+m)!(j-m)!(j+n)!(j-n)!)
            / ((j+n-k)! k! (j-m-k)! (k-n+m)!) cos(b/2)^(2j-2k+n-m) sin(b/2)^(2k-n+m)."""
    jpm, jmm = (two_j + two_m) // 2, (two_j - two_m) // 2
    jpn, jmn = (two_j + two_n) // 2, (two_j - two_n) // 2
    nm = (two_n - two_m) // 2
    beta = mp.mpf(beta)
    c, s = mp.cos(beta / 2), mp.sin(beta / 2)
    pref = mp.sqrt(mp.factorial(jpm) * mp.factorial(jmm) * mp.factorial(jpn) * mp.factorial(jmn))
    tot = mp.mpf(0)
    for k in range(0, two_j + 1):
        a1, a2, a3 = jpn - k, jmm - k, k - nm
        if a1 < 0 or a2 < 0 or a3 < 0:
            continue
        den = mp.factorial(a1) * mp.factorial(k) * mp.factorial(a2) * mp.factorial(a3)
        tot += (-1) ** ((k - nm) % 2) * pref / den * c ** (two_j - 2 * k + nm) * s ** (2 * k - nm)
    return tot


@lru_cache(maxsize=None)
def d_int(l, m, n, beta_key):
    return float(d_jacobi(2 * l, 2 * m, 2 * n, mp.mpf(beta_key)))


def delta_exact(l):
    """Delta^l = d^l(pi/2) as a float64 (2l+1)^2 array (row m+l, column n+l)."""
    P = 2 * l + 1
    out = np.empty((P, P))
    half_pi = mp.pi / 2
    for i in range(P):
        for k in range(P):
            out[i, k] = float(d_jacobi(2 * l, 2 * (i - l), 2 * (k - l), half_pi))
    return out


def spin_sh(l, m, s, theta, phi):
    """sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/4pi) D^{l*}_{m,-s}(phi, theta, 0)
    (Eq. ssh_wigner) with D_{mn}(a,b,c) = e^{-ima} d_{mn}(b) e^{-inc}
    (Eq. d_decomp), i.e. (-1)^s sqrt((2l+1)/4pi) e^{i m phi} d^l_{m,-s}(theta)."""
    d = float(d_sum(2 * l, 2 * m, -2 * s, mp.mpf(theta)))
    return (-1) ** s * np.sqrt((2 * l + 1) / (4 * np.pi)) * np.exp(1j * m * phi) * d


def scalar_sh_textbook(l, m, theta, phi):
    """Scalar Y_lm for l <= 2 with the Condon-Shortley phase (Sec. III-A)."""
    c, s = np.cos(theta), np.sin(theta)
    e = np.exp(1j * m * phi)
    table = {
        (0, 0): 1 / np.sqrt(4 * np.pi),
        (1, 0): np.sqrt(3 / (4 * np.pi)) * c,
        (1, 1): -np.sqrt(3 / (8 * np.pi)) * s,
        (1, -1): np.sqrt(3 / (8 * np.pi)) * s,
        (2, 0): np.sqrt(5 / (16 * np.pi)) * (3 * c * c - 1),
        (2, 1): -np.sqrt(15 / (8 * np.pi)) * s * c,
        (2, -1): np.sqrt(15 / (8 * np.pi)) * s * c,
        (2, 2): np.sqrt(15 / (32 * np.pi)) * s * s,
        (2, -2): np.sqrt(15 / (32 * np.pi)) * s * s,
    }
    return table[(l, m)] * e


def brute_force_inverse(flm, L, s):
    """f(theta_t, phi_p) = sum_lm f_lm sY_lm(theta_t, phi_p) on the MW grid,
    pole stored as f(pi, 0): the definition of the inverse (Sec. III-B)."""
    M = 2 * L - 1
    th = np.pi * (2 * np.arange(L) + 1) / M
    ph = 2 * np.pi * np.arange(M) / M
    rings = np.zeros((L, M), dtype=np.complex128)
    for l in range(abs(s), L):
        for m in range(-l, l + 1):
            c = flm[l * l + l + m]
            if c == 0:
                continue
            for t in range(L):
                d = float(d_sum(2 * l, 2 * m, -2 * s, mp.pi * (2 * t + 1) / M))
                rings[t] += c * (-1) ** s * np.sqrt((2 * l + 1) / (4 * np.pi)) * d * np.exp(1j * m * ph)
    out = np.empty((L - 1) * M + 1, dtype=np.complex128)
    out[: (L - 1) * M] = rings[: L - 1].ravel()
    out[(L - 1) * M] = rings[L - 1, 0]
    return out


def delta_half_pi_exact(l, m, n):
    """d^l_{mn}(pi/2) for integer l from Wigner's explicit sum (d_sum) at
    cos = sin = 1/sqrt2: with the terms regrouped into binomials,
      d^l_{mn}(pi/2) = 2^-l sqrt((l+m)!(l-m)! / ((l+n)!(l-n)!))
                       * sum_k (-1)^(k-n+m) C(l+n, k) C(l-n, k-n+m),
    whose sum is an exact integer; only the final square root of an exact
    rational is rounded (40 digits)."""
    from math import comb, factorial
    T = 0
    for k in range(0, l + n + 1):
        j = k - n + m
        if 0 <= j <= l - n:
            T += (-1) ** (j % 2) * comb(l + n, k) * comb(l - n, j)
    if T == 0:
        return mp.mpf(0)
    num = T * T * factorial(l + m) * factorial(l - m)
    den = factorial(l + n) * factorial(l - n) * 4 ** l
    with mp.workdps(40):
        v = mp.sqrt(mp.mpf(num) / mp.mpf(den))
    return v if T > 0 else -v
