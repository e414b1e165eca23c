"""Pins of the oracle's forward and inverse transforms (Sec. IV) against the
definition of the inverse (brute-force synthesis with spin harmonics), textbook
scalar harmonics, the exact round trip forward(inverse(f)) = f, a hand-worked
L = 1 case, and the identities of Sec. IV-B and IV-G."""
import os

import numpy as np
import pytest

import oracle
from exact_wigner import brute_force_inverse, scalar_sh_textbook
from paper_1110_6298_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_flm(L, s, seed, cl=wl.cl_white):
    return wl.gaussian_flm(np.random.default_rng(abs(seed)), L, s, cl)


def test_l1_worked_case():
    vals = {}
    with open(os.path.join(GOLD, "l1_worked.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    L, s = 1, 0
    f = oracle.inverse(np.array([1.0 + 0j]), L, s)
    assert f.shape == (1,) and abs(f[0] - vals["map_value"]) < 1e-15
    G_mt = oracle.phi_dft(f, L, s)
    assert abs(G_mt[0, 0] - vals["G_0_theta0"]) < 1e-15
    F = oracle.theta_dft(oracle.theta_extend(G_mt, L, s), L)
    assert abs(F[0, 0] - vals["F_00"]) < 1e-15
    G = oracle.weight_convolution(F, L)
    assert abs(G[0, 0] - vals["G_00"]) < 1e-15
    assert abs(oracle.forward(f, L, s)[0] - vals["f_00"]) < 1e-15


@pytest.mark.parametrize("L,s", [(2, 0), (3, 1), (4, -2), (6, 3), (8, 0), (9, -1)])
def test_inverse_vs_brute_force_synthesis(L, s):
    flm = rand_flm(L, s, 10 * L + s)
    a = oracle.inverse(flm, L, s)
    b = brute_force_inverse(flm, L, s)
    assert np.max(np.abs(a - b)) < 1e-13 * max(1, np.max(np.abs(b)))


@pytest.mark.parametrize("l,m", [(0, 0), (1, -1), (1, 0), (1, 1), (2, -2), (2, -1), (2, 0), (2, 1), (2, 2)])
def test_scalar_closed_forms(l, m):
    L = 5
    flm = np.zeros(L * L, dtype=complex)
    flm[l * l + l + m] = 1
    f = oracle.inverse(flm, L, 0)
    M = 2 * L - 1
    th = oracle.theta_nodes(L)
    ph = oracle.phi_nodes(L)
    ref = np.array([scalar_sh_textbook(l, m, t, p) for t in th[:-1] for p in ph] +
                   [scalar_sh_textbook(l, m, th[-1], 0.0)])
    assert f.shape == (oracle.sample_count(L),) and len(ref) == (L - 1) * M + 1
    assert np.max(np.abs(f - ref)) < 1e-14


@pytest.mark.parametrize("L,s", [(1, 0), (2, 1), (3, 0), (4, -3), (8, 2), (17, 5), (32, 0), (64, -2),
                                 (128, 1), (256, 2)])
def test_round_trip_exact(L, s):
    # forward(inverse(f)) = f for band-limited f (Sec. IV-E closing remark); the
    # paper protocol draws Re/Im uniformly in [-1, 1] (Sec. V-D)
    flm = wl.uniform_flm(np.random.default_rng(L + 100 * abs(s) + 7), L, s)
    f = oracle.inverse(flm, L, s)
    back = oracle.forward(f, L, s)
    err = np.max(np.abs(back - flm))
    assert err < 1e-11, err
    ell = wl.ell_of_index(L)
    assert np.all(back[ell < abs(s)] == 0)


def test_round_trip_fft_convolution_route():
    L, s = 24, 1
    flm = rand_flm(L, s, 5)
    f = oracle.inverse(flm, L, s)
    assert np.max(np.abs(oracle.forward(f, L, s, conv="fft") - flm)) < 1e-12


def test_forward_is_a_projection_on_non_bandlimited_maps():
    # forward(inverse(forward(x))) = forward(x) for any map x
    L, s = 12, 2
    x = wl.gaussian_map(np.random.default_rng(3), L)
    a = oracle.forward(x, L, s)
    b = oracle.forward(oracle.inverse(a, L, s), L, s)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_forward_m_subset_matches_full():
    L, s = 20, -1
    x = wl.gaussian_map(np.random.default_rng(4), L)
    full = oracle.forward(x, L, s)
    ms = [-19, -4, 0, 3, 19]
    sub = oracle.forward(x, L, s, m_list=ms)
    ell = wl.ell_of_index(L)
    mm = np.arange(L * L) - ell * ell - ell
    sel = np.isin(mm, ms)
    assert np.max(np.abs(sub[sel] - full[sel])) < 1e-15 * np.max(np.abs(full))
    assert np.all(np.isnan(sub[~sel]))


def test_gmt_equals_2pi_fmt():
    # Eq. (Gmt_Fmt): G_m(theta) = 2 pi F_m(theta) for band-limited signals
    L, s = 10, 2
    flm = rand_flm(L, s, 8)
    f = oracle.inverse(flm, L, s)
    G_mt = oracle.phi_dft(f, L, s)
    F_mt = oracle.theta_synthesis(oracle.inverse_wigner(flm, L, s), L)
    assert np.max(np.abs(G_mt - 2 * np.pi * F_mt)) < 1e-13


def test_fmm_reflection_and_pole_continuity():
    L = 9
    m = np.arange(-(L - 1), L)
    for s in (0, 1, -2, 3):
        flm = rand_flm(L, s, 20 + s)
        F = oracle.inverse_wigner(flm, L, s)
        sign = ((-1.0) ** ((m + s) % 2))[:, None]
        # Eq. (Fmm_sym1): F_{m,-m'} = (-1)^(m+s) F_mm'
        assert np.max(np.abs(F[:, ::-1] - sign * F)) < 1e-14
        # footnote of Sec. IV-B: F_m(theta*) = 0 at the poles for m+s odd
        for th in (0.0, np.pi):
            Fm = F @ np.exp(1j * m * th)
            assert np.max(np.abs(Fm[(m + s) % 2 == 1])) < 1e-13


def test_pole_ring_representation():
    # the inverse on the pole ring is f(pi,0) e^{i s phi_p}; the pole sample is its p=0 value
    L = 7
    for s in (0, 2, -3):
        flm = rand_flm(L, s, 30 + s)
        ring = oracle.inverse_rings(flm, L, s, [L - 1])[0]
        f = oracle.inverse(flm, L, s)
        pole = f[-1]
        assert np.max(np.abs(ring - pole * np.exp(1j * s * oracle.phi_nodes(L)))) < 1e-13


def test_inverse_rings_match_inverse():
    L, s = 16, -2
    flm = rand_flm(L, s, 9)
    f = oracle.inverse(flm, L, s)
    M = 2 * L - 1
    ts = [0, 5, L - 2]
    rings = oracle.inverse_rings(flm, L, s, ts)
    for r, t in enumerate(ts):
        assert np.max(np.abs(rings[r] - f[t * M:(t + 1) * M])) < 1e-13


def test_spin_conjugate_symmetry():
    # Sec. III-B: sY*_lm = (-1)^(s+m) (-s)Y_{l,-m}, so conj(inverse(f, s)) is the
    # inverse of g, spin -s, with g_{l,-m} = (-1)^(s+m) conj(f_lm)
    L, s = 8, 3
    flm = rand_flm(L, s, 11)
    g = np.zeros_like(flm)
    for l in range(L):
        for m in range(-l, l + 1):
            g[l * l + l - m] = (-1) ** ((s + m) % 2) * np.conj(flm[l * l + l + m])
    a = np.conj(oracle.inverse(flm, L, s))
    b = oracle.inverse(g, L, -s)
    assert np.max(np.abs(a - b)) < 1e-13


def test_real_signal_symmetry():
    # Sec. IV-G: for real spin-0 signals F_{-m,-m'} = conj(F_mm') and the map is real
    L = 10
    flm = rand_flm(L, 0, 12)
    for l in range(L):
        for m in range(1, l + 1):
            flm[l * l + l - m] = (-1) ** m * np.conj(flm[l * l + l + m])
        flm[l * l + l] = flm[l * l + l].real
    F = oracle.inverse_wigner(flm, L, 0)
    assert np.max(np.abs(F[::-1, ::-1] - np.conj(F))) < 1e-14
    assert np.max(np.abs(oracle.inverse(flm, L, 0).imag)) < 1e-13


def test_spins_give_equal_round_trip_error_scale():
    # Sec. V-D: the error is the same for different spins (to statistical noise)
    L = 64
    errs = []
    for s in (0, 2, 10):
        flm = wl.uniform_flm(np.random.default_rng(s), L, s)
        errs.append(np.max(np.abs(oracle.forward(oracle.inverse(flm, L, s), L, s) - flm)))
    assert max(errs) < 1e-12 and max(errs) / min(errs) < 20


def gmm_integral_err(L=6, s=1, seed=13):
    """Max error of the oracle's G_mm' against Eq. (Gmm) integrated numerically:
    G_mm' = int_0^pi G_m(theta) e^{-i m' theta} sin(theta) dtheta with the
    band-limited G_m(theta) = 2 pi sum_m'' F_mm'' e^{i m'' theta} (Eq. Gmt_Fmt)."""
    from scipy import integrate
    flm = rand_flm(L, s, seed)
    f = oracle.inverse(flm, L, s)
    F = oracle.theta_dft(oracle.theta_extend(oracle.phi_dft(f, L, s), L, s), L)
    G = oracle.weight_convolution(F, L)
    ms = np.arange(-(L - 1), L)
    err = 0.0
    for mi in (0, L - 1, 2 * L - 3):
        for mpi in range(2 * L - 1):
            def integrand(th, part):
                v = 2 * np.pi * np.sum(F[mi] * np.exp(1j * ms * th)) * np.exp(-1j * ms[mpi] * th) * np.sin(th)
                return v.real if part == 0 else v.imag
            re, _ = integrate.quad(integrand, 0, np.pi, args=(0,), epsabs=1e-13, limit=200)
            im, _ = integrate.quad(integrand, 0, np.pi, args=(1,), epsabs=1e-13, limit=200)
            err = max(err, abs(G[mi, mpi] - (re + 1j * im)))
    return err


def test_gmm_equals_integral_definition():
    # the theta DFT + weight convolution chain reproduces the integral Eq. (Gmm)
    assert gmm_integral_err() < 1e-10
