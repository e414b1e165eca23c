"""Mutation checks: plant a plausible mistake in the oracle (on the CPU, via
monkeypatch) and show that a pin catches it.  Each pin below is one of the
tests in test_oracle_*.py; here it must FAIL on the mutated oracle."""
import numpy as np
import pytest

import oracle
import oracle.mw_oracle as om
from paper_1110_6298_gb300 import workloads as wl


def round_trip_err(L=12, s=1):
    flm = wl.uniform_flm(np.random.default_rng(0), L, s)
    return np.max(np.abs(om.forward(om.inverse(flm, L, s), L, s) - flm))


def test_unmutated_passes():
    assert round_trip_err() < 1e-12


def test_weight_sign_flip_caught(monkeypatch):
    # The odd weights w(+-1) cancel exactly in f_lm (the extended G~_m is
    # reflection-symmetric about theta = pi, so their contribution is odd in m'
    # while Delta_{m'm} Delta_{m',-s} is even), so the round trip cannot see this
    # mutation; the integral pin of Eq. (Gmm) on G_mm' does.
    from test_oracle_transforms import gmm_integral_err
    good = om.weight
    assert gmm_integral_err() < 1e-10
    monkeypatch.setattr(om, "weight", lambda k: np.conj(good(k)))   # -i pi/2 at k = +1
    assert round_trip_err() < 1e-12
    assert gmm_integral_err() > 1e-3


def test_dropped_extension_sign_caught(monkeypatch):
    def bad_extend(G_mt, L, s):
        M = 2 * L - 1
        ext = np.empty((M, M), dtype=np.complex128)
        ext[:L] = G_mt
        for t in range(L, M):
            ext[t] = G_mt[2 * L - 2 - t]      # (-1)^(m+s) dropped
        return ext
    monkeypatch.setattr(om, "theta_extend", bad_extend)
    assert round_trip_err() > 1e-3


def test_dropped_half_sample_phase_caught(monkeypatch):
    def bad_theta_dft(G_ext, L):
        M = 2 * L - 1
        spec = om.sfft.fftshift(om.sfft.fft(G_ext, axis=0), axes=0)
        return spec.T / (2 * np.pi * M)       # e^{-i m' pi / M} dropped
    monkeypatch.setattr(om, "theta_dft", bad_theta_dft)
    assert round_trip_err() > 1e-3


def test_wrong_prefactor_caught(monkeypatch):
    good = om.forward_wigner

    def bad(G, L, s, m_list=None):              # i^(m+s) -> i^-(m+s)
        out = good(G, L, s, m_list)
        ell = wl.ell_of_index(L)
        m = np.arange(L * L) - ell * ell - ell
        return out * (1j ** ((-2 * (m + s)) % 4))
    monkeypatch.setattr(om, "forward_wigner", bad)
    assert round_trip_err() > 1e-3


def test_transposed_delta_caught():
    # using Delta_{m m'} in place of Delta_{m' m} breaks the Fourier relation pin
    l, b = 5, 1.234
    D = oracle.delta_plane(l)
    m = np.arange(-l, l + 1)
    ph = 1j ** ((m[None, :] - m[:, None]) % 4)
    good = (ph * np.einsum("pm,pn,p->mn", D, D, np.exp(1j * m * b))).real
    bad = (ph * np.einsum("mp,pn,p->mn", D, D, np.exp(1j * m * b))).real
    ref = oracle.wigner_plane(2 * l, b)
    assert np.max(np.abs(good - ref)) < 1e-13
    assert np.max(np.abs(bad - ref)) > 1e-3
