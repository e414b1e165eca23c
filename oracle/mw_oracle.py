"""Plain FP64 oracle of the MW transforms, step by step in the paper's order.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function follows a
passage of McEwen & Wiaux (2011), cited beside it, and uses the paper's notation:
L band limit, s spin, M = 2L-1, theta_t / phi_p the sampling nodes, G_m(theta_t),
F_mm', G_mm', f_lm.  FFTs (scipy.fft) and a matrix product stand in for the
library primitives; there is no blocking or fusion beyond what the equations say.
The O(L^3) Wigner stages run in C (mw_oracle.c) for speed only.

Array conventions (all complex128):
  map   : [N_MW]  rings t = 0..L-2 of M samples at phi_p, then the pole f(pi, 0)
  flm   : [L*L]   index l*l + l + m; entries with l < |s| are zero on output
  G_mt  : [L, M]  G_m(theta_t), axis 1 indexed by m + L - 1
  F, G  : [M, M]  F_mm' / G_mm', indexed [m + L - 1, m' + L - 1]
Batched variants take a leading batch axis; all maps of one call share s.
"""
import ctypes
import os

import numpy as np
import scipy.fft as sfft

from . import build as _build

_lib = None


def _c():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_wigner_plane.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        lib.orc_forward_wigner.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip,
                                           ctypes.c_int, dp]
        lib.orc_inverse_wigner.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_inverse_rings.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                          ctypes.c_int, dp, dp]
        for f in (lib.orc_wigner_plane, lib.orc_forward_wigner, lib.orc_inverse_wigner,
                  lib.orc_inverse_rings, lib.orc_num_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads():
    """Threads the C part uses (OpenMP)."""
    return int(_c().orc_num_threads())


# --------------------------------------------------------------------------
# Sampling (Sec. IV-C, Eqs. nodes_theta, nodes_phi)
# --------------------------------------------------------------------------

def sample_count(L):
    """N_MW = (L-1)(2L-1) + 1 (Sec. IV-C)."""
    return (L - 1) * (2 * L - 1) + 1


def theta_nodes(L, extended=False):
    """theta_t = pi (2t+1) / (2L-1), t = 0..L-1 (Eq. nodes_theta); with
    extended=True t runs over 0..2L-2, the periodic extension of Sec. IV-C."""
    n = 2 * L - 1 if extended else L
    t = np.arange(n)
    return np.pi * (2 * t + 1) / (2 * L - 1)


def phi_nodes(L):
    """phi_p = 2 pi p / (2L-1), p = 0..2L-2 (Eq. nodes_phi)."""
    return 2 * np.pi * np.arange(2 * L - 1) / (2 * L - 1)


def weight(k):
    """w(k) = int_0^pi sin(theta) e^{i k theta} dtheta, closed form of Sec. IV-D:
    +-i pi/2 at k = +-1, 0 for other odd k, 2/(1-k^2) for even k."""
    k = np.asarray(k)
    out = np.zeros(k.shape, dtype=np.complex128)
    even = (k % 2) == 0
    out[even] = 2.0 / (1.0 - k[even].astype(np.float64) ** 2)
    out[k == 1] = 1j * np.pi / 2
    out[k == -1] = -1j * np.pi / 2
    return out


# --------------------------------------------------------------------------
# Wigner planes (Sec. III-C; Risbo's recursion, Sec. V-B)
# --------------------------------------------------------------------------

def wigner_plane(two_j, beta=np.pi / 2):
    """d^j(beta) for j = two_j/2, full (2j+1)^2 plane, row m + j, column n + j."""
    P = two_j + 1
    out = np.empty((P, P), dtype=np.float64)
    if _c().orc_wigner_plane(int(two_j), float(beta), _dp(out)) != 0:
        raise MemoryError("orc_wigner_plane failed")
    return out


def delta_plane(l):
    """Delta^l = d^l(pi/2), rows m + l, columns n + l."""
    return wigner_plane(2 * l, np.pi / 2)


def delta_top_row(l):
    """Delta^l_{l,m}, m = 0..l, as (mantissa, exponent) pairs with value
    mantissa * 2^exponent: Delta^l_{l,m} = (-1)^(l-m) 2^-l sqrt(C(2l, l+m)),
    the closed form of d^l_{l,m}(beta) = sqrt(C(2l, l+m)) cos^(l+m)(beta/2)
    (-sin(beta/2))^(l-m) at beta = pi/2 (Sec. III-C conventions).  The
    binomial is an exact integer; the exponent keeps values far below the
    double range (2^-l at m = l) exact in range."""
    from math import comb, frexp, sqrt
    mant = np.empty(l + 1)
    expo = np.empty(l + 1, dtype=np.int64)
    for m in range(l + 1):
        c = comb(2 * l, l + m)
        e2 = c.bit_length() - 60
        e2 -= e2 % 2                          # even shift, so the root is exact in the exponent
        r = sqrt(c >> e2 if e2 > 0 else c << -e2)
        fm, fe = frexp(r)
        mant[m] = fm if (l - m) % 2 == 0 else -fm
        expo[m] = fe + e2 // 2 - l
    return mant, expo


def delta_plane_tn(l):
    """Quarter plane Delta^l_{m',m}, m', m = 0..l (rows m', columns m), by
    the Trapani-Navaza recursion (cited in Sec. V-B as the alternative to
    Risbo's): each column m starts from the top row Delta^l_{l,m} and recurses
    down the first index with the three-term relation of d^l at beta = pi/2,
      sqrt((l+m')(l-m'+1)) Delta_{m'-1,m}
        = 2 m Delta_{m',m} - sqrt((l-m')(l+m'+1)) Delta_{m'+1,m},
    stopping at m' = 0 (below it the recursion would run into the decaying
    region near m' = -l, where it is unstable).  Each column is carried as
    value = x * 2^E with one exponent E per column (rescaled whenever |x|
    exceeds 2^64), so start values far below the double range stay exact."""
    mant, expo = delta_top_row(l)
    m = np.arange(l + 1, dtype=np.float64)
    E = expo.copy()
    cur = mant.copy()
    prev = np.zeros(l + 1)
    out = np.zeros((l + 1, l + 1))
    out[l] = np.ldexp(cur, E)
    for mp in range(l, 0, -1):
        a = np.sqrt(float((l - mp) * (l + mp + 1)))
        b = np.sqrt(float((l + mp) * (l - mp + 1)))
        new = (2.0 * m * cur - a * prev) / b
        prev, cur = cur, new
        big = np.abs(cur) > 2.0 ** 64
        cur = np.where(big, cur * 2.0 ** -64, cur)
        prev = np.where(big, prev * 2.0 ** -64, prev)
        E = np.where(big, E + 64, E)
        out[mp - 1] = np.ldexp(cur, E)
    return out


# --------------------------------------------------------------------------
# Forward transform (Sec. IV-D), one step per function
# --------------------------------------------------------------------------

def _check(L, s):
    if L < 1 or abs(s) >= L:
        raise ValueError("need L >= 1 and |s| < L")


def pole_ring(f_pole, L, s):
    """The pole samples f(pi, phi_p) = f(pi, 0) e^{i s phi_p}: only m = s
    survives at theta = pi because d^l_{m,-s}(pi) vanishes for m != s
    (Eq. wignerd_sym2 at beta = 0), so one stored sample fixes the ring."""
    return f_pole * np.exp(1j * s * phi_nodes(L))


def map_to_rings(f_map, L, s):
    """[N_MW] map -> [L, M] samples f(theta_t, phi_p) with the pole ring expanded."""
    M = 2 * L - 1
    f_map = np.asarray(f_map, dtype=np.complex128)
    rings = np.empty((L, M), dtype=np.complex128)
    rings[: L - 1] = f_map[: (L - 1) * M].reshape(L - 1, M)
    rings[L - 1] = pole_ring(f_map[(L - 1) * M], L, s)
    return rings


def phi_dft(f_map, L, s):
    """G_m(theta_t) = 2pi/(2L-1) sum_p f(theta_t, phi_p) e^{-i m phi_p},
    t = 0..L-1 (Sec. IV-D, first display).  Returns G_mt [L, M]."""
    M = 2 * L - 1
    rings = map_to_rings(f_map, L, s)
    return (2 * np.pi / M) * sfft.fftshift(sfft.fft(rings, axis=1), axes=1)


def theta_extend(G_mt, L, s):
    """Periodic extension to t = 0..2L-2 (Sec. IV-D, second display):
    G~_m(theta_t) = G_m(theta_t) for t < L and (-1)^(m+s) G_m(theta_{2L-2-t})
    for t >= L.  Returns [M (t), M (m)]."""
    M = 2 * L - 1
    m = np.arange(-(L - 1), L)
    sign = np.where((m + s) % 2 == 0, 1.0, -1.0)
    ext = np.empty((M, M), dtype=np.complex128)
    ext[:L] = G_mt
    for t in range(L, M):
        ext[t] = sign * G_mt[2 * L - 2 - t]
    return ext


def theta_dft(G_ext, L):
    """F_mm' = 1/(2pi(2L-1)) sum_t G~_m(theta_t) e^{-i m' theta_t}, t over the
    2L-1 extended nodes (Sec. IV-D, third display).  With theta_t = 2pi t/M +
    pi/M the sum is a length-M DFT times the phase e^{-i m' pi / M}.
    Returns F [M (m), M (m')]."""
    M = 2 * L - 1
    mp = np.arange(-(L - 1), L)
    spec = sfft.fftshift(sfft.fft(G_ext, axis=0), axes=0)  # [m', m]
    spec = spec * np.exp(-1j * mp * np.pi / M)[:, None]
    return spec.T / (2 * np.pi * M)


def weight_matrix(L):
    """W[m'', m'] = w(m'' - m') for |m''|, |m'| <= L-1 (Eq. Gmm_convolution)."""
    m = np.arange(-(L - 1), L)
    return weight(m[:, None] - m[None, :])


def weight_convolution(F, L, rows=None):
    """G_mm' = 2 pi sum_m'' F_mm'' w(m'' - m'), |m'| <= L-1 (Eq. Gmm_convolution),
    evaluated as written with one matrix product.  rows: optional m indices
    (offset by L-1) to restrict to."""
    Fr = F if rows is None else F[rows]
    return 2 * np.pi * (Fr @ weight_matrix(L))


def weight_convolution_fft(F, L, N=None):
    """The same G_mm' by the paper's fast route (Sec. IV-D, after Eq.
    Gmm_convolution): zero-pad F_mm'' to |m''| <= 2L-2 (any length N >= 4L-3
    keeps the aliasing outside |m'| <= L-1), inverse-transform it and the
    reflected weights, multiply, and transform back."""
    if N is None:
        N = 4 * L - 3
    if N < 4 * L - 3:
        raise ValueError("N must be >= 4L-3")
    k = np.arange(N)
    kk = np.where(k <= N // 2, k, k - N)          # signed frequency of each slot
    wk = np.where(np.abs(kk) <= 2 * L - 2, weight(kk), 0)
    x = np.zeros(F.shape[:-1] + (N,), dtype=np.complex128)
    m = np.arange(-(L - 1), L)
    x[..., m % N] = F
    X = sfft.ifft(x, axis=-1) * N                  # F on the fine theta grid
    V = sfft.fft(wk)                               # inverse DFT of reflected weights
    Y = sfft.fft(X * V, axis=-1) / N               # = sum_m'' F_mm'' w(m''-m')
    return 2 * np.pi * Y[..., m % N]


def forward_wigner(G, L, s, m_list=None):
    """f_lm from G_mm' by Eq. (flm_wig).  G: [B, M, M] (or [M, M]).  m_list
    restricts the computed m (others are returned as NaN)."""
    _check(L, s)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    single = G.ndim == 2
    Gb = G[None] if single else G
    B = Gb.shape[0]
    out = np.zeros((B, L * L), dtype=np.complex128)
    if m_list is not None:
        out[:] = np.nan
        ml = np.ascontiguousarray(np.asarray(m_list, dtype=np.int32))
        mptr, nm = ml.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(ml)
    else:
        mptr, nm = None, 0
    rc = _c().orc_forward_wigner(L, s, B, _dp(Gb.view(np.float64)), mptr, nm,
                                 _dp(out.view(np.float64)))
    if rc != 0:
        raise RuntimeError("orc_forward_wigner failed")
    if m_list is not None:  # entries l < |s| of computed columns are zero
        for m in m_list:
            for l in range(abs(m), L):
                if l < abs(s):
                    out[:, l * l + l + m] = 0
    return out[0] if single else out


def forward(f_map, L, s, m_list=None, conv="direct"):
    """MW forward transform (Sec. IV-D): phi DFT, extension, theta DFT, weight
    convolution, Wigner stage.  f_map: [N_MW] or [B, N_MW].  With m_list only
    those m are evaluated (the extension, DFT and convolution of the other m are
    skipped because each m is independent until the Wigner stage)."""
    _check(L, s)
    f_map = np.asarray(f_map, dtype=np.complex128)
    single = f_map.ndim == 1
    fb = f_map[None] if single else f_map
    M = 2 * L - 1
    rows = None if m_list is None else np.asarray(m_list) + L - 1
    Gs = []
    for f in fb:
        G_mt = phi_dft(f, L, s)
        if rows is not None:
            keep = np.zeros(M, dtype=bool)
            keep[rows] = True
            G_mt = np.where(keep[None, :], G_mt, 0)
        F = theta_dft(theta_extend(G_mt, L, s), L)
        if conv == "direct":
            Gmm = np.zeros((M, M), dtype=np.complex128)
            if rows is None:
                Gmm = weight_convolution(F, L)
            else:
                Gmm[rows] = weight_convolution(F, L, rows)
        else:
            Gmm = weight_convolution_fft(F, L)
        Gs.append(Gmm)
    out = forward_wigner(np.stack(Gs), L, s, m_list)
    return out[0] if single else out


# --------------------------------------------------------------------------
# Inverse transform (Sec. IV-E)
# --------------------------------------------------------------------------

def inverse_wigner(flm, L, s):
    """F_mm' from f_lm by Eq. (Fmm), every (m, m') computed directly.
    flm: [B, L*L] or [L*L].  Returns [B, M, M] (or [M, M])."""
    _check(L, s)
    flm = np.ascontiguousarray(flm, dtype=np.complex128)
    single = flm.ndim == 1
    fb = flm[None] if single else flm
    B = fb.shape[0]
    M = 2 * L - 1
    F = np.empty((B, M, M), dtype=np.complex128)
    if _c().orc_inverse_wigner(L, s, B, _dp(fb.view(np.float64)), _dp(F.view(np.float64))) != 0:
        raise RuntimeError("orc_inverse_wigner failed")
    return F[0] if single else F


def theta_synthesis(F, L):
    """F_m(theta_t) = sum_m' F_mm' e^{i m' theta_t} (Eq. Fmt) on the extended
    nodes, keeping t = 0..L-1 (Sec. IV-E).  Returns F_mt [L, M]."""
    M = 2 * L - 1
    mp = np.arange(-(L - 1), L)
    x = F * np.exp(1j * mp * np.pi / M)[None, :]              # [m, m']
    vals = sfft.ifft(sfft.ifftshift(x, axes=1), axis=1) * M   # [m, t]
    return vals[:, :L].T


def phi_synthesis(F_mt, L):
    """f(theta_t, phi_p) = sum_m F_m(theta_t) e^{i m phi_p} (Eq. f_pfft); the
    rings t = 0..L-2 are kept whole and the pole ring only at phi = 0."""
    M = 2 * L - 1
    rings = sfft.ifft(sfft.ifftshift(F_mt, axes=1), axis=1) * M
    out = np.empty(sample_count(L), dtype=np.complex128)
    out[: (L - 1) * M] = rings[: L - 1].reshape(-1)
    out[(L - 1) * M] = rings[L - 1, 0]
    return out


def inverse(flm, L, s):
    """MW inverse transform (Sec. IV-E): Wigner stage, theta synthesis, phi
    synthesis.  flm: [L*L] or [B, L*L]."""
    _check(L, s)
    flm = np.asarray(flm, dtype=np.complex128)
    single = flm.ndim == 1
    Fb = inverse_wigner(flm[None] if single else flm, L, s)
    out = np.stack([phi_synthesis(theta_synthesis(F, L), L) for F in Fb])
    return out[0] if single else out


def inverse_rings(flm, L, s, t_list):
    """Inverse-transform samples on chosen rings only, for spot checks of large
    transforms: F_m(theta_t) = (-1)^s sum_l sqrt((2l+1)/4pi) d^l_{m,-s}(theta_t)
    f_lm with d^l_{m,-s}(theta) from the Delta planes by Eq. (wigner_sum_reln),
    then the phi synthesis of Eq. (f_pfft).  Returns [B, len(t_list), M]
    (ring t = L-1 is the pole: all M entries equal f(pi,0) e^{i s phi_p})."""
    _check(L, s)
    flm = np.ascontiguousarray(flm, dtype=np.complex128)
    single = flm.ndim == 1
    fb = flm[None] if single else flm
    B = fb.shape[0]
    M = 2 * L - 1
    th = np.ascontiguousarray(theta_nodes(L)[np.asarray(t_list)], dtype=np.float64)
    Fmt = np.empty((B, len(th), M), dtype=np.complex128)
    if _c().orc_inverse_rings(L, s, B, _dp(fb.view(np.float64)), len(th), _dp(th),
                              _dp(Fmt.view(np.float64))) != 0:
        raise RuntimeError("orc_inverse_rings failed")
    vals = sfft.ifft(sfft.ifftshift(Fmt, axes=2), axis=2) * M
    return vals[0] if single else vals


# --------------------------------------------------------------------------
# Adjoints (Hermitian transposes), stage by stage in reverse order
# --------------------------------------------------------------------------

def forward_wigner_adjoint(y, L, s):
    """(Eq. flm_wig)^H.  The conjugate transpose of f_lm = c_m N_l sum_m'
    Delta_{m'm} Delta_{m',-s} G_mm' with c_m = (-1)^s i^(m+s) is
    G_mm' = conj(c_m) sum_l N_l Delta_{m'm} Delta_{m',-s} y_lm, and
    conj(c_m) = (-1)^s i^-(m+s): exactly the map of Eq. (Fmm)."""
    return inverse_wigner(y, L, s)


def inverse_wigner_adjoint(X, L, s):
    """(Eq. Fmm)^H, which by the same argument is the map of Eq. (flm_wig)."""
    return forward_wigner(X, L, s)


def forward_adjoint(y, L, s):
    """forward^H: Wigner^H, convolution^H, theta-DFT^H, extension^H, phi-DFT^H."""
    _check(L, s)
    y = np.asarray(y, dtype=np.complex128)
    single = y.ndim == 1
    Gh = forward_wigner_adjoint(y[None] if single else y, L, s)
    M = 2 * L - 1
    W = weight_matrix(L)
    mp = np.arange(-(L - 1), L)
    m = mp
    phi = phi_nodes(L)
    th = theta_nodes(L, extended=True)
    sign = np.where((m + s) % 2 == 0, 1.0, -1.0)
    outs = []
    for G in Gh:
        Fh = 2 * np.pi * (G @ W.conj().T)                                    # conv^H
        E = np.exp(1j * np.outer(mp, th))                                     # [m', t]
        Gext = (Fh @ E).T / (2 * np.pi * M)                                   # [t, m]
        Gmt = Gext[:L].copy()                                                 # extension^H
        for t in range(0, L - 1):
            Gmt[t] += sign * Gext[2 * L - 2 - t]
        P = np.exp(1j * np.outer(m, phi))                                     # [m, p]
        rings = (2 * np.pi / M) * (Gmt @ P)                                   # [t, p]
        out = np.empty(sample_count(L), dtype=np.complex128)
        out[: (L - 1) * M] = rings[: L - 1].reshape(-1)
        out[(L - 1) * M] = np.sum(np.exp(-1j * s * phi) * rings[L - 1])
        outs.append(out)
    out = np.stack(outs)
    return out[0] if single else out


def inverse_adjoint(x, L, s):
    """inverse^H: phi-synthesis^H, theta-synthesis^H, Wigner^H."""
    _check(L, s)
    x = np.asarray(x, dtype=np.complex128)
    single = x.ndim == 1
    xb = x[None] if single else x
    M = 2 * L - 1
    m = np.arange(-(L - 1), L)
    phi = phi_nodes(L)
    th = theta_nodes(L)
    Fs = []
    for v in xb:
        Fmt = np.zeros((L, M), dtype=np.complex128)
        rings = v[: (L - 1) * M].reshape(L - 1, M)
        Fmt[: L - 1] = rings @ np.exp(-1j * np.outer(phi, m))                # [t, m]
        Fmt[L - 1] = v[(L - 1) * M]
        F = (np.exp(-1j * np.outer(th, m)).T @ Fmt).T                          # [m, m']
        Fs.append(F)
    out = inverse_wigner_adjoint(np.stack(Fs), L, s)
    return out[0] if single else out


# --------------------------------------------------------------------------
# Quadrature (Sec. IV-F, Eq. quadrature)
# --------------------------------------------------------------------------

def quadrature_sample_count(L):
    """L(L-1) + 1 samples: L-1 rings of L samples in phi and the pole (Sec. IV-F)."""
    return L * (L - 1) + 1


def quadrature_phi_nodes(L):
    """phi'_p = 2 pi p / L, p = 0..L-1 (Sec. IV-F)."""
    return 2 * np.pi * np.arange(L) / L


def quadrature_v(L):
    """v(theta_t) = 1/(2L-1) sum_{|m'| <= L-1} w(-m') e^{i m' theta_t} on the
    extended nodes t = 0..2L-2 (Sec. IV-F, second display).  Real by the
    symmetry of w; the real part is returned."""
    mp = np.arange(-(L - 1), L)
    th = theta_nodes(L, extended=True)
    v = (weight(-mp)[None, :] * np.exp(1j * np.outer(th, mp))).sum(axis=1) / (2 * L - 1)
    return v.real


def quadrature_weights(L, s=0):
    """q(theta_t), t = 0..L-1 (Sec. IV-F, first display):
    q_t = (2 pi / L) [ v(theta_t) + (1 - delta_{t,L-1}) (-1)^s v(theta_{2L-2-t}) ],
    reading the garbled Kronecker delta as delta_{t,L-1}."""
    v = quadrature_v(L)
    t = np.arange(L)
    sg = -1.0 if (s % 2) else 1.0
    fold = np.where(t == L - 1, 0.0, sg * v[2 * L - 2 - t])
    return 2 * np.pi / L * (v[:L] + fold)


def quadrature_integrate(f_q, L, s=0):
    """I = sum_{t,p} f(theta_t, phi'_p) q(theta_t) (Eq. quadrature) for maps in
    the quadrature layout: rings t = 0..L-2 of L samples at phi'_p, then one pole
    sample f(pi, 0); on the pole ring f(pi, phi) = f(pi, 0) e^{i s phi}, so its L
    samples sum to L f(pi, 0) for s = 0 and to 0 otherwise (|s| < L).
    f_q: [n] or [B, n] with n = L(L-1)+1.  Returns a complex scalar per map."""
    f_q = np.asarray(f_q, dtype=np.complex128)
    single = f_q.ndim == 1
    fb = f_q[None] if single else f_q
    q = quadrature_weights(L, s)
    rings = fb[:, : (L - 1) * L].reshape(fb.shape[0], L - 1, L)
    out = (rings.sum(axis=2) * q[None, : L - 1]).sum(axis=1)
    if s == 0:
        out = out + q[L - 1] * L * fb[:, (L - 1) * L]
    return out[0] if single else out


def quadrature_samples(flm, L, s):
    """Band-limited f on the quadrature grid: the rings on the MW phi nodes
    (inverse_rings, Eqs. Fmm, Fmt, f_pfft), their phi coefficients F_m(theta_t)
    (a length-(2L-1) DFT, exact for |m| <= L-1), then f(theta_t, phi'_p) =
    sum_m F_m(theta_t) e^{i m phi'_p} summed directly.  Returns the quadrature
    layout (L-1 rings, then the pole)."""
    flm = np.asarray(flm, dtype=np.complex128)
    M = 2 * L - 1
    rings_mw = inverse_rings(flm, L, s, np.arange(L))    # [L][M]: f(theta_t, phi_p)
    Fk = sfft.fft(rings_mw, axis=1) / M                 # [L][M]: F_m at index m mod M
    m = np.arange(-(L - 1), L)
    Fmt = Fk[:, m % M]
    ph = quadrature_phi_nodes(L)
    rings = Fmt @ np.exp(1j * np.outer(m, ph))           # [L][L]
    out = np.empty(quadrature_sample_count(L), dtype=np.complex128)
    out[: (L - 1) * L] = rings[: L - 1].ravel()
    out[(L - 1) * L] = rings[L - 1, 0]
    return out


# --------------------------------------------------------------------------
# Real spin-0 signals (Sec. IV-G)
# --------------------------------------------------------------------------

def _neg_m_sign(L):
    """(-1)^m of every packed index l*l + l + m."""
    m = np.concatenate([np.arange(-l, l + 1) for l in range(L)])
    return np.where(m % 2 == 0, 1.0, -1.0)


def _mirror_index(L):
    """Packed index of (l, -m) for every packed index of (l, m)."""
    return np.concatenate([l * l + l - np.arange(-l, l + 1) for l in range(L)])


def fill_negative_m(flm, L):
    """Complete coefficients known for m >= 0 with the reality condition of a
    real scalar signal (Sec. IV-G): f_{l,-m} = (-1)^m conj(f_lm)."""
    flm = np.array(flm, dtype=np.complex128)
    pos = np.concatenate([l * l + l + np.arange(0, l + 1) for l in range(L)])
    neg = _mirror_index(L)[pos]
    flm[..., neg] = _neg_m_sign(L)[pos] * np.conj(flm[..., pos])
    return flm


def hermitian_part(flm, L):
    """Coefficients of Re(f) for a scalar signal f with coefficients f_lm:
    conj(f) has coefficients (-1)^m conj(f_{l,-m}) (the relation behind the
    reality condition of Sec. IV-G), so Re(f) has
    (f_lm + (-1)^m conj(f_{l,-m})) / 2."""
    flm = np.asarray(flm, dtype=np.complex128)
    return 0.5 * (flm + _neg_m_sign(L) * np.conj(flm[..., _mirror_index(L)]))


def forward_real(f_map, L):
    """Forward transform of real scalar maps (Sec. IV-G): only m >= 0 is
    evaluated through the phi DFT, extension, theta DFT, convolution and Wigner
    stage (each m is independent until the end), and m < 0 follows from the
    reality condition.  f_map: real [N_MW] or [B, N_MW]."""
    f_map = np.asarray(f_map)
    if np.iscomplexobj(f_map):
        raise TypeError("forward_real takes real maps")
    half = forward(f_map.astype(np.complex128), L, 0, m_list=range(0, L))
    return fill_negative_m(half, L)


def inverse_real(flm, L):
    """Real part of the inverse transform of scalar coefficients (Sec. IV-G):
    the inverse of their Hermitian part.  For those F_{-m,-m'} = conj(F_mm'),
    so only the rows m >= 0 go through the theta synthesis (Eq. Fmt), and the
    phi synthesis (Eq. f_pfft) is the real inverse DFT of F_m(theta_t),
    m = 0..L-1.  flm: [L*L] or [B, L*L]; returns real maps."""
    _check(L, 0)
    flm = np.asarray(flm, dtype=np.complex128)
    single = flm.ndim == 1
    h = hermitian_part(flm[None] if single else flm, L)
    M = 2 * L - 1
    outs = []
    for F in inverse_wigner(h, L, 0):
        F_mt = theta_synthesis(F[L - 1:], L)             # [t, m >= 0]
        rings = sfft.irfft(F_mt, n=M, axis=1) * M        # F_0 + 2 Re sum_{m>0} F_m e^{i m phi_p}
        out = np.empty(sample_count(L), dtype=np.float64)
        out[: (L - 1) * M] = rings[: L - 1].reshape(-1)
        out[(L - 1) * M] = rings[L - 1, 0]
        outs.append(out)
    out = np.stack(outs)
    return out[0] if single else out


# --------------------------------------------------------------------------
# Error measures (relative max and relative RMS, plus the paper's max-abs)
# --------------------------------------------------------------------------

def rel_errors(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    d = np.abs(x - ref)
    return {
        "max_abs": float(d.max()) if d.size else 0.0,
        "rel_max": float(d.max() / max(np.abs(ref).max(), 1e-300)) if d.size else 0.0,
        "rel_rms": float(np.linalg.norm((x - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300)),
    }
