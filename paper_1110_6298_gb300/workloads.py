"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out in the library's
buffer order (f_lm at index l*l + l + m; maps as (L-1) rings of 2L-1 samples
plus one pole sample).  It contains none of the transforms' arithmetic and is
the one module that both the CUDA path's tests/benchmarks and the oracle
consume.

Seeds: numpy.random.Generator(PCG64(11106298 + k)) for workload k, with f_lm
drawn in index order.  The paper's own accuracy protocol draws real and
imaginary parts uniformly in [-1, 1] (Sec. V-D); the other workloads draw
complex Gaussian coefficients with E|f_lm|^2 = C_l (real and imaginary parts
i.i.d. N(0, C_l / 2)), zero for l < |s| where spin-s harmonics do not exist.
"""
import numpy as np

SEED_BASE = 11106298


def rng(k: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(k)))


def flm_size(L: int) -> int:
    return L * L


def map_size(L: int) -> int:
    return (L - 1) * (2 * L - 1) + 1


def ell_of_index(L: int) -> np.ndarray:
    """l of every packed index l*l + l + m."""
    return np.repeat(np.arange(L), 2 * np.arange(L) + 1)


def gaussian_flm(g: np.random.Generator, L: int, s: int, cl) -> np.ndarray:
    """Complex Gaussian f_lm with E|f_lm|^2 = cl(l); zero for l < |s|."""
    ell = ell_of_index(L)
    var = np.asarray(cl(ell.astype(np.float64)), dtype=np.float64)
    var = np.where(ell < abs(s), 0.0, var)
    re = g.standard_normal(L * L)
    im = g.standard_normal(L * L)
    return (re + 1j * im) * np.sqrt(var / 2.0)


def uniform_flm(g: np.random.Generator, L: int, s: int) -> np.ndarray:
    """Re, Im uniform on [-1, 1] (the paper's accuracy protocol); zero for l < |s|."""
    ell = ell_of_index(L)
    x = g.uniform(-1, 1, L * L) + 1j * g.uniform(-1, 1, L * L)
    return np.where(ell < abs(s), 0, x)


def uniform_flm_real(g: np.random.Generator, L: int) -> np.ndarray:
    """Coefficients of a real scalar signal: one complex draw per packed index
    (Re, Im uniform on [-1, 1], as uniform_flm), then the m = 0 entries keep
    their real part and each entry m < 0 is laid out as (-1)^m times the
    conjugate of the entry at +m, the structure the reality condition of
    Sec. IV-G fixes."""
    x = g.uniform(-1, 1, L * L) + 1j * g.uniform(-1, 1, L * L)
    ell = ell_of_index(L)
    m = np.arange(L * L) - ell * ell - ell
    mirror = ell * ell + ell - m
    sign = np.where(m % 2 == 0, 1.0, -1.0)
    out = np.where(m > 0, x, np.where(m == 0, x.real + 0j, sign * np.conj(x[mirror])))
    return out


def gaussian_real_map(g: np.random.Generator, L: int) -> np.ndarray:
    """I.i.d. real N(0, 1) samples on every grid point."""
    return g.standard_normal(map_size(L))


def gaussian_map(g: np.random.Generator, L: int) -> np.ndarray:
    """I.i.d. complex N(0, 1) samples (Re, Im ~ N(0, 1/2)) on every grid point."""
    n = map_size(L)
    return (g.standard_normal(n) + 1j * g.standard_normal(n)) * np.sqrt(0.5)


# ---- the five workloads ---------------------------------------------------

def cl_white(ell):
    return np.ones_like(ell)


def cl_config2(ell):
    return 1.0 / ((ell + 1.0) * (ell + 2.0))


def cl_red(ell):
    return 1.0 / (ell + 1.0) ** 2


def workload_small():
    """L=32, s=0, one map, Re/Im ~ N(0, 1/2) for all l < 32."""
    g = rng(1)
    return dict(L=32, spins=[0], flm=[gaussian_flm(g, 32, 0, cl_white)])


def workload_l256_s2():
    """L=256, s=2, one map, E|f_lm|^2 = 1/((l+1)(l+2)) for 2 <= l < 256."""
    g = rng(2)
    return dict(L=256, spins=[2], flm=[gaussian_flm(g, 256, 2, cl_config2)])


def workload_ragged(n_maps: int = 64):
    """64 maps with L_b uniform on {64,128,256,384,512} and s_b uniform on
    {0,+1,-1,+2,-2}; E|f_lm|^2 = 1/(l+1)^2, zero for l < |s_b|."""
    g = rng(3)
    Ls = g.choice([64, 128, 256, 384, 512], size=n_maps)
    ss = g.choice([0, 1, -1, 2, -2], size=n_maps)
    flm = [gaussian_flm(g, int(L), int(s), cl_red) for L, s in zip(Ls, ss)]
    return dict(Ls=[int(x) for x in Ls], spins=[int(x) for x in ss], flm=flm)


def workload_l2048_b16(n_maps: int = 16, L: int = 2048, seed: int = 4):
    """L=2048, B=16: maps 0..7 spin 0 and maps 8..15 spin 2, E|f_lm|^2 = 1/(l+1)^2.
    Another seed gives an independent batch of the same shape."""
    g = rng(seed)
    spins = [0] * (n_maps // 2) + [2] * (n_maps - n_maps // 2)
    flm = [gaussian_flm(g, L, s, cl_red) for s in spins]
    return dict(L=L, spins=spins, flm=flm)


def workload_grad_l512_b32(n_maps: int = 32, L: int = 512):
    """L=512, B=32 spin-0 maps of i.i.d. N(0,1) samples and Gaussian targets."""
    g = rng(5)
    maps = [gaussian_map(g, L) for _ in range(n_maps)]
    targets = [gaussian_flm(g, L, 0, cl_white) for _ in range(n_maps)]
    return dict(L=L, spins=[0] * n_maps, maps=maps, targets=targets)
