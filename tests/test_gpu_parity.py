"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (relative max error max|x - x_o| / max|x_o|): 1e-12 for the FP64
path and 1e-6 for both mixed paths (BF16x3 and TF32x3 contractions).  Sizes span several 64-wide tiles / chunks
with ragged tails (L = 65, 130, 200), the degenerate cases (L = 1, L = 2, |s| =
L-1), batches of mixed spin, host and device pointers, and the full
L = 2048 x 16 workload on sampled outputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402

TOL = {"fp64": 1e-12, "mixed": 1e-6, "mixed_tf32": 1e-6}


@pytest.fixture(scope="module")
def mw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6298_gb300 import build
    build.build()
    from paper_1110_6298_gb300 import mw as m
    m.lib()
    return m


def relmax(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rand_flm_batch(L, spins, seed, cl=wl.cl_white):
    g = wl.rng(1000 + seed)
    return np.stack([wl.gaussian_flm(g, L, s, cl) for s in spins])


def rand_map_batch(L, n, seed):
    g = wl.rng(2000 + seed)
    return np.stack([wl.gaussian_map(g, L) for _ in range(n)])


def oracle_by_spin(fn, x, L, spins):
    """Apply an oracle function map-by-spin-group (the oracle takes one spin per call)."""
    out = [None] * len(spins)
    for s in sorted(set(spins)):
        idx = [b for b, t in enumerate(spins) if t == s]
        r = fn(x[idx], L, s)
        for k, b in enumerate(idx):
            out[b] = r[k]
    return np.stack(out)


CASES = [(1, [0]), (2, [1, 0, -1]), (3, [0, 2]), (7, [-3]), (32, [0]), (65, [2, -1, 0]), (130, [1, 1, 0]),
         (200, [-2, 5])]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_tf32"])
@pytest.mark.parametrize("L,spins", CASES)
def test_inverse(mw, prec, L, spins):
    flm = rand_flm_batch(L, spins, L)
    plan = mw.Plan(L, spins, precision=prec)
    got = plan.inverse(torch.from_numpy(flm).cuda()).cpu().numpy()
    ref = oracle_by_spin(oracle.inverse, flm, L, spins)
    assert relmax(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_tf32"])
@pytest.mark.parametrize("L,spins", CASES)
def test_forward_non_bandlimited(mw, prec, L, spins):
    x = rand_map_batch(L, len(spins), L)
    plan = mw.Plan(L, spins, precision=prec)
    got = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle_by_spin(oracle.forward, x, L, spins)
    assert relmax(got, ref) < TOL[prec]
    ell = wl.ell_of_index(L)
    for b, s in enumerate(spins):
        assert np.all(got[b][ell < abs(s)] == 0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_tf32"])
@pytest.mark.parametrize("L,spins", [(2, [1]), (9, [0, -2]), (65, [3, 0]), (130, [-1])])
def test_adjoints(mw, prec, L, spins):
    plan = mw.Plan(L, spins, precision=prec)
    y = rand_flm_batch(L, spins, 7 * L)
    x = rand_map_batch(L, len(spins), 7 * L)
    got_fa = plan.forward_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    got_ia = plan.inverse_adjoint(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(got_fa, oracle_by_spin(oracle.forward_adjoint, y, L, spins)) < TOL[prec]
    assert relmax(got_ia, oracle_by_spin(oracle.inverse_adjoint, x, L, spins)) < TOL[prec]


def test_round_trip_l256_s2(mw):
    # L = 256, spin 2, E|f_lm|^2 = 1/((l+1)(l+2)) for l >= 2: FP64 inverse + forward vs the oracle
    w = wl.workload_l256_s2()
    L, s = w["L"], w["spins"][0]
    flm = np.stack(w["flm"])
    plan = mw.Plan(L, [s], precision="fp64")
    f = plan.inverse(torch.from_numpy(flm).cuda())
    back = plan.forward(f).cpu().numpy()
    ref_map = oracle.inverse(flm[0], L, s)
    assert relmax(f.cpu().numpy()[0], ref_map) < 1e-12
    assert relmax(back[0], oracle.forward(f.cpu().numpy()[0], L, s)) < 1e-12
    assert np.max(np.abs(back[0] - flm[0])) < 1e-11


def test_host_pointers_match_device(mw):
    L, spins = 40, [0, 2]
    flm = rand_flm_batch(L, spins, 3)
    plan = mw.Plan(L, spins, precision="fp64")
    dev = plan.inverse(torch.from_numpy(flm).cuda()).cpu()
    host = plan.inverse(torch.from_numpy(flm))
    assert torch.equal(dev, host)
    back_h = plan.forward(host)
    back_d = plan.forward(host.cuda()).cpu()
    assert torch.equal(back_h, back_d)


def test_bitwise_reproducible(mw):
    L, spins = 100, [1, 1, -2]
    x = torch.from_numpy(rand_map_batch(L, 3, 5)).cuda()
    for prec in ("fp64", "mixed"):
        plan = mw.Plan(L, spins, precision=prec)
        a = plan.forward(x).clone()
        b = plan.forward(x)
        assert torch.equal(a, b)


def test_batch_equals_single(mw):
    L, spins = 33, [0, 3, -1]
    flm = rand_flm_batch(L, spins, 9)
    batch = mw.Plan(L, spins).inverse(torch.from_numpy(flm).cuda()).cpu().numpy()
    for b, s in enumerate(spins):
        one = mw.Plan(L, [s]).inverse(torch.from_numpy(flm[b:b + 1]).cuda()).cpu().numpy()
        assert relmax(batch[b], one[0]) < 1e-15


def test_rejects_bad_arguments(mw):
    with pytest.raises(mw.MWError):
        mw.Plan(8, [8])
    with pytest.raises(mw.MWError):
        mw.Plan(0, [0])
    plan = mw.Plan(8, [0])
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(5, dtype=torch.complex128, device="cuda"))


# Sampled outputs of the full-size workload: 16 rings of the inverse (the
# first and last few, the pole, and the interior), 16 m-columns of the forward
# (|m| = 0, 1, 2, 3 and up to L-1 = 2047 on both signs).
FULL_RINGS = [0, 1, 2, 255, 511, 767, 1023, 1279, 1535, 1791, 2000, 2043, 2044, 2045, 2046, 2047]
FULL_MS = [-2047, -2046, -2045, -1500, -1000, -517, -3, -1, 0, 1, 2, 517, 1200, 1999, 2046, 2047]
_ORACLE_CACHE = {}


def _cached(key, fn):
    """Oracle references of the full-size workload, computed once per module
    (they do not depend on the GPU path's precision)."""
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = fn()
    return _ORACLE_CACHE[key]


def _full_size_maps(mw, flm, L, spins):
    """The forward's full-size input: the FP64-path inverse of the workload's
    coefficients (band-limited maps, the same for every precision tested)."""
    def make():
        p = mw.Plan(L, spins, precision="fp64")
        x = p.inverse(torch.from_numpy(flm).cuda()).cpu().numpy()
        p.close()
        return x
    return _cached(("maps64", L), make)


@pytest.mark.parametrize("prec", ["mixed", "mixed_tf32", "fp64"])
def test_full_size_l2048_b16_sampled(mw, prec):
    """The benchmarked workload (L = 2048, 16 maps: 8 of spin 0, 8 of spin 2),
    in the benchmark's launch configuration, checked on sampled outputs: the
    inverse on 16 rings including t = L-2 and the pole (oracle ring
    synthesis), the forward of the GPU map on 16 m columns including
    |m| = L-1 (oracle forward restricted to those m), and the round trip."""
    w = wl.workload_l2048_b16()
    L, spins = w["L"], w["spins"]
    flm = np.stack(w["flm"])
    plan = mw.Plan(L, spins, precision=prec)
    f_gpu = plan.inverse(torch.from_numpy(flm).cuda())
    back = plan.forward(f_gpu).cpu().numpy()
    f_np = f_gpu.cpu().numpy()
    del f_gpu
    x = _full_size_maps(mw, flm, L, spins)
    fx = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    M = 2 * L - 1
    ell = wl.ell_of_index(L)
    sel = np.isin(np.arange(L * L) - ell ** 2 - ell, FULL_MS)
    for s, idx in ((0, [0, 7]), (2, [8, 15])):
        ref_r = _cached(("rings", s), lambda: oracle.inverse_rings(flm[idx], L, s, FULL_RINGS))
        for k, b in enumerate(idx):
            got_r = np.stack([f_np[b][t * M:(t + 1) * M] for t in FULL_RINGS[:-1]])
            assert relmax(got_r, ref_r[k][:-1]) < TOL[prec]
            # the pole ring is f(pi, 0) e^{i s phi}: its one stored sample is the phi = 0 entry
            assert abs(f_np[b][(L - 1) * M] - ref_r[k][-1][0]) / np.max(np.abs(ref_r[k])) < TOL[prec]
        ref_f = _cached(("fwd", s), lambda: oracle.forward(x[idx], L, s, m_list=FULL_MS))
        for k, b in enumerate(idx):
            assert relmax(fx[b][sel], ref_f[k][sel]) < TOL[prec]
            # band-limited input: the round trip is the identity
            assert np.max(np.abs(back[b] - flm[b])) / np.max(np.abs(flm[b])) < (1e-11 if prec == "fp64" else 1e-6)
