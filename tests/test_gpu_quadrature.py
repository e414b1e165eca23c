"""The MW quadrature rule (Sec. IV-F) on the GPU against the oracle: the weights
q(theta_t) for several band limits and both spin parities, batched integrals
of arbitrary maps in the quadrature layout (the rule is a definite weighted
sum), exactness on band-limited maps (sqrt(4 pi) f_00 for spin 0), bitwise
reproducibility and argument checks.  FP64 throughout: 1e-12 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def mw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6298_gb300 import build
    build.build()
    from paper_1110_6298_gb300 import mw as m
    m.lib()
    return m


@pytest.mark.parametrize("L", [1, 2, 5, 64, 257, 2048])
@pytest.mark.parametrize("s", [0, 1, -2])
def test_weights(mw, L, s):
    if abs(s) >= L:
        pytest.skip("|s| >= L")
    got = mw.quadrature_weights(L, s).cpu().numpy()
    ref = oracle.quadrature_weights(L, s)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < TOL


@pytest.mark.parametrize("L,spins", [(1, [0]), (3, [0, 1, -2]), (33, [0, 2, 0, -1]), (200, [1, 0])])
def test_integrals_of_arbitrary_maps(mw, L, spins):
    g = wl.rng(4000 + L)
    n = mw.quadrature_size(L)
    maps = np.stack([g.normal(size=n) + 1j * g.normal(size=n) for _ in spins])
    plan = mw.Plan(L, spins, precision="fp64")
    got = plan.quadrature(torch.from_numpy(maps).cuda()).cpu().numpy()
    ref = np.array([oracle.quadrature_integrate(maps[b], L, s) for b, s in enumerate(spins)])
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < TOL
    again = plan.quadrature(torch.from_numpy(maps).cuda()).cpu().numpy()
    assert np.array_equal(got, again)


def test_exact_on_band_limited_maps(mw):
    L = 24
    g = wl.rng(41)
    flm = wl.gaussian_flm(g, L, 0, wl.cl_white)
    fq = oracle.quadrature_samples(flm, L, 0)
    plan = mw.Plan(L, 0, precision="mixed")
    got = plan.quadrature(torch.from_numpy(fq).cuda()).cpu().numpy()[0]
    assert abs(got - np.sqrt(4 * np.pi) * flm[0]) < 1e-12 * np.max(np.abs(fq))


def test_rejects_bad_arguments(mw):
    with pytest.raises(mw.MWError):
        mw.quadrature_weights(4, 4)
    with pytest.raises(mw.MWError):
        mw.quadrature_weights(0, 0)
