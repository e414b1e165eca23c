"""mw_inverse_noalloc, the allocation-free inverse transform, against mw_inverse.

The entry point serves callers that cannot allocate device memory (code inside
a custom allocator's callbacks, hosts that forbid allocation after start-up,
processes whose free device memory belongs to another pool): all of its
intermediates live in one static device array, so it takes no plan.  Here it
runs through the C ABI twice in a row on different inputs -- the second call
finds the first call's leftovers in the shared array -- and each result must
match the plan-based FP64 mw_inverse on the same input to the FP64 parity
tolerance, 1e-12 relative max error.  The file sorts last so that a run that
stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1110_6298_gb300 import workloads as wl  # noqa: E402

TOL = 1e-12
CASES = [(1, 0), (2, -1), (7, 3), (33, 0), (64, 2), (100, -5), (128, 1), (128, 127)]


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
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def flm_of(L, s, seed):
    return torch.from_numpy(wl.gaussian_flm(wl.rng(7000 + seed), L, s, wl.cl_white)).cuda()


@pytest.mark.parametrize("L,s", CASES)
def test_two_calls_in_a_row_match_plan_inverse(mw, L, s):
    x1, x2 = flm_of(L, s, 2 * L), flm_of(L, s, 2 * L + 1)
    ref = mw.Plan(L, s, precision="fp64")
    r1, r2 = ref.inverse(x1).reshape(-1), ref.inverse(x2).reshape(-1)
    torch.cuda.synchronize()
    n = mw.map_size(L)
    y1 = torch.full((n,), float("nan"), dtype=torch.complex128, device="cuda")
    y2 = torch.full((n,), float("nan"), dtype=torch.complex128, device="cuda")
    mw.inverse_noalloc(L, s, x1, y1)
    mw.inverse_noalloc(L, s, x2, y2)
    torch.cuda.synchronize()
    e1 = relmax(y1.cpu().numpy(), r1.cpu().numpy())
    e2 = relmax(y2.cpu().numpy(), r2.cpu().numpy())
    assert e1 < TOL and e2 < TOL, (e1, e2)


def test_rejects_sizes_beyond_the_maximum(mw):
    L = mw.NOALLOC_MAX_L + 1
    x = torch.zeros(mw.flm_size(L), dtype=torch.complex128, device="cuda")
    y = torch.zeros(mw.map_size(L), dtype=torch.complex128, device="cuda")
    with pytest.raises(mw.MWError) as ei:
        mw.inverse_noalloc(L, 0, x, y)
    assert ei.value.status == mw.MW_EINVAL


def test_rejects_host_buffers_and_bad_spin(mw):
    import ctypes
    L = 8
    xh = torch.zeros(mw.flm_size(L), dtype=torch.complex128)
    yh = torch.zeros(mw.map_size(L), dtype=torch.complex128)
    st = mw.lib().mw_inverse_noalloc(L, 0, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(yh.data_ptr()), None)
    assert st == mw.MW_EINVAL
    x = torch.zeros(mw.flm_size(L), dtype=torch.complex128, device="cuda")
    y = torch.zeros(mw.map_size(L), dtype=torch.complex128, device="cuda")
    with pytest.raises(mw.MWError):
        mw.inverse_noalloc(L, L, x, y)
