"""The split-BF16 contraction pipeline (kernels_tc2.cu) on the GPU: results
that do not depend on how many spin groups one pass of the pipeline carries
(MW_TC2_GROUPS=1 or 2; each group's sums run in the same order either way),
with a spin-group count that leaves a partial last pass, and agreement with
the FP64 oracle on every map."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def mw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6298_gb300 import build
    build.build()
    from paper_1110_6298_gb300 import mw as m
    m.lib()
    return m


def plan_with_groups(mw, n, *args, **kw):
    old = os.environ.get("MW_TC2_GROUPS")
    os.environ["MW_TC2_GROUPS"] = str(n)
    try:
        return mw.Plan(*args, **kw)
    finally:
        if old is None:
            del os.environ["MW_TC2_GROUPS"]
        else:
            os.environ["MW_TC2_GROUPS"] = old


@pytest.mark.parametrize("L", [37, 200, 530])
def test_groups_per_pass_bitwise_and_oracle(mw, L):
    # 9 maps of spin 0 (groups of 8 and 1), 7 of spin -2: three groups, so a
    # two-group pass leaves one group alone; L = 530 spans two plane chunks
    spins = [0] * 9 + [-2] * 7
    g = wl.rng(500 + L)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])).cuda()
    x = torch.from_numpy(np.stack([wl.gaussian_map(g, L) for _ in spins])).cuda()
    out = {}
    for n in (1, 2):
        p = plan_with_groups(mw, n, L, spins, precision="mixed")
        out[n] = (p.inverse(flm), p.forward(x))
        p.sync()
        p.close()
    assert torch.equal(out[1][0], out[2][0])
    assert torch.equal(out[1][1], out[2][1])
    maps, fwd = out[2][0].cpu().numpy(), out[2][1].cpu().numpy()
    for b in (0, 8, 9, 15):
        s = spins[b]
        ref = oracle.inverse(flm[b].cpu().numpy(), L, s)
        assert np.max(np.abs(maps[b] - ref)) / np.max(np.abs(ref)) < 1e-6
        ref = oracle.forward(x[b].cpu().numpy(), L, s)
        assert np.max(np.abs(fwd[b] - ref)) / np.max(np.abs(ref)) < 1e-6


@pytest.mark.parametrize("spins", [[1] * 16, [2] * 8 + [-2] * 8, [3] * 12], ids=["twin", "signs", "twin-ragged"])
def test_twin_and_shared_spin_row(mw, spins):
    # [1] * 16: two full groups of one spin, so a two-group pass forms A once
    # and multiplies it into both groups' B with one N = 64 MMA per product;
    # [2] * 8 + [-2] * 8: spins s and -s read one spin row but keep two A
    # tiles (the sign pattern differs); [3] * 12: a twin pass whose second
    # group holds 4 maps.  Every result must match the one-group-per-pass run
    # bit for bit and the oracle within the mixed path's 1e-6.
    L = 160
    g = wl.rng(900 + len(spins) + spins[-1])
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])).cuda()
    x = torch.from_numpy(np.stack([wl.gaussian_map(g, L) for _ in spins])).cuda()
    out = {}
    for n in (1, 2):
        p = plan_with_groups(mw, n, L, spins, precision="mixed")
        out[n] = (p.inverse(flm), p.forward(x))
        p.sync()
        p.close()
    assert torch.equal(out[1][0], out[2][0])
    assert torch.equal(out[1][1], out[2][1])
    maps, fwd = out[2][0].cpu().numpy(), out[2][1].cpu().numpy()
    for b in (0, 7, 8, len(spins) - 1):
        s = spins[b]
        ref = oracle.inverse(flm[b].cpu().numpy(), L, s)
        assert np.max(np.abs(maps[b] - ref)) / np.max(np.abs(ref)) < 1e-6
        ref = oracle.forward(x[b].cpu().numpy(), L, s)
        assert np.max(np.abs(fwd[b] - ref)) / np.max(np.abs(ref)) < 1e-6
