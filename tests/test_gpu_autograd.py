"""Gradients through the hand-written adjoint kernels (torch.autograd.Function).

Workload: L = 512, 32 spin-0 maps of i.i.d. complex N(0,1) samples, seeded
Gaussian targets, loss = sum_b sum_lm |forward(map_b)_lm - target_lm|^2.  The
autograd gradient (forward^H applied to 2 x residual on the GPU) is checked
against (a) central finite differences in FP64 with step 1e-6 on 64 random
coordinates (real and imaginary parts perturbed separately; the loss
difference is summed term by term so that it is not lost to rounding) and (b)
the oracle's stage-wise adjoint on a subset of the maps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1110_6298_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6298_gb300 import build
    build.build()
    from paper_1110_6298_gb300 import autograd, mw
    mw.lib()
    return autograd, mw


def test_forward_gradient_l512_b32(ag):
    autograd, mw = ag
    w = wl.workload_grad_l512_b32()
    L, B = w["L"], len(w["maps"])
    maps = torch.from_numpy(np.stack(w["maps"])).cuda().requires_grad_(True)
    target = torch.from_numpy(np.stack(w["targets"])).cuda()
    plan = mw.Plan(L, [0] * B, precision="fp64")
    flm = autograd.mw_forward(maps, plan)
    loss = (flm - target).abs().pow(2).sum()
    loss.backward()
    grad = maps.grad.detach().cpu().numpy()
    resid = (flm - target).detach().cpu().numpy()

    # (b) oracle adjoint on four maps
    for b in (0, 7, 19, 31):
        ref = oracle.forward_adjoint(2 * resid[b], L, 0)
        assert np.max(np.abs(grad[b] - ref)) / np.max(np.abs(ref)) < 1e-12

    # (a) central finite differences, step 1e-6, one map at a time
    one = mw.Plan(L, [0], precision="fp64")
    g = np.random.default_rng(5)
    x0 = maps.detach()
    nmw = mw.map_size(L)
    h = 1e-6
    for _ in range(32):
        b = int(g.integers(B))
        k = int(g.integers(nmw))
        for part in (1.0, 1j):
            xp = x0[b:b + 1].clone()
            xm = x0[b:b + 1].clone()
            xp[0, k] += h * part
            xm[0, k] -= h * part
            rp = (one.forward(xp) - target[b:b + 1]).abs().pow(2)
            rm = (one.forward(xm) - target[b:b + 1]).abs().pow(2)
            fd = float((rp - rm).sum().item()) / (2 * h)
            an = grad[b, k].real if part == 1.0 else grad[b, k].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9 * np.max(np.abs(grad)), (b, k, part, fd, an)


def test_inverse_gradient(ag):
    autograd, mw = ag
    L, spins = 40, [2, -1]
    g = wl.rng(77)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_white) for s in spins])).cuda()
    flm.requires_grad_(True)
    tgt = torch.from_numpy(np.stack([wl.gaussian_map(g, L) for _ in spins])).cuda()
    plan = mw.Plan(L, spins, precision="fp64")
    out = autograd.mw_inverse(flm, plan)
    loss = (out - tgt).abs().pow(2).sum()
    loss.backward()
    resid = (out - tgt).detach().cpu().numpy()
    for b, s in enumerate(spins):
        ref = oracle.inverse_adjoint(2 * resid[b], L, s)
        got = flm.grad[b].cpu().numpy()
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12
