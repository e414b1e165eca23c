"""Pins of the oracle's adjoints: the stage-wise adjoints against the dense
conjugate transpose of the oracle's own forward/inverse (built column by
column from unit vectors), and dot-product tests at larger L."""
import numpy as np
import pytest

import oracle
from paper_1110_6298_gb300 import workloads as wl


def dense(op, n_in, dtype=np.complex128):
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, dtype=dtype)
        e[k] = 1
        cols.append(op(e))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("L,s", [(1, 0), (2, 1), (3, 0), (4, -2), (5, 1)])
def test_adjoints_equal_dense_conjugate_transpose(L, s):
    nmap, nlm = oracle.sample_count(L), L * L
    A = dense(lambda x: oracle.forward(x, L, s), nmap)          # [nlm, nmap]
    Ainv = dense(lambda f: oracle.inverse(f, L, s), nlm)        # [nmap, nlm]
    g = np.random.default_rng(L)
    y = g.standard_normal(nlm) + 1j * g.standard_normal(nlm)
    x = g.standard_normal(nmap) + 1j * g.standard_normal(nmap)
    assert np.max(np.abs(oracle.forward_adjoint(y, L, s) - A.conj().T @ y)) < 1e-12
    assert np.max(np.abs(oracle.inverse_adjoint(x, L, s) - Ainv.conj().T @ x)) < 1e-12


@pytest.mark.parametrize("L,s", [(16, 0), (33, 2), (64, -1)])
def test_dot_product(L, s):
    g = np.random.default_rng(L + abs(s))
    x = wl.gaussian_map(g, L)
    y = wl.gaussian_flm(g, L, s, wl.cl_white)
    lhs = np.vdot(y, oracle.forward(x, L, s))                  # <F x, y>
    rhs = np.vdot(oracle.forward_adjoint(y, L, s), x)          # <x, F^H y>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    f = wl.gaussian_flm(g, L, s, wl.cl_white)
    lhs = np.vdot(x, oracle.inverse(f, L, s))
    rhs = np.vdot(oracle.inverse_adjoint(x, L, s), f)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_round_trip_identity():
    # forward o inverse = I on band-limited f  =>  inverse^H o forward^H = I
    L, s = 20, 1
    y = wl.gaussian_flm(np.random.default_rng(1), L, s, wl.cl_white)
    back = oracle.inverse_adjoint(oracle.forward_adjoint(y, L, s), L, s)
    assert np.max(np.abs(back - y)) < 1e-12
