"""FP64 CPU oracle for the MW spin spherical harmonic transforms
(McEwen & Wiaux, "A novel sampling theorem on the sphere", IEEE TSP 2011).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or run anything in
this package.  The CUDA library and its Python binding never import it, and the
two share no code: the only thing both sides consume is the seeded input
generator, which lives in a module of its own and holds none of the method's
arithmetic.

Parity status: every function here is pinned by a test against something other
than itself (closed forms, Wigner's explicit d sum, brute-force synthesis with
spin spherical harmonics, exact round trips, numerical quadrature, dense
adjoints); see tests/test_oracle_*.py.
"""
from .mw_oracle import *  # noqa: F401,F403
