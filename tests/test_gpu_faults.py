"""Failure detection without faulting the GPU: a zero pivot assembled on
purpose, the library's bounded device waits made to expire on conditions
nothing satisfies, a non-finite medium.  Each returns its status code to the
host and leaves the context usable."""
import math
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def solver(dim, n):
    from paper_1705_09443_gb300 import LSSolver
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, dim, 3, 0.15, (0.8, 1.2), 60 + dim)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    return LSSolver(n, om, mt, b_pml=3 if dim == 3 else 6, b_slab=3), mt


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 6)])
def test_zero_pivot_returns_singular_and_context_recovers(dim, n):
    from paper_1705_09443_gb300 import GmresOptions, LssError
    s, mt = solver(dim, n)
    s.test_inject(1, a=1, b=0)
    with pytest.raises(LssError) as e:
        s.factor()
    assert e.value.code == -4
    s.set_medium(mt)       # re-assembles the subproblems
    s.factor()
    g = s.plane_wave_rhs(np.eye(dim)[:1])
    _, st = s.solve(g, GmresOptions(30, 1e-8, 100))
    assert st[0]["converged"] and st[0]["relres_true"] <= 1e-8


def test_bounded_waits_expire_with_timeout_and_context_recovers():
    from paper_1705_09443_gb300 import GmresOptions, LssError
    s, mt = solver(2, 16)
    t0 = time.time()
    with pytest.raises(LssError) as e:
        s.test_inject(2)
    assert e.value.code == -6
    assert time.time() - t0 < 30           # two expiring waits of about 2 s each, a third that does not wait
    g = s.plane_wave_rhs(np.eye(2)[:1])
    _, st = s.solve(g, GmresOptions(30, 1e-8, 100))
    assert st[0]["converged"]


def test_non_finite_medium_is_rejected():
    from paper_1705_09443_gb300 import LssError
    s, mt = solver(2, 16)
    bad = mt.clone()
    bad[3, 4] = float("nan")
    with pytest.raises(LssError) as e:
        s.set_medium(bad)
    assert e.value.code == -1
