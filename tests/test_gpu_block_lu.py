"""Block LU (Thomas) slab solves against the cyclic reduction and the oracle.

With at least 16 right-hand sides the sweep solves its 16-wide slabs by the
block LU factorization along x2 (bottom-up Schur complements T_k, stored as
T_k^{-1}, V_k = -T_k^{-1} B_k, Y_k = -T_k^{-1} C_k; a bottom-up and a top-down
sweep of dense 16 x NRB products); the 32-wide slabs and every solve with
fewer right-hand sides keep the block cyclic reduction (LSS_SLAB_SOLVE=cr
forces it everywhere).  Both are exact factorizations of the same slab
subproblems, so P agrees to rounding: 1e-11 in FP64 (subproblem condition
numbers up to ~1e4), and within 1e-5 in mixed precision; P matches the
oracle's Algorithm 2 to 1e-10; the FGMRES iteration counts are unchanged.
Cases: R = 16, 20 (a partial column group), 33 and 64 (32-column groups), one
and two fronts, ragged last slabs, the fronts meeting in slab 0.
"""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def make(n, b_pml, b_slab, fronts, precision, seed):
    from paper_1705_09443_gb300 import LSSolver
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 2, 4, 0.1, (0.8, 1.2), seed)
    s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=b_pml, b_slab=b_slab,
                 precision=precision, fronts=fronts)
    return s, m, om


def both(s, x, monkeypatch):
    xd = torch.tensor(x, dtype=torch.complex128, device="cuda")
    monkeypatch.setenv("LSS_SLAB_SOLVE", "cr")
    y_cr = s.apply_P(xd).cpu().numpy()
    monkeypatch.delenv("LSS_SLAB_SOLVE")
    y_lu = s.apply_P(xd).cpu().numpy()
    return y_lu, y_cr


@pytest.mark.parametrize("n,b_pml,b_slab,fronts,R", [(64, 12, 4, 2, 16), (64, 12, 4, 1, 20), (50, 8, 3, 2, 33),
                                                     (37, 6, 4, 1, 64), (9, 3, 3, 2, 16), (100, 12, 5, 2, 17)])
def test_block_lu_equals_cyclic_reduction_fp64(n, b_pml, b_slab, fronts, R, monkeypatch):
    s, m, om = make(n, b_pml, b_slab, fronts, 0, 3 + n)
    x = crand((R, n, n), 5 + R)
    y_lu, y_cr = both(s, x, monkeypatch)
    for r in range(R):
        assert rel(y_lu[r], y_cr[r]) <= 1e-11, r
    pb = O.Problem2D(n, om, m, O.Params(b_pml=b_pml, b_slab=b_slab, fronts=fronts))
    for r in (0, R - 1):
        assert rel(y_lu[r], pb.precondition(x[r])) <= 1e-10


def test_block_lu_mixed_and_solve(monkeypatch):
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    n, R = 128, 32
    s, m, om = make(n, 12, 4, 2, LSS_MIXED, 7)
    x = crand((R, n, n), 9)
    y_lu, y_cr = both(s, x, monkeypatch)
    assert rel(y_lu, y_cr) <= 1e-5
    th = np.linspace(0.1, 6.0, R)
    g = s.plane_wave_rhs(np.stack([np.cos(th), np.sin(th)], -1))
    u, st = s.solve(g, GmresOptions(30, 1e-8, 200))
    monkeypatch.setenv("LSS_SLAB_SOLVE", "cr")
    u_cr, st_cr = s.solve(g, GmresOptions(30, 1e-8, 200))
    for r in range(R):
        assert st[r]["relres_true"] <= 1e-8 and abs(st[r]["iters"] - st_cr[r]["iters"]) <= 1
