"""The recursive approach of Sec. 3.1 through the C ABI against the oracle's
recursive sweep, element by element.

Every slab subproblem is swept along x2 over quasi-1D sub-slab problems
(block tridiagonal along x3, factored by block Gaussian elimination); the
slab operator T~_i is that inner sweep.  Covered: T~_i of every slab at 1e-10
in FP64 (first, middle and last slabs: left-padded, unpadded and ragged
sub-slab problems); P at 1e-10 for one to six slabs, with one and two fronts;
the FGMRES solution at 1e-10 with iterations +-1 at 1e-8; the mixed form
within 1e-4 of the oracle's P and +2 iterations; the 3D workload (n = 64)
solved to relres 1e-8 measured with the oracle's operator, within one
iteration of the non-recursive approach (the paper reports zero or one
more).  Tolerances as for the non-recursive 3D path.
"""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D3 = np.ones(3) / math.sqrt(3.0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


def make(n, b, bs, seed, precision=0, fronts=1):
    from paper_1705_09443_gb300 import LSSolver
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 3, 3, 0.15, (0.8, 1.2), seed)
    s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=b, b_slab=bs,
                 precision=precision, fronts=fronts, recursive=True)
    pb = O.Problem3D(n, om, m, O.Params(b_pml=b, b_slab=bs, fronts=fronts, recursive=True))
    return s, m, om, pb


@pytest.fixture(scope="module")
def n8():
    return make(8, 3, 3, 9)


def test_slab_operators_match_oracle(n8):
    s, m, om, pb = n8
    assert s.n_slabs == pb.n_slabs == 4
    for i in range(pb.n_slabs):
        nl = pb.slab_last[i] - pb.slab_first[i] + 1
        v = crand((nl, pb.n_tot, pb.n_tot), 100 + i)
        w = s.apply_slab(i, to_dev(v[None])).cpu().numpy()[0]
        assert rel(w, pb.T(i, v)) <= 1e-10, i


@pytest.mark.parametrize("n,b,bs,fronts", [(6, 2, 20, 1), (6, 2, 4, 1), (7, 2, 3, 1), (9, 2, 2, 1), (8, 3, 3, 2),
                                           (9, 2, 2, 2)])
def test_preconditioner_matches_oracle(n, b, bs, fronts):
    s, m, om, pb = make(n, b, bs, 3 + n, fronts=fronts)
    assert s.n_slabs == pb.n_slabs
    x = crand((2, n, n, n), 8 + n)
    y = s.apply_P(to_dev(x)).cpu().numpy()
    for r in range(2):
        assert rel(y[r], pb.precondition(x[r])) <= 1e-10


def test_solution_and_mixed(n8):
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    s, m, om, pb = n8
    g = s.plane_wave_rhs(D3[None])
    u, st = s.solve(g, GmresOptions(30, 1e-13, 200))
    ref, _, _, _ = O.solve(8, om, m, D3, problem=pb, tol=1e-13)
    assert st[0]["converged"] and rel(u[0].cpu().numpy(), ref.x) <= 1e-10
    _, st8 = s.solve(g, GmresOptions(30, 1e-8, 200))
    ref8, _, _, _ = O.solve(8, om, m, D3, problem=pb, tol=1e-8)
    assert abs(st8[0]["iters"] - ref8.iters) <= 1
    s32, _, _, _ = make(8, 3, 3, 9, precision=LSS_MIXED)
    x = crand((1, 8, 8, 8), 5)
    assert rel(s32.apply_P(to_dev(x)).cpu().numpy()[0], pb.precondition(x[0])) <= 1e-4
    _, st32 = s32.solve(g, GmresOptions(30, 1e-8, 200))
    assert st32[0]["relres_true"] <= 1e-8 and st32[0]["iters"] <= st8[0]["iters"] + 2


def test_3d_workload_recursive_mixed():
    """n = 64, omega/2pi = 16, 17 slabs x 17 sub-slab problems of up to
    18 x 18 x 82 unknowns: relres <= 1e-8 with the oracle's operator and at
    most one iteration more than the non-recursive approach."""
    from paper_1705_09443_gb300 import GmresOptions, LSSolver, LSS_MIXED
    w = synth.WORKLOADS["3d_n64"]
    m, dirs = synth.make_workload(w)
    its = []
    for recursive in (True, False):
        s = LSSolver(w.n, w.omega, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=w.b_pml,
                     b_slab=w.b_slab, precision=LSS_MIXED, recursive=recursive)
        g = s.plane_wave_rhs(dirs)
        u, st = s.solve(g, GmresOptions(30, 1e-8, 200))
        its.append(st[0]["iters"])
        if recursive:
            kw = O.nystrom_weights(3, w.n, w.omega, w.n)
            g_ref = O.ls_rhs(m, w.omega, kw, dirs[0])
            res = g_ref - O.ls_apply(u[0].cpu().numpy(), m, w.omega, kw)
            assert np.linalg.norm(res) / np.linalg.norm(g_ref) <= 1e-8 * (1 + 1e-6)
        del s
    assert its[0] <= its[1] + 1


def test_recursive_is_3d_only():
    from paper_1705_09443_gb300 import LSSolver, LssError
    m = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(LssError):
        LSSolver(16, 10.0, m, b_pml=4, recursive=True)
