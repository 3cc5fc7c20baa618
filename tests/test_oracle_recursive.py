"""Pins of the oracle's recursive approach (Sec. 3.1) against the mathematics
(no GPU).

Each quasi-2D slab subproblem S_i is itself swept along x2: sub-slabs E_j
(the partition of x2 that the slabs use of x1), each padded before its first
x2-layer with b_aux auxiliary PML layers whose rows take the auxiliary
profile along x2, the layer's own profile along x1 and the physical one along
x3.  Checks:
  * with the exact Schur inverses of S_i's elimination along x2 the inner
    sweep is S_i^{-1}: the recursive T~_i equals the non-recursive T~_i;
  * in a homogeneous medium (m = 0) the construction is symmetric under the
    exchange of x1 and x2: sub-slab j of slab i is the transposed image of
    sub-slab i of slab j, so the inner auxiliary rows carry exactly the
    profiles the outer ones carry (a planted slip that gives the corner rows
    the physical x1 profile breaks it);
  * the inner sweep is an approximation (T~_i differs from the exact slab
    solve by a few percent here) that leaves the GMRES iteration count within
    one of the non-recursive one (the paper reports zero or one more).
"""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def pair():
    n = 5
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 3, 3, 0.2, (0.8, 1.2), 3)
    rec = O.Problem3D(n, om, m, O.Params(b_pml=2, b_slab=2, recursive=True))
    non = O.Problem3D(n, om, m, O.Params(b_pml=2, b_slab=2))
    return rec, non


def test_exact_inner_sweep_is_the_slab_solve(pair):
    rec, non = pair
    assert rec.n_slabs == 4
    for i in range(rec.n_slabs):
        nl = rec.slab_last[i] - rec.slab_first[i] + 1
        v = crand((nl, rec.n_tot, rec.n_tot), 10 + i)
        assert rel(rec.T_recursive(i, v, T=rec.exact_inner_ops(i)), non.T(i, v)) <= 1e-12


def test_inner_sweep_approximates_the_slab_solve(pair):
    rec, non = pair
    for i in range(rec.n_slabs):
        nl = rec.slab_last[i] - rec.slab_first[i] + 1
        v = crand((nl, rec.n_tot, rec.n_tot), 20 + i)
        err = rel(rec.T(i, v), non.T(i, v))
        assert 1e-4 <= err <= 0.2


def _swap_defect(pb, i, j, seed):
    """|| T~_{i,j} v - swap(T~_{j,i} swap(v)) || / || T~_{i,j} v || on D_i x E_j,
    for v supported on D_i x E_j."""
    na_i, na_j = pb.n_aux[i], pb.n_aux[j]
    nd_i = pb.slab_last[i] - pb.slab_first[i] + 1
    nd_j = pb.slab_last[j] - pb.slab_first[j] + 1
    v = np.zeros((len(pb.slab_layers[i]), nd_j, pb.n_tot), complex)
    v[na_i:] = crand((nd_i, nd_j, pb.n_tot), seed)
    a = pb._Tinner(i, j, v)[na_i:]
    vs = np.zeros((len(pb.slab_layers[j]), nd_i, pb.n_tot), complex)
    vs[na_j:] = np.transpose(v[na_i:], (1, 0, 2))
    b = np.transpose(pb._Tinner(j, i, vs)[na_j:], (1, 0, 2))
    return rel(b, a)


def _homogeneous(n=6):
    om = 2 * math.pi * (n + 1) / 8
    return O.Problem3D(n, om, np.zeros((n, n, n)), O.Params(b_pml=2, b_slab=2, recursive=True))


def test_x1_x2_exchange_symmetry():
    pb = _homogeneous()
    assert pb.n_slabs == 4
    for (i, j) in [(1, 2), (0, 3), (1, 1), (3, 2)]:
        assert _swap_defect(pb, i, j, 30 + 4 * i + j) <= 1e-12


def test_planted_slip_breaks_the_exchange_symmetry():
    pb = _homogeneous()
    pb.sigma1_of = lambda i, x1: pb.sigma(np.array([x1 - 1, x1, x1 + 1]))   # physical x1 profile everywhere
    pb._gcache.clear()
    pb._inner_factor()
    assert _swap_defect(pb, 1, 2, 34) >= 1e-4


def test_recursive_preconditioner_iterations():
    n = 12
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 3, 3, 0.15, (0.8, 1.2), 5)
    d = np.ones(3) / math.sqrt(3.0)
    it = []
    for recursive in (False, True):
        res, relres, _, _ = O.solve(n, om, m, d, O.Params(b_pml=4, b_slab=4, recursive=recursive), tol=1e-8)
        assert relres <= 1e-8
        it.append(res.iters)
    assert it[1] <= it[0] + 1
