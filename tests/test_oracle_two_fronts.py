"""Pins of the oracle's two-front sweep (Sec. 2.4 remark 1; the setting of the
experiments in Sec. 2.5) against the mathematics (no GPU).

The left front eliminates slabs 0..c-1 toward the middle slab c = (l-1)//2,
the right front slabs l-1..c+1; c takes its couplings from both neighbours and
both fronts substitute back.  Checks:
  * with the exact Schur inverses (restrictions of H_{[0:i]}^{-1},
    H_{[i:l]}^{-1} and H^{-1}) the two-front sweep is H^{-1} (2D for one to
    six slabs with a ragged last slab, and 3D);
  * the first and the last slab carry no auxiliary layers, so their T~ are
    exact: T~_0 = T_[0] and T~_{l-1} is the restriction of H_{[l-1:l]}^{-1};
  * on a medium symmetric under x1 -> n+1-x1 with mirror-symmetric slabs,
    a right-padded slab of the two-front sweep is the x1-mirror image of the
    left-padded mirror slab of the one-front sweep, and the middle slab
    (padded on both sides) commutes with the mirror: the right-side auxiliary
    PML is the left one reflected, profile and local frequencies included;
  * as a preconditioner it is as good as one front (GMRES iterations within one).
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


def problem2(n=10, b=3, bs=3, fronts=2, symmetric=False, seed=3):
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), seed)
    if symmetric:
        m = 0.5 * (m + m[::-1])
    return O.Problem2D(n, om, m, O.Params(b_pml=b, b_slab=bs, fronts=fronts)), m, om


@pytest.mark.parametrize("bs", [20, 6, 4, 3, 2])
def test_exact_two_front_sweep_is_H_inverse_2d(bs):
    pb, _, _ = problem2(bs=bs)
    H = pb.assemble_H().toarray()
    f = crand((pb.n_tot, pb.n_tot), bs)
    ut = pb.sweep(f, T=pb.exact_T_ops_two_fronts())
    assert rel(ut.reshape(-1), np.linalg.solve(H, f.reshape(-1))) <= 1e-12


def test_exact_two_front_sweep_is_H_inverse_3d():
    n = 5
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 3, 3, 0.2, (0.8, 1.2), 3)
    pb = O.Problem3D(n, om, m, O.Params(b_pml=2, b_slab=2, fronts=2))
    assert pb.n_slabs == 4
    H = pb.assemble_H().toarray()
    f = crand((pb.n_tot,) * 3, 4)
    ut = pb.sweep(f, T=pb.exact_T_ops_two_fronts())
    assert rel(ut.reshape(-1), np.linalg.solve(H, f.reshape(-1))) <= 1e-12


def test_auxiliary_sides():
    pb, _, _ = problem2(bs=2)          # 6 slabs, c = 2
    assert pb.n_slabs == 6
    assert [pb.aux_sides(i) for i in range(6)] == [
        (False, False), (True, False), (True, True), (False, True), (False, True), (False, False)]
    assert pb.n_aux == [0, 3, 3, 0, 0, 0]
    widths = [pb.slab_last[i] - pb.slab_first[i] + 1 for i in range(6)]
    assert [pb.n_layers[i] - widths[i] for i in range(6)] == [0, 3, 6, 3, 3, 0]


def test_boundary_slabs_are_exact():
    pb, _, _ = problem2(bs=3)
    T_ex = pb.exact_T_ops_two_fronts()
    for i in (0, pb.n_slabs - 1):
        nl = pb.slab_last[i] - pb.slab_first[i] + 1
        v = crand((nl, pb.n_tot), 10 + i)
        assert rel(pb.T(i, v), T_ex(i, v)) <= 1e-12


def test_right_padding_mirrors_left_padding():
    n, bs = 10, 3                      # n + 2 = 12 normal layers: 4 mirror-symmetric slabs
    one, m, om = problem2(n=n, bs=bs, fronts=1, symmetric=True)
    two = O.Problem2D(n, om, m, O.Params(b_pml=3, b_slab=bs, fronts=2))
    L = one.n_slabs
    assert L == 4
    for i in range(L):
        assert one.slab_first[i] + one.slab_last[L - 1 - i] == n + 1
    # slab 2 of the two-front sweep (right padding) against slab 1 of the one-front sweep (left padding)
    nl = one.slab_last[1] - one.slab_first[1] + 1
    v = crand((nl, one.n_tot), 5)
    assert rel(two.T(2, v[::-1])[::-1], one.T(1, v)) <= 1e-12
    # a planted slip: the right profile shifted by one layer breaks the mirror
    bad = O.Problem2D(n, om, m, O.Params(b_pml=3, b_slab=bs, fronts=2))
    bad.right_sigma = lambda e, a1: O.pml_sigma(np.array([a1 - 1, a1, a1 + 1]) - e + n, n, bad.b_aux,
                                                 bad.p.C, bad.omega)
    bad._gcache.clear()
    bad._factor()
    assert rel(bad.T(2, v[::-1])[::-1], one.T(1, v)) >= 1e-3


def test_middle_slab_commutes_with_the_mirror():
    n, bs = 7, 3                       # 9 normal layers: 3 slabs, the middle one its own mirror
    pb, _, _ = problem2(n=n, bs=bs, symmetric=True)
    assert pb.n_slabs == 3 and pb.slab_first[1] + pb.slab_last[1] == n + 1
    assert pb.aux_sides(1) == (True, True)
    nl = pb.slab_last[1] - pb.slab_first[1] + 1
    v = crand((nl, pb.n_tot), 6)
    assert rel(pb.T(1, v[::-1])[::-1], pb.T(1, v)) <= 1e-12


def test_right_padding_mirrors_left_padding_3d():
    n = 6                              # 8 normal layers, slabs of 2: 4 slabs
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 3, 3, 0.2, (0.8, 1.2), 5)
    m = 0.5 * (m + m[::-1])
    one = O.Problem3D(n, om, m, O.Params(b_pml=2, b_slab=2))
    two = O.Problem3D(n, om, m, O.Params(b_pml=2, b_slab=2, fronts=2))
    assert one.n_slabs == 4
    v = crand((2, one.n_tot, one.n_tot), 7)
    assert rel(two.T(2, v[::-1])[::-1], one.T(1, v)) <= 1e-12


def test_two_fronts_precondition_as_well_as_one():
    n = 48
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 2, 4, 0.08, (0.8, 1.2), 1706)
    it = []
    for fronts in (1, 2):
        res, relres, _, _ = O.solve(n, om, m, (1.0, 0.0), O.Params(b_pml=8, b_slab=4, fronts=fronts), tol=1e-8)
        assert relres <= 1e-8
        it.append(res.iters)
    assert it[1] <= it[0] + 1


def test_transposed_two_front_sweep_is_refused():
    pb, _, _ = problem2(bs=4)
    with pytest.raises(ValueError):
        pb.precondition_transpose(np.zeros((pb.n, pb.n), dtype=np.complex128))
