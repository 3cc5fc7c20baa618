"""Pins of the 3D oracle (Sec. 3.1) against the mathematics (no GPU).

The 3D construction repeats Sec. 2.2-2.4 with the 27-point neighbourhood and
the 26 directions of {-1,0,1}^3 minus 0.  Each test checks one part against
something other than itself: symmetry of the stencils under the cube group,
annihilation of plane waves, dense linear algebra on tiny grids (one slab =
H^{-1}, exact Schur sweep = H^{-1}, GMRES = dense LU), and the exactness and
adjoint statements of Sec. 2.3.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth


def problem3(n=5, b=2, bs=2, freq=None, seed=3, gauss=True, C=10.0):
    freq = freq if freq is not None else (n + 1) / 8
    om = 2 * math.pi * freq
    m = synth.gaussian_medium(n, 3, 3, 0.2, (0.8, 1.2), seed) if gauss else np.zeros((n, n, n))
    return O.Problem3D(n, om, m, O.Params(b_pml=b, b_slab=bs, C=C)), m, om


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def cube_group():
    """The 48 symmetries of the cube acting on 3x3x3 arrays: axis permutations
    composed with reflections."""
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            def g(A, perm=perm, flips=flips):
                B = np.transpose(A, perm)
                for a, f in enumerate(flips):
                    if f:
                        B = np.flip(B, axis=a)
                return B
            yield g


# ---------------------------------------------------------------- alpha / beta

def test_alpha_3d_unit_phase_and_cube_symmetry():
    a, b, s = O.interior_stencils(3, 8, 2 * math.pi * 1.5)
    assert a.size == 27
    assert np.linalg.norm(a) == pytest.approx(1.0, abs=1e-14)
    assert a[13].imag == 0 and a[13].real > 0
    A = a.reshape(3, 3, 3)
    Bt = b.reshape(3, 3, 3)
    count = 0
    for g in cube_group():
        assert np.allclose(g(A), A, atol=1e-9)
        assert np.allclose(g(Bt), Bt, atol=1e-9 * np.abs(Bt).max())
        count += 1
    assert count == 48
    # a simple smallest singular value: the minimiser is well defined
    assert s[-2] / s[-1] > 10


def test_alpha_3d_approximately_annihilates_plane_waves():
    """alpha^* exp(i omega r.p) on the 27 points is small for every unit r and
    falls as h -> 0 at fixed omega (alpha discretises the Helmholtz operator)."""
    om = 2 * math.pi * 1.0
    mu = O.neighbourhood_offsets(3)
    rng = np.random.default_rng(5)
    dirs = rng.standard_normal((12, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    res = []
    for n in (8, 16):
        a, _, _ = O.interior_stencils(3, n, om)
        h = 1 / (n + 1)
        res.append(max(abs(np.vdot(a, np.exp(1j * om * h * (mu @ r)))) for r in dirs))
    assert res[0] < 1e-2 and res[1] < res[0] / 4


def test_local_equation_bound_3d_against_dense_solution():
    """Eq. (local_c_approx) in 3D at points whose neighbourhood lies in I: the
    remainder alpha^* u + omega^2 beta^* (m u) - alpha^* g is the far part of
    the convolution, at most omega^2 sigma_min ||m u||."""
    n = 6
    om = 2 * math.pi * 1.2
    m = synth.gaussian_medium(n, 3, 2, 0.2, (0.8, 1.2), 7)
    a, beta, s = O.interior_stencils(3, n, om)
    kw = O.nystrom_weights(3, n, om, n)
    A = O.dense_ls_matrix(n, om, m, kw)
    g = O.ls_rhs(m, om, kw, (0.48, 0.6, 0.64))
    u = np.linalg.solve(A, g.reshape(-1)).reshape(g.shape)
    bound = om ** 2 * s[-1] * np.linalg.norm(m * u)
    worst = 0
    for i in itertools.product(range(1, n - 1), repeat=3):
        sl = tuple(slice(c - 1, c + 2) for c in i)
        r = np.vdot(a, u[sl].reshape(-1)) + om ** 2 * np.vdot(beta, (m * u)[sl].reshape(-1)) \
            - np.vdot(a, g[sl].reshape(-1))
        worst = max(worst, abs(r))
    assert worst <= bound * (1 + 1e-8)
    assert worst > 1e-6 * bound        # the bound is not vacuous at this size


# ---------------------------------------------------------------- gamma

def test_gamma_3d_annihilates_26_directions_and_is_unique():
    rng = np.random.default_rng(1)
    h = 1 / 17
    mu = O.neighbourhood_offsets(3)
    R = O.pml_directions(3)
    assert R.shape == (26, 3)
    for _ in range(4):
        om = rng.uniform(8, 30)
        sig = [np.array([-0.02, -0.01, -0.003]) * rng.uniform(0.5, 2), np.zeros(3),
               np.array([0.001, 0.004, 0.009]) * rng.uniform(0.5, 2)]
        c = O.pml_stencil(om, h, sig)
        gamma = np.conj(c)
        dz = np.stack([mu[:, a] * h + 1j * (sig[a][mu[:, a] + 1] - sig[a][1]) for a in range(3)], axis=1)
        F = np.exp(1j * om * dz @ R.T)
        assert np.linalg.norm(gamma.conj() @ F) <= 1e-13 * np.linalg.norm(F)
        sv = np.linalg.svd(F, compute_uv=False)
        assert sv[-1] > 1e-12 * sv[0]          # rank 26: unique up to phase
        assert np.linalg.norm(gamma) == pytest.approx(1.0, abs=1e-14)


def test_pml_stencils_3d_mirror_symmetric():
    pb, _, _ = problem3(n=4, b=2, bs=3, gauss=False)
    n, b = pb.n, pb.b
    for i1 in range(-b, 0):
        for i2 in range(-b, n + 2 + b):
            for i3 in (-b, -1, 0, 2, n + 1 + b):
                c = pb.row(i1, i2, i3)
                assert np.allclose(pb.row(n + 1 - i1, i2, i3), c[::-1, :, :], atol=1e-12)
                assert np.allclose(pb.row(i1, n + 1 - i2, i3), c[:, ::-1, :], atol=1e-12)
                assert np.allclose(pb.row(i1, i2, n + 1 - i3), c[:, :, ::-1], atol=1e-12)
                assert np.allclose(pb.row(i2, i1, i3), np.transpose(c, (1, 0, 2)), atol=1e-12)
                assert np.allclose(pb.row(i3, i2, i1), np.transpose(c, (2, 1, 0)), atol=1e-12)


# ---------------------------------------------------------------- H, sweep

def test_3d_zero_medium_one_slab_preconditioner_is_identity():
    pb, _, _ = problem3(n=4, b=2, bs=10, gauss=False)
    assert pb.n_slabs == 1
    g = crand((4, 4, 4), 0)
    assert np.linalg.norm(pb.precondition(g) - g) <= 1e-11 * np.linalg.norm(g)


def test_3d_one_slab_sweep_is_exact_inverse_of_H():
    pb, _, _ = problem3(n=4, b=2, bs=10)
    H = pb.assemble_H().toarray()
    r = crand((4, 4, 4), 1)
    f = pb.sparsify_rhs(r)
    ut = np.linalg.solve(H, f.reshape(-1)).reshape(f.shape)
    assert np.linalg.norm(pb.precondition(r) - pb.extract(ut)) <= 1e-11 * np.linalg.norm(ut)


def test_3d_sweep_with_exact_schur_inverses_solves_H():
    pb, _, _ = problem3(n=5, b=2, bs=2)
    assert pb.n_slabs >= 3
    H = pb.assemble_H().toarray()
    f = crand((pb.n_tot,) * 3, 2)
    ut = pb.sweep(f, T=pb.exact_T_ops())
    ref = np.linalg.solve(H, f.reshape(-1)).reshape(f.shape)
    assert np.linalg.norm(ut - ref) <= 1e-10 * np.linalg.norm(ref)


def test_3d_first_moving_pml_operator_is_exact():
    pb, _, _ = problem3(n=5, b=2, bs=2)
    T = pb.exact_T_ops()
    w = pb.slab_last[0] - pb.slab_first[0] + 1
    v = crand((w, pb.n_tot, pb.n_tot), 3)
    assert np.linalg.norm(pb.T(0, v) - T(0, v)) <= 1e-11 * np.linalg.norm(T(0, v))


def test_3d_subproblem_rows_of_D_are_rows_of_H():
    pb, _, _ = problem3(n=4, b=2, bs=2)
    H = pb.assemble_H().toarray()
    nt, b = pb.n_tot, pb.b
    for i in range(1, pb.n_slabs):
        M, layers, na = pb.subproblem(i)
        M = M.toarray()
        s, e = pb.slab_first[i], pb.slab_last[i]
        for x1 in range(s, e + 1):
            a = layers.index(x1)
            for q in range(0, nt * nt, 7):
                rS = M[a * nt * nt + q].reshape(len(layers), nt * nt)
                rH = H[(x1 + b) * nt * nt + q].reshape(nt, nt * nt)
                assert np.array_equal(rS[na:], rH[s + b:e + b + 1])
                assert np.array_equal(rS[na - 1], rH[s - 1 + b])
                assert np.all(rS[:na - 1] == 0)


def test_3d_preconditioner_transpose_is_bilinear_adjoint():
    pb, _, _ = problem3(n=5, b=2, bs=2)
    x, y = crand((5, 5, 5), 4), crand((5, 5, 5), 5)
    lhs = np.sum(pb.precondition(x) * y)
    rhs = np.sum(x * pb.precondition_transpose(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- GMRES / solve

def test_3d_gmres_matches_dense_solve_and_preconditioner_is_accurate():
    n = 8
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, 3, 3, 0.15, (0.8, 1.2), 9)
    d = np.ones(3) / math.sqrt(3)
    res, relres, pb, g = O.solve(n, om, m, d, O.Params(b_pml=3, b_slab=3), tol=1e-12)
    A = O.dense_ls_matrix(n, om, m, pb.kw)
    u = np.linalg.solve(A, g.reshape(-1)).reshape(g.shape)
    assert np.linalg.norm(res.x - u) <= 1e-10 * np.linalg.norm(u)
    # 'fairly accurate' (Sec. 2.4): P g close to A^{-1} g, few iterations (Sec. 3.2)
    assert np.linalg.norm(pb.precondition(g) - u) <= 0.1 * np.linalg.norm(u)
    assert res.iters <= 10


def test_3d_zero_medium_gives_zero_field():
    n = 6
    res, relres, pb, g = O.solve(n, 2 * math.pi, np.zeros((n, n, n)), (1.0, 0.0, 0.0),
                                 O.Params(b_pml=2, b_slab=3))
    assert np.all(g == 0) and np.all(res.x == 0) and res.iters == 0
