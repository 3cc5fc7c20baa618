"""Pins of the CPU oracle against the mathematics (no GPU).

Each test checks one oracle function against something other than itself:
closed forms, brute-force quadrature or summation, dense linear algebra on
tiny grids, and invariants the paper states (Sec. 2.1-2.4).
"""
import math

import numpy as np
import pytest
import scipy.special as sps
from scipy import integrate

from oracle import lss_oracle as O
import synth


def small_problem(n=10, b=3, bs=3, freq=None, seed=3, C=10.0, gauss=True):
    freq = freq if freq is not None else (n + 1) / 8
    om = 2 * math.pi * freq
    if gauss:
        m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), seed)
    else:
        m = np.zeros((n, n))
    return O.Problem2D(n, om, m, O.Params(b_pml=b, b_slab=bs, C=C)), m, om


# ---------------------------------------------------------------- Green / k_0

def test_green_solves_helmholtz_away_from_origin():
    """(-Laplace - omega^2) G = 0 for x != 0 (Sec. 2.2.1), 4th-order differences."""
    om = 2 * math.pi * 3.0
    d = 1e-3
    for x0 in [(0.3, 0.1), (-0.2, 0.45), (0.05, -0.6)]:
        def G(dx, dy):
            return O.green(2, om, math.hypot(x0[0] + dx, x0[1] + dy))
        lap = 0
        for (ax, ay) in [(1, 0), (0, 1)]:
            lap += (-G(2 * d * ax, 2 * d * ay) + 16 * G(d * ax, d * ay) - 30 * G(0, 0)
                    + 16 * G(-d * ax, -d * ay) - G(-2 * d * ax, -2 * d * ay)) / (12 * d * d)
        res = -lap - om ** 2 * G(0, 0)
        assert abs(res) < 1e-5 * om ** 2 * abs(G(0, 0))
    # 3D: the same for exp(i omega r)/(4 pi r)
    for x0 in [(0.3, 0.1, 0.2), (-0.25, 0.4, 0.1)]:
        def G3(v):
            return O.green(3, om, np.linalg.norm(np.asarray(x0) + v))
        lap = 0
        for a in range(3):
            e = np.zeros(3)
            e[a] = d
            lap += (-G3(2 * e) + 16 * G3(e) - 30 * G3(0 * e) + 16 * G3(-e) - G3(-2 * e)) / (12 * d * d)
        assert abs(-lap - om ** 2 * G3(0 * e)) < 1e-5 * om ** 2 * abs(G3(0 * e))


def test_green_log_singularity_2d():
    """G(r) = -(1/2pi)(log(omega r/2) + gamma_E) + i/4 + O(r^2 log r) as r -> 0."""
    om = 7.0
    for r in [1e-4, 1e-5]:
        lim = -(math.log(om * r / 2) + np.euler_gamma) / (2 * math.pi) + 0.25j
        assert abs(O.green(2, om, r) - lim) < 10 * (om * r) ** 2 * abs(math.log(om * r))


@pytest.mark.parametrize("n,freq", [(64, 8.0), (16, 8.0), (256, 32.0)])
def test_k0_matches_adaptive_cartesian_quadrature_2d(n, freq):
    """k_0 (cell integral, polar closed form) against scipy.dblquad of G over the
    four quadrants of the cell, with the singularity at a corner."""
    om = 2 * math.pi * freq
    h = 1.0 / (n + 1)
    k0 = O.cell_integral_G(2, om, h)

    def f(y, x):
        return 0.25j * sps.hankel1(0, om * math.hypot(x, y))
    re = integrate.dblquad(lambda y, x: f(y, x).real, 0, h / 2, 0, h / 2, epsabs=0, epsrel=1e-12)[0]
    im = integrate.dblquad(lambda y, x: f(y, x).imag, 0, h / 2, 0, h / 2, epsabs=0, epsrel=1e-12)[0]
    assert abs(k0 - 4 * (re + 1j * im)) <= 1e-11 * abs(k0)


def test_k0_matches_adaptive_cartesian_quadrature_3d():
    om = 2 * math.pi * 4.0
    h = 1.0 / 17

    def g(z, y, x):
        r = math.sqrt(x * x + y * y + z * z)
        return np.exp(1j * om * r) / (4 * math.pi * r)
    k0 = O.cell_integral_G(3, om, h)
    re = integrate.tplquad(lambda z, y, x: g(z, y, x).real, 0, h / 2, 0, h / 2, 0, h / 2,
                           epsabs=0, epsrel=1e-10)[0]
    im = integrate.tplquad(lambda z, y, x: g(z, y, x).imag, 0, h / 2, 0, h / 2, 0, h / 2,
                           epsabs=0, epsrel=1e-10)[0]
    assert abs(k0 - 8 * (re + 1j * im)) <= 1e-9 * abs(k0)


def test_nystrom_weights_are_even_and_pointwise():
    kw = O.nystrom_weights(2, 12, 9.0, 12)
    assert np.allclose(kw, kw[::-1, :], rtol=0, atol=0)
    assert np.allclose(kw, kw[:, ::-1], rtol=0, atol=0)
    assert np.allclose(kw, kw.T, rtol=0, atol=0)
    h = 1 / 13
    assert kw[12 + 3, 12 + 4] == pytest.approx(0.25j * sps.hankel1(0, 9.0 * 5 * h) * h * h, rel=1e-15)


def test_nystrom_sum_converges_to_the_integral():
    """sum_j k_{i-j} f_j approximates int G(p_i - y) f(y) dy (Sec. 2.1) for a smooth
    bump f; reference by adaptive quadrature in polar coordinates about p_i.  With
    the cell-integral k_0 the error falls as O(h^2); a wrong diagonal weight
    leaves an O(h^2 log h) error that is several times larger."""
    om = 2 * math.pi * 4

    def f(x, y):
        return np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.08 ** 2))

    def g(r, th):
        return 0.25j * sps.hankel1(0, om * r) * f(0.5 + r * math.cos(th), 0.5 + r * math.sin(th)) * r
    re = integrate.dblquad(lambda r, th: g(r, th).real, 0, 2 * math.pi, 1e-300, 0.6,
                           epsabs=1e-14, epsrel=1e-12)[0]
    im = integrate.dblquad(lambda r, th: g(r, th).imag, 0, 2 * math.pi, 1e-300, 0.6,
                           epsabs=1e-14, epsrel=1e-12)[0]
    ref = re + 1j * im
    errs = []
    for n in (63, 127):
        h = 1 / (n + 1)
        kw = O.nystrom_weights(2, n, om, n)
        xs = np.arange(1, n + 1) * h
        X, Y = np.meshgrid(xs, xs, indexing="ij")
        i = (n + 1) // 2
        idx = n + i - 1 - np.arange(n)
        S = np.sum(kw[idx[:, None], idx[None, :]] * f(X, Y))
        errs.append(abs(S - ref) / abs(ref))
    assert errs[0] < 6e-3 and errs[1] < 1.5e-3 and errs[0] / errs[1] > 3.8


# ---------------------------------------------------------------- LS operator

@pytest.mark.parametrize("n", [5, 7, 12])
def test_ls_apply_fft_equals_direct_sum(n):
    rng = np.random.default_rng(n)
    om = 2 * math.pi * 3.0
    kw = O.nystrom_weights(2, n, om, n)
    m = rng.uniform(-0.5, 0.5, (n, n))
    u = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = O.ls_apply(u, m, om, kw)
    b = O.ls_apply_direct(u, m, om, kw)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_ls_apply_fft_equals_direct_sum_3d():
    n = 5
    rng = np.random.default_rng(1)
    om = 2 * math.pi * 2.0
    kw = O.nystrom_weights(3, n, om, n)
    m = rng.uniform(-0.5, 0.5, (n, n, n))
    u = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    a = O.ls_apply(u, m, om, kw)
    b = O.ls_apply_direct(u, m, om, kw)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_ls_transpose_is_bilinear_adjoint():
    n = 9
    rng = np.random.default_rng(2)
    om = 2 * math.pi * 2.0
    kw = O.nystrom_weights(2, n, om, n)
    m = rng.uniform(-0.5, 0.5, (n, n))
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lhs = np.sum(O.ls_apply(x, m, om, kw) * y)
    rhs = np.sum(x * O.ls_apply_transpose(y, m, om, kw))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


# ---------------------------------------------------------------- alpha / beta

def test_alpha_unit_phase_and_d4_symmetry():
    a, b, s = O.interior_stencils(2, 32, 2 * math.pi * 4)
    assert np.linalg.norm(a) == pytest.approx(1.0, abs=1e-14)
    assert a[4].imag == 0 and a[4].real > 0
    A = a.reshape(3, 3)
    for T in (A.T, A[::-1, :], A[:, ::-1], A[::-1, ::-1]):
        assert np.allclose(T, A, atol=1e-10)
    assert s[-1] / s[0] < 1e-3 and s[-2] / s[-1] > 10


def test_alpha_approximately_annihilates_plane_waves():
    """alpha discretises (-Laplace - omega^2): alpha^* exp(i omega r.p) on mu is
    O((omega h)^k) and falls as h -> 0 at fixed omega."""
    om = 2 * math.pi * 2.0
    res = []
    for n in (16, 32):
        a, _, _ = O.interior_stencils(2, n, om)
        h = 1 / (n + 1)
        mu = O.neighbourhood_offsets(2)
        worst = 0
        for th in np.linspace(0, 2 * math.pi, 13):
            r = np.array([math.cos(th), math.sin(th)])
            w = np.exp(1j * om * h * (mu @ r))
            worst = max(worst, abs(np.vdot(a, w)))
        res.append(worst)
    assert res[0] < 1e-2 and res[1] < res[0] / 4


def test_local_equation_bound_against_dense_solution():
    """For the exact discrete LS solution, the truncation in Eq. (local_c_approx) is
    omega^2 alpha^* K_{mu_i,mu_i^c}[mu]_{mu_i^c}; its size is at most
    omega^2 sigma_min ||m u||.  A wrong beta (missing conjugate, transposed K)
    exceeds this bound by orders of magnitude."""
    n = 16
    om = 2 * math.pi * 2.5
    m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), 5)
    a, beta, s = O.interior_stencils(2, n, om)
    kw = O.nystrom_weights(2, n, om, n)
    A = O.dense_ls_matrix(n, om, m, kw)
    g = O.ls_rhs(m, om, kw, (0.6, 0.8))
    u = np.linalg.solve(A, g.reshape(-1)).reshape(n, n)
    bound = om ** 2 * s[-1] * np.linalg.norm(m * u)
    # u on Z^2 is defined by Eq. (LS_d_c) itself: u_i = g_i - omega^2 (K m u)_i, g = 0 off I
    kx = O.nystrom_weights(2, n, om, n + 1)
    up = np.zeros((n + 2, n + 2), complex)
    gp = np.zeros((n + 2, n + 2), complex)
    mp = np.zeros((n + 2, n + 2))
    gp[1:-1, 1:-1], mp[1:-1, 1:-1] = g, m
    mu_src = (m * u).reshape(-1)
    src = np.array(np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")).reshape(2, -1).T
    for i1 in range(n + 2):
        for i2 in range(n + 2):
            off = np.array([i1, i2])[None, :] - src + n + 1
            up[i1, i2] = gp[i1, i2] - om ** 2 * np.sum(kx[tuple(off.T)] * mu_src)
    assert np.linalg.norm(up[1:-1, 1:-1] - u) <= 1e-10 * np.linalg.norm(u)
    worst = 0
    for i1 in range(1, n + 1):
        for i2 in range(1, n + 1):
            U = up[i1 - 1:i1 + 2, i2 - 1:i2 + 2].reshape(-1)
            Gl = gp[i1 - 1:i1 + 2, i2 - 1:i2 + 2].reshape(-1)
            MU = (mp * up)[i1 - 1:i1 + 2, i2 - 1:i2 + 2].reshape(-1)
            r = np.vdot(a, U) + om ** 2 * np.vdot(beta, MU) - np.vdot(a, Gl)
            worst = max(worst, abs(r))
    assert worst <= bound * (1 + 1e-8)
    # the bound is tight enough to matter: the neglected part is not trivially small
    assert bound < 1e-2 * om ** 2 * np.linalg.norm(kw) * np.max(np.abs(m * u))


def test_local_equation_identity_defines_beta():
    """Eq. (local_lc) holds exactly for the dense solution; with beta^* = alpha^*
    K_{mu,mu} (Eq. beta) the remainder is exactly the far part
    omega^2 alpha^* K_{mu_i,mu_i^c}[mu]_{mu_i^c}, summed here term by term."""
    n = 12
    om = 2 * math.pi * 2.5
    m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), 6)
    a, beta, s = O.interior_stencils(2, n, om)
    kw = O.nystrom_weights(2, n, om, n + 1)
    A = O.dense_ls_matrix(n, om, m, O.nystrom_weights(2, n, om, n))
    g = O.ls_rhs(m, om, O.nystrom_weights(2, n, om, n), (0.6, 0.8))
    u = np.linalg.solve(A, g.reshape(-1)).reshape(n, n)
    mu = O.neighbourhood_offsets(2)
    for i in [(3, 4), (6, 6), (8, 2)]:                  # 0-based points of I, interior
        U = np.array([u[i[0] + o[0], i[1] + o[1]] for o in mu])
        MU = np.array([m[i[0] + o[0], i[1] + o[1]] * u[i[0] + o[0], i[1] + o[1]] for o in mu])
        Gl = np.array([g[i[0] + o[0], i[1] + o[1]] for o in mu])
        far = 0
        for j1 in range(n):
            for j2 in range(n):
                if max(abs(j1 - i[0]), abs(j2 - i[1])) <= 1:
                    continue
                col = np.array([kw[i[0] + o[0] - j1 + n + 1, i[1] + o[1] - j2 + n + 1] for o in mu])
                far += np.vdot(a, col) * m[j1, j2] * u[j1, j2]
        lhs = np.vdot(a, U) + om ** 2 * np.vdot(beta, MU) + om ** 2 * far
        assert abs(lhs - np.vdot(a, Gl)) <= 1e-11 * (abs(np.vdot(a, U)) + abs(np.vdot(a, Gl)))


# ---------------------------------------------------------------- sigma / gamma

def test_sigma_profile_values():
    n, b, C, om = 10, 4, 8.0, 3.0
    s = O.pml_sigma(np.arange(-b - 1, n + 3 + b), n, b, C, om)
    assert s[0] == pytest.approx(-C / om)          # Dirichlet layer x = -h - eta
    assert s[b] == 0.0                             # idx -1, x = -h
    assert np.all(s[b:b + n + 4] == 0)             # idx -1 .. n+2
    assert s[-1] == pytest.approx(C / om)
    # antisymmetric under the reflection idx -> n+1-idx
    assert np.allclose(s, -s[::-1], atol=1e-15)


def test_gamma_annihilates_and_is_unique():
    rng = np.random.default_rng(0)
    h = 1 / 33
    for _ in range(5):
        om = rng.uniform(10, 60)
        s1 = np.array([-0.02, -0.01, -0.003]) * rng.uniform(0.5, 2.0)
        s2 = np.array([0.0, 0.0, 0.0]) if rng.random() < 0.5 else np.array([0.001, 0.004, 0.009])
        c = O.pml_stencil(om, h, [s1, s2])
        gamma = np.conj(c)
        mu = O.neighbourhood_offsets(2)
        R = O.pml_directions(2)
        dz = np.stack([mu[:, 0] * h + 1j * (s1[mu[:, 0] + 1] - s1[1]),
                       mu[:, 1] * h + 1j * (s2[mu[:, 1] + 1] - s2[1])], axis=1)
        F = np.exp(1j * om * dz @ R.T)
        assert np.linalg.norm(gamma.conj() @ F) <= 1e-13 * np.linalg.norm(F)
        sv = np.linalg.svd(F, compute_uv=False)
        assert sv[-1] > 1e-10 * sv[0]              # rank 8: gamma unique up to phase
        assert np.linalg.norm(gamma) == pytest.approx(1.0, abs=1e-14)


def test_pml_stencils_mirror_symmetric():
    """Sec. 2.2.2: by the symmetry of the stretching, the PML stencil at a
    mirrored point is the mirrored stencil."""
    pb, _, _ = small_problem(n=10, b=4, bs=3, gauss=False)
    n, b = pb.n, pb.b
    for i1 in range(-b, 0):
        for i2 in range(-b, n + 2 + b):
            c = pb.row(i1, i2)
            assert np.allclose(pb.row(n + 1 - i1, i2), c[::-1, :], atol=1e-12)
            assert np.allclose(pb.row(i1, n + 1 - i2), c[:, ::-1], atol=1e-12)
            assert np.allclose(pb.row(i2, i1), c.T, atol=1e-12)


def test_frequency_samples_reading():
    m = np.array([[-0.5, 0.2], [0.1, 0.0]])
    s = O.frequency_samples(m, 2.0, 4)
    assert s[0] == pytest.approx(4 * 0.8) and s[-1] == pytest.approx(4 * 1.5) and len(s) == 4
    assert O.nearest_sample(np.array([0.0, 1.0, 2.0]), 0.5) == 0   # tie -> lower
    assert O.nearest_sample(np.array([0.0, 1.0, 2.0]), 1.6) == 2
    assert len(O.frequency_samples(np.zeros((3, 3)), 2.0, 5)) == 1


# ---------------------------------------------------------------- H, sweep

def test_sparsified_system_m0_reproduces_rhs():
    """m = 0: u = g solves H u~ = f exactly (u~ = g on I, 0 elsewhere), so the
    one-slab preconditioner is the identity."""
    pb, _, _ = small_problem(n=9, b=3, bs=20, gauss=False)
    assert pb.n_slabs == 1
    rng = np.random.default_rng(0)
    g = rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9))
    assert np.linalg.norm(pb.precondition(g) - g) <= 1e-11 * np.linalg.norm(g)


def test_one_slab_sweep_is_exact_inverse_of_H():
    pb, _, _ = small_problem(n=9, b=3, bs=20)
    H = pb.assemble_H().toarray()
    rng = np.random.default_rng(1)
    r = rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9))
    f = pb.sparsify_rhs(r)
    ut = np.linalg.solve(H, f.reshape(-1)).reshape(f.shape)
    assert np.linalg.norm(pb.precondition(r) - pb.extract(ut)) <= 1e-11 * np.linalg.norm(ut)


def test_sweep_with_exact_schur_inverses_solves_H():
    """Algorithm 2 with the exact T_[i] (restrictions of H_[1:i,1:i]^{-1}, Eq. Hwv)
    is block Gaussian elimination: it returns H^{-1} f."""
    pb, _, _ = small_problem(n=10, b=3, bs=3)
    assert pb.n_slabs >= 3
    H = pb.assemble_H().toarray()
    rng = np.random.default_rng(2)
    f = rng.standard_normal((pb.n_tot, pb.n_tot)) + 1j * rng.standard_normal((pb.n_tot, pb.n_tot))
    ut = pb.sweep(f, T=pb.exact_T_ops())
    ref = np.linalg.solve(H, f.reshape(-1)).reshape(f.shape)
    assert np.linalg.norm(ut - ref) <= 1e-10 * np.linalg.norm(ref)


def test_first_moving_pml_operator_is_exact():
    """T~_[1] = T_[1] (Sec. 2.3)."""
    pb, _, _ = small_problem(n=10, b=3, bs=3)
    T = pb.exact_T_ops()
    rng = np.random.default_rng(3)
    w = pb.slab_last[0] - pb.slab_first[0] + 1
    v = rng.standard_normal((w, pb.n_tot)) + 1j * rng.standard_normal((w, pb.n_tot))
    assert np.linalg.norm(pb.T(0, v) - T(0, v)) <= 1e-11 * np.linalg.norm(T(0, v))


def test_subproblem_rows_of_D_are_rows_of_H():
    """Eq. (Hwv_approx): the rows of D_i are H's rows; the coupling to D_{i-1}'s
    last layer lands on the adjacent auxiliary layer, the coupling to D_{i+1} is
    dropped."""
    pb, _, _ = small_problem(n=10, b=3, bs=3)
    H = pb.assemble_H().toarray()
    nt, b = pb.n_tot, pb.b
    for i in range(1, pb.n_slabs):
        M, layers, na = pb.subproblem(i)
        M = M.toarray()
        s, e = pb.slab_first[i], pb.slab_last[i]
        for x1 in range(s, e + 1):
            a = layers.index(x1)
            for i2 in range(nt):
                rS = M[a * nt + i2].reshape(len(layers), nt)
                rH = H[(x1 + b) * nt + i2].reshape(nt, nt)
                assert np.array_equal(rS[na:], rH[s + b:e + b + 1])
                assert np.array_equal(rS[na - 1], rH[s - 1 + b])
                assert np.all(rS[:na - 1] == 0)


def test_preconditioner_transpose_is_bilinear_adjoint():
    pb, _, _ = small_problem(n=10, b=3, bs=3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    y = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    lhs = np.sum(pb.precondition(x) * y)
    rhs = np.sum(x * pb.precondition_transpose(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- GMRES / solve

def test_gmres_matches_dense_solve():
    n = 12
    om = 2 * math.pi * 2.0
    m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), 9)
    res, relres, pb, g = O.solve(n, om, m, (1.0, 0.0), O.Params(b_pml=4, b_slab=3), tol=1e-13)
    A = O.dense_ls_matrix(n, om, m, pb.kw)
    u = np.linalg.solve(A, g.reshape(-1)).reshape(n, n)
    assert np.linalg.norm(res.x - u) <= 1e-11 * np.linalg.norm(u)
    # unpreconditioned GMRES reaches the same solution
    r2 = O.gmres(lambda v: O.ls_apply(v, m, om, pb.kw), lambda v: v, g, restart=60, tol=1e-13)
    assert np.linalg.norm(r2.x - u) <= 1e-11 * np.linalg.norm(u)


def test_zero_medium_gives_zero_field():
    n = 16
    res, relres, pb, g = O.solve(n, 2 * math.pi * 2, np.zeros((n, n)), (1.0, 0.0),
                                 O.Params(b_pml=4, b_slab=4))
    assert np.all(g == 0) and np.all(res.x == 0) and res.iters == 0


def test_reciprocity_of_point_source_response():
    """(A^{-1} K)_{ab} = (A^{-1} K)_{ba}: K is complex symmetric (k even)."""
    n = 12
    om = 2 * math.pi * 2.0
    m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), 11)
    pb = O.Problem2D(n, om, m, O.Params(b_pml=4, b_slab=3))
    A = lambda u: O.ls_apply(u, m, om, pb.kw)  # noqa: E731
    a, bb = (2, 3), (8, 9)

    def resp(src, rcv):
        e = np.zeros((n, n), complex)
        e[src] = 1
        rhs = O.ls_apply(e, np.ones((n, n)), om, pb.kw) - e      # omega^2 K e
        x = O.gmres(A, pb.precondition, rhs, tol=1e-13).x
        return x[rcv]
    assert abs(resp(a, bb) - resp(bb, a)) <= 1e-10 * abs(resp(a, bb))


def test_preconditioner_approximates_inverse():
    """The sweep is 'fairly accurate': P g is close to A^{-1} g, and GMRES needs few
    iterations (Sec. 2.5).  A sign error in the PML or in beta breaks both."""
    n = 48
    om = 2 * math.pi * (n + 1) / 8
    m, _ = synth.make_workload("2d_n64", n=n)
    res, relres, pb, g = O.solve(n, om, m, (1.0, 0.0), tol=1e-12)
    u = res.x
    assert np.linalg.norm(pb.precondition(g) - u) <= 0.1 * np.linalg.norm(u)
    res8, _, _, _ = O.solve(n, om, m, (1.0, 0.0), tol=1e-8, problem=pb)
    assert res8.iters <= 6 and relres <= 1e-11
