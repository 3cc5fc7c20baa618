"""Pins of the oracle's incident field, right-hand side and medium gradient
(no GPU).

plane_wave / ls_rhs are checked through physics they must satisfy rather than
by restating their formula:
  * the total field v = u + u_I of the exact discrete LS solution satisfies the
    sparsified local equation alpha^* v + omega^2 beta^* (m v) ~ 0 (Sec. 2.2.1)
    at points whose neighbourhood lies in I: the convolution remainders are
    bounded by omega^2 sigma_min (||m u|| + ||m u_I||), and alpha annihilates a
    plane wave only if its wavenumber on the grid is omega h with
    h = 1/(n+1) (a wrong grid spacing or frequency scale breaks this);
  * a smooth scatterer scatters forward: with the outgoing Green's function
    (i/4) H_0^(1) of Sec. 1, the scattered field of exp(i omega d.p) is larger
    downstream (along +d) than upstream or to the sides (a sign error in the
    exponent, or the direction applied to the wrong axis, reverses this).
The dense-adjoint gradient is checked against central differences of the
misfit with dense solves.
"""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth


def test_total_field_satisfies_the_sparsified_local_equation():
    n = 20
    om = 2 * math.pi * 2.5
    m = synth.gaussian_medium(n, 2, 3, 0.12, (0.8, 1.2), 31)
    a, beta, s = O.interior_stencils(2, n, om)
    kw = O.nystrom_weights(2, n, om, n)
    A = O.dense_ls_matrix(n, om, m, kw)
    d = (0.8, 0.6)
    uI = O.plane_wave(n, om, d)
    g = O.ls_rhs(m, om, kw, d)
    u = np.linalg.solve(A, g.reshape(-1)).reshape(n, n)
    v = u + uI
    bound = om ** 2 * s[-1] * (np.linalg.norm(m * u) + np.linalg.norm(m * uI))
    worst = 0.0
    for i1 in range(1, n - 1):
        for i2 in range(1, n - 1):
            sl = (slice(i1 - 1, i1 + 2), slice(i2 - 1, i2 + 2))
            r = np.vdot(a, v[sl].reshape(-1)) + om ** 2 * np.vdot(beta, (m * v)[sl].reshape(-1))
            worst = max(worst, abs(r))
    # plus alpha's own plane-wave residual on the grid (tiny at 8+ points per wavelength)
    assert worst <= 1.5 * bound
    # the same check with the incident field on a grid of spacing 1/n fails
    xs = np.meshgrid(np.arange(1, n + 1) / n, np.arange(1, n + 1) / n, indexing="ij")
    wrong = np.exp(1j * om * (d[0] * xs[0] + d[1] * xs[1]))
    vw = u + wrong
    worst_w = max(abs(np.vdot(a, vw[i1 - 1:i1 + 2, i2 - 1:i2 + 2].reshape(-1))
                      + om ** 2 * np.vdot(beta, (m * vw)[i1 - 1:i1 + 2, i2 - 1:i2 + 2].reshape(-1)))
                  for i1 in range(1, n - 1) for i2 in range(1, n - 1))
    assert worst_w > 10 * bound


@pytest.mark.parametrize("d", [(1.0, 0.0), (0.0, -1.0), (-0.6, 0.8)])
def test_smooth_scatterer_scatters_forward(d):
    n = 31
    om = 2 * math.pi * 4.0
    h = 1 / (n + 1)
    xs = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    c = 1 + 0.1 * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.1 ** 2))
    m = 1 - 1 / c ** 2
    kw = O.nystrom_weights(2, n, om, n)
    A = O.dense_ls_matrix(n, om, m, kw)
    g = O.ls_rhs(m, om, kw, d)
    u = np.linalg.solve(A, g.reshape(-1)).reshape(n, n)

    def at(dx, dy):
        return abs(u[int(round((0.5 + dx) / h)) - 1, int(round((0.5 + dy) / h)) - 1])
    r = 0.375
    dv = np.asarray(d) / np.linalg.norm(d)
    fwd = at(r * dv[0], r * dv[1])
    back = at(-r * dv[0], -r * dv[1])
    side = max(at(-r * dv[1], r * dv[0]), at(r * dv[1], -r * dv[0]))
    assert fwd > 3 * back and fwd > 2 * side


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_dense_adjoint_gradient_matches_central_differences(dim, n):
    om = 2 * math.pi * 1.5
    m = synth.gaussian_medium(n, dim, 3, 0.15, (0.8, 1.2), 40 + dim)
    rng = np.random.default_rng(41)
    if dim == 2:
        dirs = np.array([[1.0, 0.0], [0.6, 0.8]])
    else:
        dirs = np.array([[0.0, 0.0, 1.0], [0.48, 0.6, 0.64]])
    rcv = rng.integers(0, n, size=(5, dim))
    data = (rng.standard_normal((2, 5)) + 1j * rng.standard_normal((2, 5))) * 1e-2
    grad = O.misfit_gradient_dense(n, om, m, dirs, rcv, data)
    step = 1e-6
    for p in rng.integers(0, n, size=(4, dim)):
        p = tuple(p)
        mp, mm = m.copy(), m.copy()
        mp[p] += step
        mm[p] -= step
        fd = (O.misfit(n, om, mp, dirs, rcv, data) - O.misfit(n, om, mm, dirs, rcv, data)) / (2 * step)
        assert abs(grad[p] - fd) <= 1e-7 * max(abs(fd), 1e-3 * np.abs(grad).max())


def test_gradient_vanishes_at_the_data_medium():
    """d = the fields of m itself: L has a minimum there, so dL/dm = 0."""
    n = 8
    om = 2 * math.pi * 1.5
    m = synth.gaussian_medium(n, 2, 3, 0.15, (0.8, 1.2), 44)
    dirs = np.array([[1.0, 0.0]])
    rcv = np.array([[0, 3], [7, 4], [2, 7]])
    kw = O.nystrom_weights(2, n, om, n)
    A = O.dense_ls_matrix(n, om, m, kw)
    u = np.linalg.solve(A, O.ls_rhs(m, om, kw, dirs[0]).reshape(-1)).reshape(n, n)
    data = u[tuple(rcv.T)][None]
    assert np.abs(O.misfit_gradient_dense(n, om, m, dirs, rcv, data)).max() <= 1e-12
