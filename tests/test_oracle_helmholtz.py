"""Pins of the oracle's Sec. 4 direct solver (the sparsified system
alpha^* u_{mu_i} = beta^* f_{mu_i} with PML rows, a delta source) against the
mathematics: the exact solution of (-Laplace - omega^2) u = delta(x - x0) is
the Green's function G(x - x0) (Sec. 1); the Nystrom solution K f satisfies
the local equations up to the far-field truncation sigma_min ||f||; the phase
error at 3 points per wavelength is of the order the paper reports (about
2.3e-4 of a wavelength per wavelength, Sec. 4)."""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O


def solve_delta(n, freq, b_pml=12):
    om = 2 * math.pi * freq
    pb = O.Problem2D(n, om, np.zeros((n, n)), O.Params(b_pml=b_pml, b_slab=n + 2))
    c = (n + 1) // 2
    u, _ = O.helmholtz_direct(pb, O.delta_source(n, (c, c)))
    h = 1.0 / (n + 1)
    xs = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    r = np.hypot(X - c * h, Y - c * h)
    G = np.zeros_like(u)
    G[r > 0] = O.green(2, om, r[r > 0])
    ann = (r > 0.1) & (r < 0.4)
    return pb, u, G, ann, om


def test_direct_solution_is_the_greens_function_at_8_ppw():
    pb, u, G, ann, om = solve_delta(63, 8.0)
    assert np.linalg.norm((u - G)[ann]) <= 5e-3 * np.linalg.norm(G[ann])
    assert np.abs(np.angle(u[ann] / G[ann])).max() <= 1e-2


def test_phase_error_per_wavelength_at_3_ppw():
    """3 points per wavelength, omega/2pi = 32: the phase drift over the
    annulus (up to 0.4 * 32 = 12.8 wavelengths) per wavelength is ~2e-4."""
    pb, u, G, ann, om = solve_delta(95, 32.0)
    drift = np.abs(np.angle(u[ann] / G[ann])).max() / (2 * math.pi) / (0.4 * 32.0)
    assert drift <= 5e-4


def test_error_falls_with_points_per_wavelength():
    errs = []
    for n in (47, 95):                      # 3 and 6 points per wavelength at omega/2pi = 16
        pb, u, G, ann, om = solve_delta(n, 16.0)
        errs.append(np.linalg.norm((u - G)[ann]) / np.linalg.norm(G[ann]))
    assert errs[1] < errs[0] / 2


def test_nystrom_solution_satisfies_the_local_equations():
    """u* = K f (the discrete convolution, = G at the grid points for a delta
    of mass 1) satisfies alpha^* u*_{mu_i} = beta^* f_{mu_i} + far part, the
    far part at most sigma_min ||f|| (Eq. beta); a conjugation slip in the
    right-hand side breaks this by orders of magnitude."""
    n = 31
    om = 2 * math.pi * 4.0
    pb = O.Problem2D(n, om, np.zeros((n, n)), O.Params(b_pml=6, b_slab=n + 2))
    c = (n + 1) // 2
    f = O.delta_source(n, (c, c))
    kw = O.nystrom_weights(2, n, om, n)
    ustar = O.ls_apply(f, np.ones((n, n)), om, kw) - f          # omega^2 K f
    ustar = ustar / om ** 2
    F = O.helmholtz_rhs(pb, f)
    b = pb.b
    bound = pb.sv[-1] * np.linalg.norm(f)
    worst = 0.0
    for i1 in range(2, n):
        for i2 in range(2, n):
            U = ustar[i1 - 2:i1 + 1, i2 - 2:i2 + 1].reshape(-1)
            worst = max(worst, abs(np.vdot(pb.alpha, U) - F[i1 + b, i2 + b]))
    assert worst <= bound * (1 + 1e-9)
    # planted slips in the right-hand side break the bound: beta instead of
    # conj(beta) (beta is nearly real here: 20x), a stray h^2 (300x)
    fp = np.zeros((n + 4, n + 4), complex)
    fp[2:n + 2, 2:n + 2] = f
    for st, factor in ((pb.beta.reshape(3, 3), 10), (np.conj(pb.beta).reshape(3, 3) / (n + 1) ** 2, 100)):
        Fw = np.zeros((pb.n_tot, pb.n_tot), complex)
        for da in (-1, 0, 1):
            for db in (-1, 0, 1):
                Fw[b:b + n + 2, b:b + n + 2] += st[da + 1, db + 1] * fp[1 + da:n + 3 + da, 1 + db:n + 3 + db]
        worst_w = max(abs(np.vdot(pb.alpha, ustar[i1 - 2:i1 + 1, i2 - 2:i2 + 1].reshape(-1)) - Fw[i1 + b, i2 + b])
                      for i1 in range(2, n) for i2 in range(2, n))
        assert worst_w > factor * bound
