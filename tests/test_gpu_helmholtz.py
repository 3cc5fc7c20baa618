"""The sparsifying scheme as a direct Helmholtz solver (Sec. 4) through the C
ABI (lss_helmholtz_solve): FGMRES on the sparsified system H u = beta^* f
preconditioned by the moving-PML sweep, against the oracle's sparse-LU solve of
the same system (1e-9), against the Green's function for a delta source at
8 points per wavelength, with the paper's order of phase error at 3 points
per wavelength, and in a heterogeneous medium."""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


def solver(n, freq, m, precision=0, b_pml=12, b_slab=4):
    from paper_1705_09443_gb300 import LSSolver
    return LSSolver(n, 2 * math.pi * freq, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=b_pml,
                    b_slab=b_slab, precision=precision)


def greens(n, freq, c):
    h = 1.0 / (n + 1)
    xs = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    r = np.hypot(X - c * h, Y - c * h)
    G = np.zeros((n, n), complex)
    G[r > 0] = O.green(2, 2 * math.pi * freq, r[r > 0])
    return G, (r > 0.1) & (r < 0.4)


def test_delta_source_matches_oracle_and_greens_function():
    from paper_1705_09443_gb300 import GmresOptions
    n, freq = 63, 8.0
    m = np.zeros((n, n))
    s = solver(n, freq, m)
    c = (n + 1) // 2
    f = O.delta_source(n, (c, c))
    u, st = s.helmholtz_solve(to_dev(f), GmresOptions(30, 1e-12, 300))
    assert st[0]["converged"] and st[0]["relres_true"] <= 1e-11
    u = u[0].cpu().numpy()
    pb = O.Problem2D(n, 2 * math.pi * freq, m, O.Params(b_pml=12, b_slab=4))
    ref, _ = O.helmholtz_direct(pb, f)
    assert rel(u, ref) <= 1e-9
    G, ann = greens(n, freq, c)
    assert np.linalg.norm((u - G)[ann]) <= 5e-3 * np.linalg.norm(G[ann])


def test_phase_error_at_3_points_per_wavelength():
    from paper_1705_09443_gb300 import GmresOptions
    n, freq = 95, 32.0
    s = solver(n, freq, np.zeros((n, n)))
    c = (n + 1) // 2
    u, st = s.helmholtz_solve(to_dev(O.delta_source(n, (c, c))), GmresOptions(30, 1e-10, 300))
    G, ann = greens(n, freq, c)
    u = u[0].cpu().numpy()
    drift = np.abs(np.angle(u[ann] / G[ann])).max() / (2 * math.pi) / (0.4 * freq)
    assert drift <= 5e-4


def test_heterogeneous_medium_matches_oracle_and_mixed_converges():
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    n, freq = 64, 8.0
    m = synth.gaussian_medium(n, 2, 4, 0.08, (0.8, 1.2), 1706)
    rng = np.random.default_rng(70)
    f = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    s = solver(n, freq, m)
    u, st = s.helmholtz_solve(to_dev(f), GmresOptions(30, 1e-12, 300))
    pb = O.Problem2D(n, 2 * math.pi * freq, m, O.Params(b_pml=12, b_slab=4))
    for r in range(2):
        ref, _ = O.helmholtz_direct(pb, f[r])
        assert rel(u[r].cpu().numpy(), ref) <= 1e-9
    _, st64 = s.helmholtz_solve(to_dev(f), GmresOptions(30, 1e-8, 300))
    s32 = solver(n, freq, m, precision=LSS_MIXED)
    u32, st32 = s32.helmholtz_solve(to_dev(f), GmresOptions(30, 1e-8, 300))
    for r in range(2):
        assert st32[r]["relres_true"] <= 1e-8
        assert st32[r]["iters"] <= st64[r]["iters"] + 2
