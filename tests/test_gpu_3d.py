"""3D path (Sec. 3.1) through the C ABI against the FP64 oracle.

Small grids with several slabs and a ragged last slab: interior stencils, the
LS operator, the right-hand side, every slab operator T~_i, the preconditioner
P and the FGMRES solution in FP64 (1e-12 for the operator and right-hand
side, 1e-10 for T~_i, P and the solution; iteration counts +-1), the mixed
form (FP32 slab factors and sweep) within +2 iterations at relres 1e-8.  The
3D workload itself (n = 64, omega/2pi = 16, 8 Gaussians, direction
(1,1,1)/sqrt3, PML 8, slabs of 4 layers) is solved in mixed precision and in
FP64 and its residual is measured with the oracle's operator.
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


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


D3 = np.ones(3) / math.sqrt(3.0)


def case(n, b, bs, seed=9, precision=0, freq=None, gauss=True):
    from paper_1705_09443_gb300 import LSSolver
    freq = freq if freq is not None else (n + 1) / 8
    om = 2 * math.pi * freq
    m = synth.gaussian_medium(n, 3, 3, 0.15, (0.8, 1.2), seed) if gauss else np.zeros((n, n, n))
    s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=b, b_slab=bs,
                 precision=precision)
    return s, m, om


@pytest.fixture(scope="module")
def n8():
    s, m, om = case(8, 3, 3)
    pb = O.Problem3D(8, om, m, O.Params(b_pml=3, b_slab=3))
    return s, m, om, pb


def test_slab_layout_matches_oracle(n8):
    s, m, om, pb = n8
    assert s.dim == 3 and s.n_tot == pb.n_tot and s.n_slabs == pb.n_slabs
    for i in range(pb.n_slabs):
        first, nl, na = s.slab_info(i)
        assert first == pb.slab_first[i] and first + nl - 1 == pb.slab_last[i] and na == pb.n_aux[i]


def test_interior_stencils_match_oracle(n8):
    s, m, om, pb = n8
    a, b = s.stencils()
    assert rel(a, pb.alpha) <= 1e-9
    assert rel(b, pb.beta) <= 1e-9


@pytest.mark.parametrize("n", [7, 12])
def test_operator_matches_oracle(n):
    s, m, om = case(n, 3, 3, seed=n)
    kw = O.nystrom_weights(3, n, om, n)
    x = crand((2, n, n, n), n)
    y = s.apply_A(to_dev(x)).cpu().numpy()
    for r in range(2):
        assert rel(y[r], O.ls_apply(x[r], m, om, kw)) <= 1e-12
    yt = s.apply_A(to_dev(x), transpose=True).cpu().numpy()
    assert rel(yt[0], O.ls_apply_transpose(x[0], m, om, kw)) <= 1e-12


def test_plane_wave_rhs_matches_oracle(n8):
    s, m, om, pb = n8
    dirs = np.stack([D3, np.array([0.0, 0.6, 0.8])])
    g = s.plane_wave_rhs(dirs).cpu().numpy()
    for r in range(2):
        assert rel(g[r], O.ls_rhs(m, om, pb.kw, dirs[r])) <= 1e-12


def test_slab_operators_match_oracle(n8):
    s, m, om, pb = n8
    for i in range(pb.n_slabs):
        nl = pb.slab_last[i] - pb.slab_first[i] + 1
        v = crand((nl, pb.n_tot, pb.n_tot), 100 + i)
        w = s.apply_slab(i, to_dev(v[None])).cpu().numpy()[0]
        assert rel(w, pb.T(i, v)) <= 1e-10, i


def test_preconditioner_matches_oracle(n8):
    s, m, om, pb = n8
    x = crand((2, 8, 8, 8), 7)
    y = s.apply_P(to_dev(x)).cpu().numpy()
    for r in range(2):
        assert rel(y[r], pb.precondition(x[r])) <= 1e-10


@pytest.mark.parametrize("n,b,bs", [(7, 2, 3), (6, 2, 20), (9, 4, 2)])
def test_preconditioner_ragged_and_one_slab(n, b, bs):
    s, m, om = case(n, b, bs, seed=3 + n)
    pb = O.Problem3D(n, om, m, O.Params(b_pml=b, b_slab=bs))
    assert s.n_slabs == pb.n_slabs
    x = crand((n, n, n), 8 + n)
    assert rel(s.apply_P(to_dev(x[None])).cpu().numpy()[0], pb.precondition(x)) <= 1e-10


def test_solution_matches_oracle_fp64(n8):
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om, pb = n8
    g = s.plane_wave_rhs(D3[None])
    u, st = s.solve(g, GmresOptions(30, 1e-13, 200))
    ref, relres, _, _ = O.solve(8, om, m, D3, problem=pb, tol=1e-13)
    assert st[0]["converged"] and st[0]["relres_true"] <= 1e-12
    assert rel(u[0].cpu().numpy(), ref.x) <= 1e-10
    _, st8 = s.solve(g, GmresOptions(30, 1e-8, 200))
    ref8, _, _, _ = O.solve(8, om, m, D3, problem=pb, tol=1e-8)
    assert abs(st8[0]["iters"] - ref8.iters) <= 1


def test_mixed_factorization_paths_agree(n8, monkeypatch):
    """The mixed 3D factorization on the tensor cores (3xTF32 rank-64 updates,
    the default) and on CUDA cores (FP32 rank-16 updates) give the same P to
    single-precision accuracy, both close to the oracle's FP64 P."""
    s64, m, om, pb = n8
    x = crand((8, 8, 8), 23)
    ref = pb.precondition(x)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("LSS_TC_UPDATE", flag)
        from paper_1705_09443_gb300 import LSS_MIXED
        s32, _, _ = case(8, 3, 3, precision=LSS_MIXED)
        out.append(s32.apply_P(to_dev(x[None])).cpu().numpy()[0])
    assert rel(out[0], out[1]) <= 1e-5
    assert rel(out[0], ref) <= 1e-4 and rel(out[1], ref) <= 1e-4


def test_mixed_precision_within_two_iterations(n8):
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    s64, m, om, pb = n8
    s32, _, _ = case(8, 3, 3, precision=LSS_MIXED)
    x = crand((8, 8, 8), 21)
    assert rel(s32.apply_P(to_dev(x[None])).cpu().numpy()[0], pb.precondition(x)) <= 1e-4
    g = s64.plane_wave_rhs(D3[None])
    _, st64 = s64.solve(g, GmresOptions(30, 1e-8, 200))
    u32, st32 = s32.solve(g, GmresOptions(30, 1e-8, 200))
    r = g[0].cpu().numpy() - O.ls_apply(u32[0].cpu().numpy(), m, om, pb.kw)
    assert np.linalg.norm(r) / np.linalg.norm(g[0].cpu().numpy()) <= 1e-8 * (1 + 1e-6)
    assert st32[0]["iters"] <= st64[0]["iters"] + 2


def test_zero_medium_gives_zero_field():
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om = case(6, 2, 3, gauss=False)
    g = s.plane_wave_rhs(D3[None])
    assert float(g.abs().max()) == 0.0
    u, st = s.solve(g, GmresOptions(30, 1e-8, 50))
    assert float(u.abs().max()) == 0.0 and st[0]["iters"] == 0


@pytest.mark.parametrize("precision", [1, 0])
def test_full_size_3d_workload(precision):
    """n = 64, omega/2pi = 16: relres <= 1e-8 measured with the oracle's operator;
    mixed within +2 iterations of FP64 (both are run, FP64 second)."""
    from paper_1705_09443_gb300 import GmresOptions, LSSolver
    w = synth.WORKLOADS["3d_n64"]
    m, dirs = synth.make_workload(w)
    s = LSSolver(w.n, w.omega, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=w.b_pml,
                 b_slab=w.b_slab, precision=precision)
    assert s.n_tot == 82 and s.n_slabs == 17
    g = s.plane_wave_rhs(dirs)
    u, st = s.solve(g, GmresOptions(30, 1e-8, 200))
    kw = O.nystrom_weights(3, w.n, w.omega, w.n)
    g_ref = O.ls_rhs(m, w.omega, kw, dirs[0])
    assert rel(g[0].cpu().numpy(), g_ref) <= 1e-12
    res = g_ref - O.ls_apply(u[0].cpu().numpy(), m, w.omega, kw)
    assert np.linalg.norm(res) / np.linalg.norm(g_ref) <= 1e-8 * (1 + 1e-6)
    assert st[0]["converged"] and st[0]["iters"] <= 12
