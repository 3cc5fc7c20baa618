"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances: the LS operator and right-hand sides are FFT convolutions in FP64
(rounding ~1e-15 * log L): 1e-12 relative.  The slab operators and the
preconditioner go through block LU of subproblems whose condition numbers are
at most ~1e4 here: 1e-10 relative.  Solutions: 1e-10 when both sides solve to
relres 1e-13; iteration counts at tol 1e-8 agree within 1.
"""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(n, freq, medium_seed=3, b_pml=12, b_slab=4, precision=0, gauss=(4, 0.08, (0.8, 1.2))):
    from paper_1705_09443_gb300 import LSSolver
    om = 2 * math.pi * freq
    if medium_seed is None:
        m = np.zeros((n, n))
    else:
        m = synth.gaussian_medium(n, 2, gauss[0], gauss[1], gauss[2], medium_seed)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    s = LSSolver(n, om, mt, b_pml=b_pml, b_slab=b_slab, precision=precision)
    return s, m, om


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


@pytest.fixture(scope="module")
def n64():
    s, m, om = make(64, 8.0, medium_seed=1706)
    pb = O.Problem2D(64, om, m, O.Params(b_pml=12, b_slab=4))
    return s, m, om, pb


@pytest.mark.parametrize("n,L_expected", [(13, 32), (64, 128), (100, 256)])
def test_ls_operator_matches_oracle(n, L_expected):
    s, m, om = make(n, (n + 1) / 8, b_pml=4)
    assert s.fft_len == L_expected
    kw = O.nystrom_weights(2, n, om, n)
    x = crand((3, n, n), n)
    y = s.apply_A(to_dev(x)).cpu().numpy()
    yt = s.apply_A(to_dev(x), transpose=True).cpu().numpy()
    for r in range(3):
        assert rel(y[r], O.ls_apply(x[r], m, om, kw)) <= 1e-12
        assert rel(yt[r], O.ls_apply_transpose(x[r], m, om, kw)) <= 1e-12


def test_plane_wave_rhs_matches_oracle(n64):
    s, m, om, pb = n64
    dirs = np.array([[1.0, 0.0], [math.cos(1.1), math.sin(1.1)]])
    g, uI = s.plane_wave_rhs(dirs, with_incident=True)
    for r in range(2):
        assert rel(uI[r].cpu().numpy(), O.plane_wave(64, om, dirs[r])) <= 1e-13
        assert rel(g[r].cpu().numpy(), O.ls_rhs(m, om, pb.kw, dirs[r])) <= 1e-12


def test_interior_stencils_match_oracle(n64):
    s, m, om, pb = n64
    a, b = s.stencils()
    assert rel(a, pb.alpha) <= 1e-9
    assert rel(b, pb.beta) <= 1e-9


def test_slab_layout_matches_oracle(n64):
    s, m, om, pb = n64
    assert s.n_slabs == pb.n_slabs and s.n_tot == pb.n_tot
    for i in range(pb.n_slabs):
        first, nl, na = s.slab_info(i)
        assert first == pb.slab_first[i] and nl == pb.slab_last[i] - pb.slab_first[i] + 1
        assert na == (0 if i == 0 else pb.b_aux)


@pytest.mark.parametrize("i", [0, 1, 8, 15, 16])
def test_slab_operator_matches_oracle(n64, i):
    """T~_i (Eq. Hwv_approx) with the stored block-LU factors vs the oracle's sparse LU."""
    s, m, om, pb = n64
    nl = pb.slab_last[i] - pb.slab_first[i] + 1
    v = crand((2, nl, pb.n_tot), 100 + i)
    w = s.apply_slab(i, to_dev(v)).cpu().numpy()
    for r in range(2):
        assert rel(w[r], pb.T(i, v[r])) <= 1e-10


def test_preconditioner_matches_oracle(n64):
    s, m, om, pb = n64
    x = crand((2, 64, 64), 7)
    y = s.apply_P(to_dev(x)).cpu().numpy()
    for r in range(2):
        assert rel(y[r], pb.precondition(x[r])) <= 1e-10


def test_solution_matches_oracle(n64):
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om, pb = n64
    d = (1.0, 0.0)
    g = s.plane_wave_rhs([d])
    u, st = s.solve(g, GmresOptions(30, 1e-13, 200))
    ref, relres, _, _ = O.solve(64, om, m, d, tol=1e-13, problem=pb)
    assert st[0]["converged"] and st[0]["relres_true"] <= 1e-12
    assert rel(u[0].cpu().numpy(), ref.x) <= 1e-10
    u8, st8 = s.solve(g, GmresOptions(30, 1e-8, 200))
    ref8, _, _, _ = O.solve(64, om, m, d, tol=1e-8, problem=pb)
    assert abs(st8[0]["iters"] - ref8.iters) <= 1
    assert st8[0]["relres_true"] <= 1e-8


def test_mixed_precision_converges_within_two_iterations(n64):
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    s64, m, om, pb = n64
    s32, _, _ = make(64, 8.0, medium_seed=1706, precision=LSS_MIXED)
    g = s64.plane_wave_rhs([(1.0, 0.0)])
    _, st64 = s64.solve(g, GmresOptions(30, 1e-8, 200))
    u32, st32 = s32.solve(g, GmresOptions(30, 1e-8, 200))
    assert st32[0]["relres_true"] <= 1e-8
    assert st32[0]["iters"] <= st64[0]["iters"] + 2
    # mixed sweep stays close to the FP64 one
    x = crand((1, 64, 64), 9)
    assert rel(s32.apply_P(to_dev(x)).cpu().numpy(), s64.apply_P(to_dev(x)).cpu().numpy()) <= 1e-4


def test_batched_rhs_equal_single_rhs_solves(n64):
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om, pb = n64
    th = np.array([0.0, 0.7, 2.0, 4.0, 5.5])
    dirs = np.stack([np.cos(th), np.sin(th)], 1)
    g = s.plane_wave_rhs(dirs)
    u, st = s.solve(g, GmresOptions(30, 1e-12, 300))
    for r in (0, 3):
        u1, st1 = s.solve(g[r:r + 1].clone(), GmresOptions(30, 1e-12, 300))
        assert rel(u[r].cpu().numpy(), u1[0].cpu().numpy()) <= 1e-10
        assert st[r]["iters"] == st1[0]["iters"]


# ---------------------------------------------------------------- edge cases

def test_ragged_small_grid_one_and_two_slabs():
    """n = 9 (ragged tiles), b = 3: a single slab holding both PMLs (exact
    H^{-1}, T~_1 = T_1) and a two-slab split."""
    for bs in (20, 6):
        s, m, om = make(9, 2.0, medium_seed=5, b_pml=3, b_slab=bs, gauss=(3, 0.15, (0.8, 1.2)))
        pb = O.Problem2D(9, om, m, O.Params(b_pml=3, b_slab=bs))
        assert s.n_slabs == pb.n_slabs == (1 if bs == 20 else 2)
        x = crand((1, 9, 9), 11)
        assert rel(s.apply_P(to_dev(x)).cpu().numpy()[0], pb.precondition(x[0])) <= 1e-10


def test_mixed_precision_odd_total_width():
    """n_tot = n + 2 + 2b odd (51 and 17): interface-map rows of odd length in
    single precision, so the recurrence's map rows start on 8-byte
    boundaries; the mixed sweep must still match the oracle to 1e-4 and the
    mixed solve converge within two iterations of FP64."""
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    for n, freq, b in ((37, 4.625, 6), (9, 2.0, 3)):
        s32, m, om = make(n, freq, medium_seed=5, b_pml=b, precision=LSS_MIXED, gauss=(3, 0.15, (0.8, 1.2)))
        s64, _, _ = make(n, freq, medium_seed=5, b_pml=b, gauss=(3, 0.15, (0.8, 1.2)))
        assert s32.n_tot % 2 == 1
        pb = O.Problem2D(n, om, m, O.Params(b_pml=b, b_slab=4))
        x = crand((1, n, n), 12)
        assert rel(s32.apply_P(to_dev(x)).cpu().numpy()[0], pb.precondition(x[0])) <= 1e-4
        assert rel(s32.apply_P(to_dev(x), transpose=True).cpu().numpy()[0], pb.precondition_transpose(x[0])) <= 1e-4
        g = s64.plane_wave_rhs([(0.6, 0.8)])
        _, st64 = s64.solve(g, GmresOptions(30, 1e-8, 200))
        _, st32 = s32.solve(g, GmresOptions(30, 1e-8, 200))
        assert st32[0]["relres_true"] <= 1e-8 and st32[0]["iters"] <= st64[0]["iters"] + 2


def test_three_runs_of_block_widths():
    """b_pml = 14, b_aux = 10, b_slab = 4: the first slab has 18 layers (32-wide
    blocks), the middle slabs 14 (16-wide), the last one 10 + 14 + a remainder
    (32-wide), so the factorization and both sweep passes run three launches on
    three streams.  FP64 and mixed preconditioners against the oracle, the
    transposed one too, and the FP64 solve."""
    from paper_1705_09443_gb300 import GmresOptions, LSSolver, LSS_MIXED
    n, freq = 40, 5.0
    om = 2 * math.pi * freq
    m = synth.gaussian_medium(n, 2, 4, 0.1, (0.8, 1.2), 77)
    pb = O.Problem2D(n, om, m, O.Params(b_pml=14, b_slab=4, b_aux=10))
    widths = [pb.n_aux[i] + pb.slab_last[i] - pb.slab_first[i] + 1 for i in range(pb.n_slabs)]
    assert widths[0] > 16 and widths[1] <= 16 and widths[-1] > 16
    x = crand((1, n, n), 13)
    for prec, tol in ((0, 1e-10), (LSS_MIXED, 1e-4)):
        s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=14, b_slab=4, b_aux=10,
                     precision=prec)
        assert rel(s.apply_P(to_dev(x)).cpu().numpy()[0], pb.precondition(x[0])) <= tol
        assert rel(s.apply_P(to_dev(x), transpose=True).cpu().numpy()[0], pb.precondition_transpose(x[0])) <= tol
        if prec == 0:
            g = s.plane_wave_rhs([(0.6, 0.8)])
            u, st = s.solve(g, GmresOptions(30, 1e-12, 200))
            ref, _, _, _ = O.solve(n, om, m, (0.6, 0.8), tol=1e-12, problem=pb)
            assert rel(u[0].cpu().numpy(), ref.x) <= 1e-10


def test_zero_medium_gives_zero_solution():
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om = make(16, 2.0, medium_seed=None, b_pml=4)
    g = s.plane_wave_rhs([(1.0, 0.0)])
    assert torch.count_nonzero(g).item() == 0
    u, st = s.solve(g, GmresOptions())
    assert torch.count_nonzero(u).item() == 0 and st[0]["iters"] == 0


def test_error_codes():
    from paper_1705_09443_gb300 import LSSolver, LssError
    m = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    s = LSSolver(16, 10.0, m, b_pml=4, factor=False)
    x = torch.zeros((1, 16, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(LssError) as e:
        s.apply_P(x)
    assert e.value.code == -3
    with pytest.raises(LssError) as e:
        LSSolver(16, 10.0, m, b_pml=16, b_slab=4)     # last slab 16 + 2 + 16 > 32 layers
    assert e.value.code == -8
    bad = m.clone()
    bad[3, 3] = float("nan")
    with pytest.raises(LssError) as e:
        LSSolver(16, 10.0, bad, b_pml=4)
    assert e.value.code == -1
