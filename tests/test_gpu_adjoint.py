"""Adjoint solve and medium gradient through the C ABI, against the oracle and
against finite differences.

P^T (transposed sweep, reversed order, transposed slab solves) is compared
with the oracle's Q^T Sweep^T E^T element by element (1e-10, the same bound as
P itself) and checked to be the bilinear adjoint of the GPU's own P.  The
adjoint solve A^T mu = rhs is compared with the oracle's right-preconditioned
GMRES on the transposed system (1e-10 at relres 1e-13, iterations +-1 at 1e-8).
The gradient of a receiver misfit through torch.autograd (backward = adjoint
solve + lss_medium_gradient) is checked against central differences of the
misfit with step 1e-6 on m: O(step^2) truncation plus solve tolerance 1e-13
amplified by 1/step, so relative agreement 1e-5.
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


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


def make(n, freq, seed, b_pml=12, b_slab=4, precision=0, gauss=(4, 0.08, (0.8, 1.2))):
    from paper_1705_09443_gb300 import LSSolver
    om = 2 * math.pi * freq
    m = synth.gaussian_medium(n, 2, gauss[0], gauss[1], gauss[2], seed)
    s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=b_pml, b_slab=b_slab,
                 precision=precision)
    return s, m, om


@pytest.fixture(scope="module")
def n64():
    s, m, om = make(64, 8.0, 1706)
    pb = O.Problem2D(64, om, m, O.Params(b_pml=12, b_slab=4))
    return s, m, om, pb


def test_transposed_preconditioner_matches_oracle(n64):
    s, m, om, pb = n64
    y = crand((2, 64, 64), 11)
    x = s.apply_P(to_dev(y), transpose=True).cpu().numpy()
    for r in range(2):
        assert rel(x[r], pb.precondition_transpose(y[r])) <= 1e-10


def test_transposed_preconditioner_is_bilinear_adjoint(n64):
    s, m, om, pb = n64
    x = crand((1, 64, 64), 12)
    y = crand((1, 64, 64), 13)
    px = s.apply_P(to_dev(x)).cpu().numpy()
    pty = s.apply_P(to_dev(y), transpose=True).cpu().numpy()
    lhs, rhs = np.sum(px * y), np.sum(x * pty)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_solve_matches_oracle(n64):
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om, pb = n64
    rhs = crand((64, 64), 14)
    A_T = lambda v: O.ls_apply_transpose(v, m, om, pb.kw)   # noqa: E731
    mu, st = s.adjoint_solve(to_dev(rhs[None]), GmresOptions(30, 1e-13, 200))
    ref = O.gmres(A_T, pb.precondition_transpose, rhs, 30, 1e-13, 200)
    assert st[0]["converged"] and st[0]["relres_true"] <= 1e-12
    assert rel(mu[0].cpu().numpy(), ref.x) <= 1e-10
    _, st8 = s.adjoint_solve(to_dev(rhs[None]), GmresOptions(30, 1e-8, 200))
    ref8 = O.gmres(A_T, pb.precondition_transpose, rhs, 30, 1e-8, 200)
    assert abs(st8[0]["iters"] - ref8.iters) <= 1
    assert st8[0]["relres_true"] <= 1e-8


def test_adjoint_solve_residual_of_the_transposed_operator(n64):
    """Independent of the oracle: A^T mu reproduces rhs with the GPU's own A^T."""
    from paper_1705_09443_gb300 import GmresOptions
    s, m, om, pb = n64
    rhs = to_dev(crand((3, 64, 64), 15))
    mu, st = s.adjoint_solve(rhs, GmresOptions(30, 1e-10, 300))
    back = s.apply_A(mu, transpose=True)
    for r in range(3):
        assert rel(back[r].cpu().numpy(), rhs[r].cpu().numpy()) <= 1e-9


def test_mixed_adjoint_converges_within_two_iterations(n64):
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    s64, m, om, pb = n64
    s32, _, _ = make(64, 8.0, 1706, precision=LSS_MIXED)
    rhs = to_dev(crand((1, 64, 64), 16))
    _, st64 = s64.adjoint_solve(rhs, GmresOptions(30, 1e-8, 200))
    _, st32 = s32.adjoint_solve(rhs, GmresOptions(30, 1e-8, 200))
    assert st32[0]["relres_true"] <= 1e-8
    assert st32[0]["iters"] <= st64[0]["iters"] + 2


def test_transposed_preconditioner_ragged_one_and_two_slabs():
    for bs in (20, 6):
        s, m, om = make(9, 2.0, 5, b_pml=3, b_slab=bs, gauss=(3, 0.15, (0.8, 1.2)))
        pb = O.Problem2D(9, om, m, O.Params(b_pml=3, b_slab=bs))
        assert s.n_slabs == pb.n_slabs
        y = crand((9, 9), 17 + bs)
        x = s.apply_P(to_dev(y[None]), transpose=True).cpu().numpy()[0]
        assert rel(x, pb.precondition_transpose(y)) <= 1e-10


def test_gradient_matches_central_differences():
    """Misfit 0.5 sum |u(receivers) - d|^2 over two plane waves, receivers on a
    ring of grid points; dL/dm through autograd against central differences."""
    from paper_1705_09443_gb300 import GmresOptions, LSSolver, ls_solve
    n = 32
    om = 2 * math.pi * 4.0
    m = synth.gaussian_medium(n, 2, 3, 0.1, (0.85, 1.15), 21)
    th = np.array([0.3, 2.1])
    dirs = np.stack([np.cos(th), np.sin(th)], 1)
    ang = 2 * np.pi * np.arange(24) / 24
    rr = np.clip(np.round(15.5 + 12 * np.cos(ang)).astype(int), 0, n - 1)
    cc = np.clip(np.round(15.5 + 12 * np.sin(ang)).astype(int), 0, n - 1)
    rows, cols = torch.tensor(rr, device="cuda"), torch.tensor(cc, device="cuda")
    d = to_dev(crand((2, 24), 22) * 1e-2)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    s = LSSolver(n, om, mt, b_pml=8, b_slab=4)
    opts = GmresOptions(30, 1e-13, 300)

    def loss(u):
        return 0.5 * (u[:, rows, cols] - d).abs().pow(2).sum()

    mg = mt.clone().requires_grad_(True)
    L0 = loss(ls_solve(mg, s, dirs, opts))
    L0.backward()
    grad = mg.grad.cpu().numpy()
    rng = np.random.default_rng(23)
    pts = [(int(a), int(b)) for a, b in zip(rng.integers(4, n - 4, 6), rng.integers(4, n - 4, 6))]
    step = 1e-6
    for (a, b) in pts:
        vals = []
        for sgn in (1, -1):
            mp = mt.clone()
            mp[a, b] += sgn * step
            with torch.no_grad():
                vals.append(float(loss(ls_solve(mp, s, dirs, opts))))
        fd = (vals[0] - vals[1]) / (2 * step)
        assert abs(grad[a, b] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max()), (a, b, grad[a, b], fd)


def test_gradient_matches_oracle_dense_adjoint():
    """dL/dm through autograd (adjoint solve + lss_medium_gradient) against the
    oracle's dense-adjoint gradient of the same receiver misfit (n = 14, two
    plane waves, eight receivers; dense solves on the oracle side)."""
    from paper_1705_09443_gb300 import GmresOptions, LSSolver, ls_solve
    n = 14
    om = 2 * math.pi * 2.0
    m = synth.gaussian_medium(n, 2, 3, 0.12, (0.85, 1.15), 31)
    dirs = np.array([[1.0, 0.0], [0.6, 0.8]])
    rng = np.random.default_rng(32)
    rcv = rng.integers(0, n, size=(8, 2))
    data = (rng.standard_normal((2, 8)) + 1j * rng.standard_normal((2, 8))) * 1e-2
    ref = O.misfit_gradient_dense(n, om, m, dirs, rcv, data)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    s = LSSolver(n, om, mt, b_pml=4, b_slab=3)
    rows = torch.tensor(rcv[:, 0], device="cuda")
    cols = torch.tensor(rcv[:, 1], device="cuda")
    d = to_dev(data)
    mg = mt.clone().requires_grad_(True)
    u = ls_solve(mg, s, dirs, GmresOptions(30, 1e-13, 300))
    (0.5 * (u[:, rows, cols] - d).abs().pow(2).sum()).backward()
    assert rel(mg.grad.cpu().numpy(), ref) <= 1e-8


def test_gradient_recomputed_forward_and_interleaved_media():
    """The backward recomputes the forward fields when they exceed the memory
    cap (here 0 bytes) and refactors when another medium was set in between:
    both give the gradient of the plain path bit for bit."""
    from paper_1705_09443_gb300 import GmresOptions, LSSolver, ls_solve
    n = 24
    om = 2 * math.pi * 3.0
    m1 = torch.tensor(synth.gaussian_medium(n, 2, 3, 0.1, (0.85, 1.15), 41), dtype=torch.float64, device="cuda")
    m2 = torch.tensor(synth.gaussian_medium(n, 2, 3, 0.1, (0.85, 1.15), 42), dtype=torch.float64, device="cuda")
    dirs = np.array([[1.0, 0.0], [0.0, 1.0]])
    s = LSSolver(n, om, m1, b_pml=6, b_slab=4)
    opts = GmresOptions(30, 1e-12, 300)

    def grad(m, cap=None, other=None):
        mg = m.clone().requires_grad_(True)
        u = ls_solve(mg, s, dirs, opts, memory_cap=cap)
        if other is not None:   # a forward with another medium before this backward
            with torch.no_grad():
                ls_solve(other, s, dirs, opts)
        u.abs().pow(2).sum().backward()
        return mg.grad
    g0 = grad(m1)
    assert torch.equal(grad(m1, cap=0), g0)
    assert torch.equal(grad(m1, other=m2), g0)
