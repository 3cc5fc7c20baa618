"""Ragged instances behind one context (lss_setup_batch), through the C ABI.

Instances of different n and omega (omega/2pi = n/8, band-limited media) are
solved together.  Two drivers: the default lockstep one (every instance's
right-hand sides are segments of one set of Krylov vectors, one host thread
issues every instance's operator and sweep) and the threaded one
(LSS_BATCH_THREADS=1: each instance's own solve on a host thread).  Threaded,
every instance must give what a context of its own gives (same kernels on the
same data: 1e-13, equal iteration counts).  Lockstep, the Krylov inner
products sum the same terms in another order (partial sums per segment), so
FP64 solutions agree to rounding growth (1e-11, iterations within one); in
mixed precision that rounding can move the single-precision sweep's results
by an ulp, and FGMRES then converges on a slightly different path: both
solutions meet relres 1e-8, and they agree to 1e-6.  The operator and
preconditioner must match the oracle (1e-12 / 1e-10 as for single contexts),
and the batch-only error paths must report the failing instance.
"""
import math

import numpy as np
import pytest

from oracle import lss_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = (24, 37, 50)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def make_batch(ns, precision=0, b_pml=6):
    from paper_1705_09443_gb300 import LSSolverBatch
    inst = synth.ragged_instances(ns, 1720)
    ms = [torch.tensor(m, dtype=torch.float64, device="cuda") for _, m, _ in inst]
    oms = [2 * math.pi * f for f, _, _ in inst]
    b = LSSolverBatch(ns, oms, ms, b_pml=b_pml, b_slab=4, precision=precision)
    return b, inst, oms


@pytest.fixture(scope="module")
def batch64():
    return make_batch(NS)


@pytest.fixture
def threaded(monkeypatch):
    monkeypatch.setenv("LSS_BATCH_THREADS", "1")


def test_batch_solve_equals_separate_contexts(batch64, threaded):
    from paper_1705_09443_gb300 import GmresOptions, LSSolver
    b, inst, oms = batch64
    th = np.array([[0.1, 1.3], [2.0, 4.4], [5.0, 0.7]])
    dirs = np.stack([np.cos(th), np.sin(th)], -1)          # (n_inst, R = 2, 2)
    g = b.plane_wave_rhs(dirs)
    u, st = b.solve(g, GmresOptions(30, 1e-10, 300))
    assert len(st) == 3 and all(len(s) == 2 for s in st)
    for q, (n, (f, m, _)) in enumerate(zip(NS, inst)):
        s = LSSolver(n, oms[q], torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=6, b_slab=4)
        g1 = s.plane_wave_rhs(dirs[q])
        assert rel(b.views(g, 2)[q].cpu().numpy(), g1.cpu().numpy()) <= 1e-13
        u1, st1 = s.solve(g1, GmresOptions(30, 1e-10, 300))
        assert rel(b.views(u, 2)[q].cpu().numpy(), u1.cpu().numpy()) <= 1e-13
        for r in range(2):
            assert st[q][r]["iters"] == st1[r]["iters"] and st[q][r]["converged"]


def test_batch_operators_match_oracle(batch64):
    b, inst, oms = batch64
    xs = [crand((1, n, n), 40 + n) for n in NS]
    x = b.pack([torch.tensor(v, dtype=torch.complex128, device="cuda") for v in xs])
    ya = b.views(b.apply_A(x), 1)
    yp = b.views(b.apply_P(x), 1)
    for q, (n, (f, m, _)) in enumerate(zip(NS, inst)):
        pb = O.Problem2D(n, oms[q], m, O.Params(b_pml=6, b_slab=4))
        assert rel(ya[q][0].cpu().numpy(), O.ls_apply(xs[q][0], m, oms[q], pb.kw)) <= 1e-12
        assert rel(yp[q][0].cpu().numpy(), pb.precondition(xs[q][0])) <= 1e-10


def test_batch_mixed_and_adjoint():
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED
    b, inst, oms = make_batch(NS, precision=LSS_MIXED)
    g = b.plane_wave_rhs(np.stack([d for _, _, d in inst]))
    u, st = b.solve(g, GmresOptions(30, 1e-8, 300))
    assert all(s[0]["converged"] and s[0]["relres_true"] <= 1e-8 for s in st)
    rhs = b.pack([torch.tensor(crand((1, n, n), 60 + n), dtype=torch.complex128, device="cuda") for n in NS])
    mu, st_t = b.adjoint_solve(rhs, GmresOptions(30, 1e-10, 300))
    back = b.views(b.apply_A(mu, transpose=True), 1)
    for q in range(3):
        assert st_t[q][0]["converged"]
        assert rel(back[q].cpu().numpy(), b.views(rhs, 1)[q].cpu().numpy()) <= 1e-9


def test_lockstep_equals_threaded(batch64, monkeypatch):
    """FP64, two right-hand sides per instance: the lockstep driver against
    the threaded one on the same batch (rounding-order differences only)."""
    from paper_1705_09443_gb300 import GmresOptions
    b, inst, oms = batch64
    th = np.array([[0.4, 2.1], [1.0, 3.3], [5.5, 0.2]])
    dirs = np.stack([np.cos(th), np.sin(th)], -1)
    g = b.plane_wave_rhs(dirs)
    u, st = b.solve(g, GmresOptions(30, 1e-10, 300))
    monkeypatch.setenv("LSS_BATCH_THREADS", "1")
    u1, st1 = b.solve(g, GmresOptions(30, 1e-10, 300))
    assert rel(u.cpu().numpy(), u1.cpu().numpy()) <= 1e-11
    for q in range(3):
        assert rel(b.views(u, 2)[q].cpu().numpy(), b.views(u1, 2)[q].cpu().numpy()) <= 1e-11
        for r in range(2):
            assert st[q][r]["converged"] and st[q][r]["relres_true"] <= 1e-10 * (1 + 1e-6)
            assert abs(st[q][r]["iters"] - st1[q][r]["iters"]) <= 1


def test_lockstep_graphs_bit_identical(batch64):
    """The lockstep iterations replayed as captured graphs (every instance's
    launches inside one graph per iteration) give the same bits as direct
    launches."""
    from paper_1705_09443_gb300 import GmresOptions
    b, inst, oms = batch64
    dirs = np.stack([d for _, _, d in inst])[:, None]
    g = b.plane_wave_rhs(dirs)
    b.use_graphs(False)
    u0, st0 = b.solve(g, GmresOptions(30, 1e-10, 300))
    b.use_graphs(True)
    for _ in range(3):                      # uncaptured first, then captured and replayed
        u, st = b.solve(g, GmresOptions(30, 1e-10, 300))
        assert torch.equal(u, u0)
        assert [x[0]["iters"] for x in st] == [x[0]["iters"] for x in st0]
    assert b.graph_count()[0] > 0


def test_lockstep_restart_and_unequal_convergence(batch64):
    """Restart length 4 (several restarts) and instances that converge at
    different iterations: the converged segments stop moving while the others
    go on; every right-hand side ends at relres 1e-10 with the oracle's
    operator."""
    from paper_1705_09443_gb300 import GmresOptions
    b, inst, oms = batch64
    dirs = np.stack([d for _, _, d in inst])[:, None]
    g = b.plane_wave_rhs(dirs)
    u, st = b.solve(g, GmresOptions(4, 1e-10, 400))
    its = [s[0]["iters"] for s in st]
    assert len(set(its)) > 1 and max(its) > 8
    for q, (n, (f, m, _)) in enumerate(zip(NS, inst)):
        kw = O.nystrom_weights(2, n, oms[q], n)
        gq = b.views(g, 1)[q][0].cpu().numpy()
        res = gq - O.ls_apply(b.views(u, 1)[q][0].cpu().numpy(), m, oms[q], kw)
        assert st[q][0]["converged"] and np.linalg.norm(res) / np.linalg.norm(gq) <= 1e-10 * (1 + 1e-6)


def test_batch_many_instances_lockstep_mixed():
    """Twelve instances in mixed precision through the lockstep driver, against
    contexts of their own: relres 1e-8 each, iterations within one, solutions
    within 1e-6."""
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED, LSSolver
    ns = synth.ragged_sizes(12, 40, 100, 1722)
    b, inst, oms = make_batch(ns, precision=LSS_MIXED, b_pml=8)
    dirs = np.stack([d for _, _, d in inst])
    b.factor()
    u, st = b.solve(b.plane_wave_rhs(dirs), GmresOptions(30, 1e-8, 100))
    for q, (n, (f, m, d)) in enumerate(zip(ns, inst)):
        s = LSSolver(n, oms[q], torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=8, b_slab=4,
                     precision=LSS_MIXED)
        u1, st1 = s.solve(s.plane_wave_rhs(d), GmresOptions(30, 1e-8, 100))
        assert abs(st[q][0]["iters"] - st1[0]["iters"]) <= 1 and st[q][0]["relres_true"] <= 1e-8
        assert rel(b.views(u, 1)[q].cpu().numpy(), u1.cpu().numpy()) <= 1e-6


def test_batch_many_instances_equal_separate_contexts(threaded):
    """Twelve instances at once in mixed precision (more concurrent streams
    than the small batch), threaded: each instance's iteration count and
    solution equal those of a context of its own."""
    from paper_1705_09443_gb300 import GmresOptions, LSS_MIXED, LSSolver
    ns = synth.ragged_sizes(12, 40, 100, 1721)
    b, inst, oms = make_batch(ns, precision=LSS_MIXED, b_pml=8)
    dirs = np.stack([d for _, _, d in inst])
    for _ in range(2):                      # the first call also uploads the per-context tables
        b.factor()
        u, st = b.solve(b.plane_wave_rhs(dirs), GmresOptions(30, 1e-8, 100))
    for q, (n, (f, m, d)) in enumerate(zip(ns, inst)):
        s = LSSolver(n, oms[q], torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=8, b_slab=4,
                     precision=LSS_MIXED)
        u1, st1 = s.solve(s.plane_wave_rhs(d), GmresOptions(30, 1e-8, 100))
        assert st[q][0]["iters"] == st1[0]["iters"] and st[q][0]["relres_true"] <= 1e-8
        assert rel(b.views(u, 1)[q].cpu().numpy(), u1.cpu().numpy()) <= 1e-12


def test_batch_errors():
    from paper_1705_09443_gb300 import LSSolverBatch, LssError
    b, inst, oms = make_batch((16, 20))
    lib = b.lib
    assert lib.lss_set_medium(b.ctx, b._ms[0].data_ptr(), None) == -1
    assert b"instance" in lib.lss_last_error(b.ctx)
    assert lib.lss_info(b.ctx, None, None, None) == -1
    import ctypes
    inst_ctx = ctypes.c_void_p()
    assert lib.lss_batch_instance(b.ctx, 5, ctypes.byref(inst_ctx)) == -1
    assert lib.lss_batch_instance(b.ctx, 1, ctypes.byref(inst_ctx)) == 0
    nt, ns_, L = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.lss_info(inst_ctx, ctypes.byref(nt), ctypes.byref(ns_), ctypes.byref(L)) == 0
    assert nt.value == 20 + 2 + 2 * 6
    with pytest.raises(ValueError):
        b.solve(torch.zeros(7, dtype=torch.complex128, device="cuda"))
    m_ok = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    m_bad = torch.zeros((12, 12), dtype=torch.float64, device="cuda")
    m_bad[3, 3] = float("nan")
    with pytest.raises(LssError) as e:       # instance 1 has a non-finite medium
        LSSolverBatch((16, 12), (10.0, 10.0), (m_ok, m_bad), b_pml=4, b_slab=4)
    assert e.value.code == -1 and "instance 1" in str(e.value)
