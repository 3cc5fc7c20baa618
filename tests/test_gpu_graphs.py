"""GMRES iterations replayed from CUDA graphs (lss_set_graphs) against the same
iterations launched kernel by kernel.

A graph replays the very kernels with the very arguments the direct path
launches, so solutions must be bit-identical and iteration counts equal: for
forward and adjoint solves, FP64 and mixed precision, after the medium and the
factorization change (graphs keep pointing at the same buffers, which now hold
the new factors), and after a solve with more right-hand sides reallocates
the workspaces (stale graphs must be dropped, not replayed).
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def solver(precision, seed=1706):
    from paper_1705_09443_gb300 import LSSolver
    m = synth.gaussian_medium(64, 2, 4, 0.08, (0.8, 1.2), seed)
    return LSSolver(64, 2 * math.pi * 8.0, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=12,
                    b_slab=4, precision=precision)


def run(s, g, graphs, adjoint=False):
    from paper_1705_09443_gb300 import GmresOptions
    s.use_graphs(graphs)
    f = s.adjoint_solve if adjoint else s.solve
    u, st = f(g, GmresOptions(30, 1e-10, 300))
    return u, [x["iters"] for x in st]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_graph_replay_is_bit_identical(precision, adjoint):
    s = solver(precision)
    g = torch.tensor(crand((2, 64, 64), 3), dtype=torch.complex128, device="cuda")
    u0, it0 = run(s, g, False, adjoint)
    run(s, g, True, adjoint)                 # sizes the workspaces, marks R = 2 as ready
    u1, it1 = run(s, g, True, adjoint)       # captures and replays
    u2, it2 = run(s, g, True, adjoint)       # replays the cached graphs
    assert it0 == it1 == it2
    assert torch.equal(u0, u1) and torch.equal(u0, u2)
    captured, refused = s.graph_count()
    assert captured >= max(it0) and refused == 0


def test_graphs_follow_new_medium_and_workspace_growth():
    from paper_1705_09443_gb300 import GmresOptions
    s = solver(0)
    g1 = torch.tensor(crand((1, 64, 64), 4), dtype=torch.complex128, device="cuda")
    for _ in range(3):
        run(s, g1, True)                     # graphs for R = 1 exist now
    m2 = synth.gaussian_medium(64, 2, 4, 0.08, (0.8, 1.2), 99)
    s.set_medium(torch.tensor(m2, dtype=torch.float64, device="cuda"))
    s.factor()
    u_g, it_g = run(s, g1, True)
    u_d, it_d = run(s, g1, False)
    assert it_g == it_d and torch.equal(u_g, u_d)
    ref = solver(0, seed=99)
    u_r, it_r = run(ref, g1, False)
    assert it_r == it_d and (torch.linalg.vector_norm(u_r - u_d) <= 1e-13 * torch.linalg.vector_norm(u_d)).item()
    g5 = torch.tensor(crand((5, 64, 64), 5), dtype=torch.complex128, device="cuda")
    run(s, g5, True)                         # grows the Krylov and sweep workspaces
    for _ in range(3):                       # uncaptured, then re-captured, then replayed
        u_g, it_g = run(s, g1, True)
        assert it_g == it_d and torch.equal(u_g, u_d)
    _, st = s.solve(g1, GmresOptions(30, 1e-10, 300))
    assert st[0]["relres_true"] <= 1e-10
