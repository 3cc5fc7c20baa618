"""Autotuner (lss_autotune): the launch parameters it picks change no result.

Every candidate computes each output with the same arithmetic in the same
order, so a solve after tuning must be bit-identical to one before it, for
FP64 and mixed precision, forward and adjoint, and for a batch of instances.
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_solves_are_bit_identical(precision):
    from paper_1705_09443_gb300 import GmresOptions, LSSolver
    m = synth.gaussian_medium(64, 2, 4, 0.08, (0.8, 1.2), 1706)
    s = LSSolver(64, 2 * math.pi * 8.0, torch.tensor(m, dtype=torch.float64, device="cuda"), precision=precision)
    rng = np.random.default_rng(7)
    g = torch.tensor(rng.standard_normal((3, 64, 64)) + 1j * rng.standard_normal((3, 64, 64)),
                     dtype=torch.complex128, device="cuda")
    o = GmresOptions(30, 1e-10, 300)
    u0, st0 = s.solve(g, o)
    mu0, _ = s.adjoint_solve(g, o)
    ch = s.autotune(3)
    assert ch["fft_col_group"] in (1, 2, 4, 8) and ch["solve_stages"] in (0, 2, 3, 4)
    assert ch["recur_stages"] in (2, 3, 4)
    for _ in range(2):                       # uncaptured, then from graphs
        u1, st1 = s.solve(g, o)
        assert [x["iters"] for x in st0] == [x["iters"] for x in st1] and torch.equal(u0, u1)
    mu1, _ = s.adjoint_solve(g, o)
    assert torch.equal(mu0, mu1)


def test_tuned_batch_is_bit_identical():
    from paper_1705_09443_gb300 import GmresOptions, LSSolverBatch, LSS_MIXED
    ns = (24, 41, 60)
    inst = synth.ragged_instances(ns, 1730)
    b = LSSolverBatch(ns, [2 * math.pi * f for f, _, _ in inst],
                      [torch.tensor(m, dtype=torch.float64, device="cuda") for _, m, _ in inst],
                      b_pml=8, precision=LSS_MIXED)
    g = b.plane_wave_rhs(np.stack([d for _, _, d in inst]))
    u0, _ = b.solve(g, GmresOptions(30, 1e-8, 100))
    b.autotune(1)
    u1, _ = b.solve(g, GmresOptions(30, 1e-8, 100))
    assert torch.equal(u0, u1)
