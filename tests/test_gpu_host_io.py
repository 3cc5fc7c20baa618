"""lss_solve_host: the solve with host buffers (copies in and out inside the
call) gives the same solution and statistics as lss_solve on device buffers,
in 2D and 3D."""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 10)])
def test_solve_host_equals_device_solve(dim, n):
    from paper_1705_09443_gb300 import GmresOptions, LSSolver
    om = 2 * math.pi * (n + 1) / 8
    m = synth.gaussian_medium(n, dim, 3, 0.15, (0.8, 1.2), 40 + dim)
    s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=4 if dim == 3 else 12,
                 b_slab=4)
    dirs = np.eye(dim)[:2]
    g = s.plane_wave_rhs(dirs)
    opts = GmresOptions(30, 1e-10, 200)
    u_dev, st_dev = s.solve(g, opts)
    g_host = g.cpu().pin_memory()
    u_host = torch.empty_like(g_host).pin_memory()
    st_host = s.solve_host(g_host, u_host, opts)
    assert torch.equal(u_host, u_dev.cpu())
    for a, b in zip(st_host, st_dev):
        assert a["iters"] == b["iters"] and a["relres_true"] == b["relres_true"]
