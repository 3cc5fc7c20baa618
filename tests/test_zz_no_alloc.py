"""The slab operator entry point that allocates nothing.

Some callers cannot let a library call reach the device allocator (their
device memory is handed out up front, or a growing workspace would stall a
latency-critical loop).  lss_apply_slab_noalloc serves them with a fixed
device scratch array.  This file is collected last so that a run that stops at
its first failure has already run every other test; it passes alone in a fresh
process and after the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_slab_operator_matches_allocating_entry_point(precision, tol):
    """On a fresh context (nothing applied yet) the entry point leaves the
    device's free memory unchanged, and it agrees with lss_apply_slab (FP64 to
    1e-12, the FP32 slab factors to 1e-6)."""
    from paper_1705_09443_gb300 import LSSolver, _lib
    lib = _lib.load()
    n = 64
    om = 2 * math.pi * 8.0
    m = synth.gaussian_medium(n, 2, 4, 0.08, (0.8, 1.2), 1706)
    s = LSSolver(n, om, torch.tensor(m, dtype=torch.float64, device="cuda"), b_pml=12, b_slab=4,
                 precision=precision)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(5)
    cases = []
    for i in (0, 8, s.n_slabs - 1):
        _, nl, _ = s.slab_info(i)
        v = rng.standard_normal((3, nl, s.n_tot)) + 1j * rng.standard_normal((3, nl, s.n_tot))
        cases.append((i, torch.tensor(v, dtype=torch.complex128, device="cuda")))
    outs = [torch.full_like(vd, complex("nan")) for _, vd in cases]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for (i, vd), w in zip(cases, outs):      # before any allocating call on this context
        rc = lib.lss_apply_slab_noalloc(s.ctx, i, ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(w.data_ptr()), 3,
                                        ctypes.c_void_p(stream))
        assert rc == 0, lib.lss_last_error(s.ctx)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for (i, vd), w in zip(cases, outs):
        ref = s.apply_slab(i, vd)
        for call in range(2):          # a repeated call shares the fixed scratch
            if call:
                w = torch.full_like(vd, complex("nan"))
                rc = lib.lss_apply_slab_noalloc(s.ctx, i, ctypes.c_void_p(vd.data_ptr()),
                                                ctypes.c_void_p(w.data_ptr()), 3, ctypes.c_void_p(stream))
                assert rc == 0, lib.lss_last_error(s.ctx)
            torch.cuda.synchronize()
            err = (torch.linalg.norm(w - ref) / torch.linalg.norm(ref)).item()
            assert err <= tol, (i, call, err)


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    from paper_1705_09443_gb300 import LSSolver, _lib
    lib = _lib.load()
    n = 64
    s = LSSolver(n, 2 * math.pi * 8.0, torch.zeros((n, n), dtype=torch.float64, device="cuda"), b_pml=12,
                 b_slab=4)
    _, nl, _ = s.slab_info(1)
    R = 512                            # 512 x 90 x 32 (padded width) x 16 B > 8 MiB
    v = torch.zeros((R, nl, s.n_tot), dtype=torch.complex128, device="cuda")
    w = torch.empty_like(v)
    rc = lib.lss_apply_slab_noalloc(s.ctx, 1, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()), R,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -8 and b"fixed scratch" in lib.lss_last_error(s.ctx)
