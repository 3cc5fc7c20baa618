"""Python wrapper of the C ABI: one LSSolver per (grid, omega, medium).

Device memory and streams come from PyTorch; every step of the solve runs in
the library's kernels.  Vectors are complex128 CUDA tensors of shape
(R, n, n) in 2D or (R, n, n, n) in 3D (or without the leading R for one
right-hand side); the grid's dimension is that of m.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _lib
from ._lib import check


@dataclasses.dataclass
class GmresOptions:
    restart: int = 30
    tol: float = 1e-8
    max_iter: int = 300


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _c128(x: torch.Tensor) -> torch.Tensor:
    if x.dtype != torch.complex128 or not x.is_cuda:
        raise TypeError("expected a complex128 CUDA tensor")
    if x.is_conj():          # a lazy conjugate view: the library needs the values in memory
        x = x.resolve_conj()
    if not x.is_contiguous():
        raise TypeError("expected a contiguous complex128 CUDA tensor")
    return x


class LSSolver:
    """Sparsify-and-sweep preconditioned LS solver (Sec. 2, Algorithms 1-2)."""

    def __init__(self, n: int, omega: float, m: torch.Tensor, b_pml: int = 12, C: float = 10.0,
                 b_slab: int = 4, b_aux: int = 0, n_samples: int = 0, precision: int = _lib.LSS_FP64,
                 factor: bool = True, stream=None, fronts: int = 1, recursive: bool = False):
        self.lib = _lib.load()
        self.n, self.omega = int(n), float(omega)
        self.fronts = int(fronts)
        self.recursive = bool(recursive)
        self.dim = m.dim()
        if m.dtype != torch.float64 or not m.is_cuda or self.dim not in (2, 3) or \
                tuple(m.shape) != (n,) * self.dim:
            raise TypeError("m must be a (n, n) or (n, n, n) float64 CUDA tensor")
        self.shape = (self.n,) * self.dim
        m = m.contiguous()
        ctx = ctypes.c_void_p()
        g = _lib.Grid(self.dim, self.n)
        p = _lib.Pml(int(b_pml), float(C))
        s = _lib.Slab(int(b_slab), int(b_aux), int(n_samples), int(fronts), int(bool(recursive)))
        check(self.lib.lss_setup(ctypes.byref(ctx), ctypes.byref(g), self.omega, m.data_ptr(), ctypes.byref(p),
                                 ctypes.byref(s), int(precision), _stream_ptr(stream)))
        self.ctx = ctx
        nt, ns, L = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.lib.lss_info(self.ctx, ctypes.byref(nt), ctypes.byref(ns), ctypes.byref(L))
        self.n_tot, self.n_slabs, self.fft_len = nt.value, ns.value, L.value
        if factor:
            self.factor(stream)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value:
            torch.cuda.synchronize()
            self.lib.lss_destroy(ctx)
            self.ctx = None

    def _check(self, code):
        return check(code, self.ctx)

    def set_medium(self, m: torch.Tensor, stream=None):
        if m.dtype != torch.float64 or not m.is_cuda or tuple(m.shape) != self.shape:
            raise TypeError("m must be a float64 CUDA tensor of the grid's shape")
        self._check(self.lib.lss_set_medium(self.ctx, m.contiguous().data_ptr(), _stream_ptr(stream)))
        self.medium_version = getattr(self, "medium_version", 0) + 1

    def profile(self, enable: bool = True):
        self._check(self.lib.lss_profile(self.ctx, int(enable)))

    def use_graphs(self, enable: bool = True):
        """Replay each GMRES iteration from a CUDA graph (lss_set_graphs)."""
        self._check(self.lib.lss_set_graphs(self.ctx, int(enable)))

    def autotune(self, R: int = 1, stream=None):
        """Launch parameters for R right-hand sides, picked by timing (lss_autotune)."""
        ch = (ctypes.c_int * 7)()
        self._check(self.lib.lss_autotune(self.ctx, int(R), ch, _stream_ptr(stream)))
        return dict(fft_col_group=ch[0], solve_rhs_global=ch[1] == 0, solve_stages=ch[2], recur_stages=ch[3],
                    wide_solve_stages=ch[4], solve_two_per_sm=ch[5] == 1, solve_rhs_per_cta=ch[6])

    def graph_count(self):
        """(captured, refused) iteration graphs held by the context."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lss_graph_count(self.ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def profile_read(self):
        """Device milliseconds and launch counts per kernel group since the last read."""
        k = len(_lib.PROF_CATEGORIES)
        ms = np.zeros(k)
        cnt = np.zeros(k, dtype=np.int64)
        self._check(self.lib.lss_profile_read(self.ctx, ms.ctypes.data, cnt.ctypes.data, k))
        return dict(zip(_lib.PROF_CATEGORIES, ms.tolist())), dict(zip(_lib.PROF_CATEGORIES, cnt.tolist()))

    def factor(self, stream=None):
        self._check(self.lib.lss_factor(self.ctx, _stream_ptr(stream)))

    def slab_info(self, i: int):
        s, nl, na = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lss_slab_info(self.ctx, i, ctypes.byref(s), ctypes.byref(nl), ctypes.byref(na)))
        return s.value, nl.value, na.value

    def stencils(self):
        """alpha, beta: 3^dim complex entries each (Eq. alpha, Eq. beta)."""
        a = np.zeros(2 * 3 ** self.dim)
        b = np.zeros(2 * 3 ** self.dim)
        self._check(self.lib.lss_get_stencils(self.ctx, a.ctypes.data, b.ctypes.data))
        return a.view(np.complex128), b.view(np.complex128)

    def _batch(self, x):
        return x if x.dim() == self.dim + 1 else x.unsqueeze(0)

    def plane_wave_rhs(self, dirs, with_incident: bool = False, stream=None):
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, self.dim))
        R = d.shape[0]
        g = torch.empty((R,) + self.shape, dtype=torch.complex128, device="cuda")
        uI = torch.empty_like(g) if with_incident else None
        self._check(self.lib.lss_plane_wave_rhs(self.ctx, d.ctypes.data, R, g.data_ptr(),
                                                uI.data_ptr() if uI is not None else None, _stream_ptr(stream)))
        return (g, uI) if with_incident else g

    def apply_A(self, x: torch.Tensor, transpose: bool = False, stream=None) -> torch.Tensor:
        x = _c128(self._batch(x))
        y = torch.empty_like(x)
        self._check(self.lib.lss_apply_A(self.ctx, x.data_ptr(), y.data_ptr(), x.shape[0], int(transpose),
                                         _stream_ptr(stream)))
        return y

    def apply_P(self, x: torch.Tensor, transpose: bool = False, stream=None) -> torch.Tensor:
        x = _c128(self._batch(x))
        y = torch.empty_like(x)
        self._check(self.lib.lss_apply_P(self.ctx, x.data_ptr(), y.data_ptr(), x.shape[0], int(transpose),
                                         _stream_ptr(stream)))
        return y

    def apply_slab(self, i: int, v: torch.Tensor, stream=None) -> torch.Tensor:
        v = _c128(self._batch(v))
        w = torch.empty_like(v)
        self._check(self.lib.lss_apply_slab(self.ctx, i, v.data_ptr(), w.data_ptr(), v.shape[0],
                                            _stream_ptr(stream)))
        return w

    def test_inject(self, what: int, a: int = 0, b: int = 0, stream=None):
        """Fault injection for tests (lss_test_inject): 1 = zero block row b of
        slab a (the next factor meets a zero pivot), 2 = bounded device waits
        that expire (returns LSS_ERR_TIMEOUT)."""
        self._check(self.lib.lss_test_inject(self.ctx, int(what), int(a), int(b), _stream_ptr(stream)))

    def solve(self, g: torch.Tensor, opts: GmresOptions | None = None, stream=None, raise_on_noconv=True):
        o = opts or GmresOptions()
        g = _c128(self._batch(g))
        u = torch.empty_like(g)
        R = g.shape[0]
        st = (_lib.Stats * R)()
        go = _lib.Gmres(o.restart, o.tol, o.max_iter)
        code = self.lib.lss_solve(self.ctx, g.data_ptr(), u.data_ptr(), R, ctypes.byref(go), st,
                                  _stream_ptr(stream))
        if code != 0 and not (code == -5 and not raise_on_noconv):
            self._check(code)
        return u, [dict(iters=s.iters, converged=bool(s.converged), relres_est=s.relres_est,
                        relres_true=s.relres_true) for s in st]

    def adjoint_solve(self, rhs: torch.Tensor, opts: GmresOptions | None = None, stream=None,
                      raise_on_noconv=True):
        """mu with (I + omega^2 M K) mu = rhs (lss_adjoint_solve)."""
        o = opts or GmresOptions()
        rhs = _c128(self._batch(rhs))
        mu = torch.empty_like(rhs)
        R = rhs.shape[0]
        st = (_lib.Stats * R)()
        go = _lib.Gmres(o.restart, o.tol, o.max_iter)
        code = self.lib.lss_adjoint_solve(self.ctx, rhs.data_ptr(), mu.data_ptr(), R, ctypes.byref(go), st,
                                          _stream_ptr(stream))
        if code != 0 and not (code == -5 and not raise_on_noconv):
            self._check(code)
        return mu, [dict(iters=s.iters, converged=bool(s.converged), relres_est=s.relres_est,
                         relres_true=s.relres_true) for s in st]

    def helmholtz_solve(self, f: torch.Tensor, opts: GmresOptions | None = None, stream=None):
        """u with alpha^* u + omega^2 beta^* (m u) = beta^* f on I^h and the PML rows
        (Sec. 4, lss_helmholtz_solve): the sparsified discretization of
        (-Laplace - omega^2 (1 - m)) u = f.  f: (R, n, n) or (n, n) complex128."""
        o = opts or GmresOptions()
        f = _c128(self._batch(f))
        u = torch.empty_like(f)
        R = f.shape[0]
        st = (_lib.Stats * R)()
        go = _lib.Gmres(o.restart, o.tol, o.max_iter)
        self._check(self.lib.lss_helmholtz_solve(self.ctx, f.data_ptr(), u.data_ptr(), R, ctypes.byref(go), st,
                                                 _stream_ptr(stream)))
        return u, [dict(iters=s.iters, converged=bool(s.converged), relres_est=s.relres_est,
                        relres_true=s.relres_true) for s in st]

    def medium_gradient(self, mu: torch.Tensor, u: torch.Tensor, dirs, stream=None) -> torch.Tensor:
        """sum_r Re((-omega^2 K mu_r) . (u_r + u_I,r)) on I (lss_medium_gradient)."""
        mu = _c128(self._batch(mu))
        u = _c128(self._batch(u))
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 2))
        grad = torch.empty((self.n, self.n), dtype=torch.float64, device="cuda")
        self._check(self.lib.lss_medium_gradient(self.ctx, mu.data_ptr(), u.data_ptr(), d.ctypes.data, d.shape[0],
                                                 grad.data_ptr(), _stream_ptr(stream)))
        return grad

    def solve_host(self, g_host: torch.Tensor, u_host: torch.Tensor, opts: GmresOptions | None = None,
                   stream=None):
        o = opts or GmresOptions()
        R = g_host.shape[0] if g_host.dim() == self.dim + 1 else 1
        st = (_lib.Stats * R)()
        go = _lib.Gmres(o.restart, o.tol, o.max_iter)
        self._check(self.lib.lss_solve_host(self.ctx, g_host.data_ptr(), u_host.data_ptr(), R, ctypes.byref(go),
                                            st, _stream_ptr(stream)))
        return [dict(iters=s.iters, converged=bool(s.converged), relres_est=s.relres_est,
                     relres_true=s.relres_true) for s in st]


class LSSolverBatch:
    """Independent problems of different size, frequency and medium behind one
    context (lss_setup_batch); calls run the instances concurrently.

    Vectors are flat complex128 CUDA tensors holding instance q's (R, n_q, n_q)
    block after the blocks of instances 0..q-1; `views` splits one."""

    def __init__(self, ns, omegas, ms, b_pml: int = 12, C: float = 10.0, b_slab: int = 4, b_aux: int = 0,
                 n_samples: int = 0, precision: int = _lib.LSS_FP64, factor: bool = True, stream=None,
                 fronts: int = 1):
        self.lib = _lib.load()
        self.ns = [int(n) for n in ns]
        self.omegas = [float(w) for w in omegas]
        if not (len(self.ns) == len(self.omegas) == len(ms)) or not self.ns:
            raise ValueError("ns, omegas and ms must have the same non-zero length")
        self._ms = []
        for n, m in zip(self.ns, ms):
            if m.dtype != torch.float64 or not m.is_cuda or tuple(m.shape) != (n, n):
                raise TypeError("each m must be a (n, n) float64 CUDA tensor")
            self._ms.append(m.contiguous())
        q = len(self.ns)
        grids = (_lib.Grid * q)(*[_lib.Grid(2, n) for n in self.ns])
        om = (ctypes.c_double * q)(*self.omegas)
        mp = (ctypes.c_void_p * q)(*[m.data_ptr() for m in self._ms])
        p = _lib.Pml(int(b_pml), float(C))
        s = _lib.Slab(int(b_slab), int(b_aux), int(n_samples), int(fronts))
        ctx = ctypes.c_void_p()
        check(self.lib.lss_setup_batch(ctypes.byref(ctx), q, grids, om, mp, ctypes.byref(p), ctypes.byref(s),
                                       int(precision), _stream_ptr(stream)))
        self.ctx = ctx
        nq, tot = ctypes.c_int(), ctypes.c_longlong()
        self._check(self.lib.lss_batch_info(self.ctx, ctypes.byref(nq), ctypes.byref(tot)))
        self.n_inst, self.elems_per_rhs = nq.value, tot.value
        if factor:
            self.factor(stream)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value:
            torch.cuda.synchronize()
            self.lib.lss_destroy(ctx)
            self.ctx = None

    def _check(self, code):
        return check(code, self.ctx)

    def views(self, flat: torch.Tensor, R: int):
        """Instance q's (R, n_q, n_q) view of a flat batch vector."""
        out, o = [], 0
        for n in self.ns:
            out.append(flat[o:o + R * n * n].view(R, n, n))
            o += R * n * n
        return out

    def pack(self, xs):
        """One flat batch vector from a list of (R, n_q, n_q) tensors."""
        return torch.cat([_c128(x).reshape(-1) for x in xs])

    def factor(self, stream=None):
        self._check(self.lib.lss_factor(self.ctx, _stream_ptr(stream)))

    def profile(self, enable: bool = True):
        self._check(self.lib.lss_profile(self.ctx, int(enable)))

    def use_graphs(self, enable: bool = True):
        self._check(self.lib.lss_set_graphs(self.ctx, int(enable)))

    def graph_count(self):
        """(captured, refused) iteration graphs held by the batch and its instances."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lss_graph_count(self.ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def autotune(self, R: int = 1, stream=None):
        """Tune every instance for R right-hand sides (lss_autotune); returns instance 0's choice."""
        ch = (ctypes.c_int * 7)()
        self._check(self.lib.lss_autotune(self.ctx, int(R), ch, _stream_ptr(stream)))
        return dict(fft_col_group=ch[0], solve_rhs_global=ch[1] == 0, solve_stages=ch[2], recur_stages=ch[3],
                    wide_solve_stages=ch[4], solve_two_per_sm=ch[5] == 1, solve_rhs_per_cta=ch[6])

    def profile_read(self):
        k = len(_lib.PROF_CATEGORIES)
        ms = np.zeros(k)
        cnt = np.zeros(k, dtype=np.int64)
        self._check(self.lib.lss_profile_read(self.ctx, ms.ctypes.data, cnt.ctypes.data, k))
        return dict(zip(_lib.PROF_CATEGORIES, ms.tolist())), dict(zip(_lib.PROF_CATEGORIES, cnt.tolist()))

    def plane_wave_rhs(self, dirs, stream=None) -> torch.Tensor:
        """dirs: (n_inst, R, 2) directions, R per instance (or (R, 2): the same for all)."""
        d = np.asarray(dirs, dtype=np.float64)
        if d.ndim == 2:
            d = np.broadcast_to(d, (self.n_inst,) + d.shape)
        d = np.ascontiguousarray(d.reshape(self.n_inst, -1, 2))
        R = d.shape[1]
        g = torch.empty(R * self.elems_per_rhs, dtype=torch.complex128, device="cuda")
        self._check(self.lib.lss_plane_wave_rhs(self.ctx, d.ctypes.data, R, g.data_ptr(), None, _stream_ptr(stream)))
        return g

    def _R(self, flat):
        R, rem = divmod(flat.numel(), self.elems_per_rhs)
        if rem or R < 1:
            raise ValueError("batch vector length must be R * sum(n_q^2)")
        return R

    def apply_A(self, x: torch.Tensor, transpose: bool = False, stream=None) -> torch.Tensor:
        x = _c128(x)
        y = torch.empty_like(x)
        self._check(self.lib.lss_apply_A(self.ctx, x.data_ptr(), y.data_ptr(), self._R(x), int(transpose),
                                         _stream_ptr(stream)))
        return y

    def apply_P(self, x: torch.Tensor, transpose: bool = False, stream=None) -> torch.Tensor:
        x = _c128(x)
        y = torch.empty_like(x)
        self._check(self.lib.lss_apply_P(self.ctx, x.data_ptr(), y.data_ptr(), self._R(x), int(transpose),
                                         _stream_ptr(stream)))
        return y

    def _solve(self, fn, g, opts, stream, raise_on_noconv):
        o = opts or GmresOptions()
        g = _c128(g)
        u = torch.empty_like(g)
        R = self._R(g)
        st = (_lib.Stats * (R * self.n_inst))()
        go = _lib.Gmres(o.restart, o.tol, o.max_iter)
        code = fn(self.ctx, g.data_ptr(), u.data_ptr(), R, ctypes.byref(go), st, _stream_ptr(stream))
        if code != 0 and not (code == -5 and not raise_on_noconv):
            self._check(code)
        stats = [dict(iters=s.iters, converged=bool(s.converged), relres_est=s.relres_est,
                      relres_true=s.relres_true) for s in st]
        return u, [stats[q * R:(q + 1) * R] for q in range(self.n_inst)]

    def solve(self, g: torch.Tensor, opts: GmresOptions | None = None, stream=None, raise_on_noconv=True):
        """u for every instance and RHS; stats[q][r]."""
        return self._solve(self.lib.lss_solve, g, opts, stream, raise_on_noconv)

    def adjoint_solve(self, rhs: torch.Tensor, opts: GmresOptions | None = None, stream=None,
                      raise_on_noconv=True):
        return self._solve(self.lib.lss_adjoint_solve, rhs, opts, stream, raise_on_noconv)
