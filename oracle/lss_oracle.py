"""FP64 CPU oracle for the sparsify-and-sweep preconditioned Lippmann-Schwinger solve.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  The CUDA
library never calls it and shares no code with it.

Liu & Ying, "Sparsify and sweep: an efficient preconditioner for the
Lippmann-Schwinger equation" (arXiv:1705.09443).  Every function follows the
paper's definitions in the paper's order and notation, in plain numpy/scipy
(complex128).  Readings where the paper is silent or garbled are marked
READING; they are:

  * k_0 (Sec. 2.1): the paper cites a Duan-Rokhlin correction without weights;
    here k_0 is the integral of G over the grid cell [-h/2, h/2]^d.
  * Eq. (alpha) drops the constraint "= 1"; alpha is a unit vector, phase fixed
    so that its centre entry is real positive (also gamma, Eq. (gamma)).
  * sigma at the Dirichlet layer is the continuous extension (-C/omega, C/omega).
  * frequency samples: endpoints included, max/min over m on I and 0, ties to
    the lower sample, a single sample when max = min (Sec. 2.3).
  * slabs: the last slab takes the remainder of the normal layers (Sec. 2.4
    remark 2); auxiliary layers are virtual copies left of D_i (Eq. Hwv_approx).
  * GMRES: right preconditioning, x0 = 0, MGS Arnoldi, Givens rotations,
    stop when |rho_{j+1}| <= tol * ||g|| (Sec. 2.5 uses "standard GMRES").

Parity pins for every function are in tests/test_oracle_*.py.  Parity
unpinned: the O(h^4 log^2) accuracy claimed for the paper's k_0 (the cell
average used here is lower order), and the exact alpha values (the paper
prints none; alpha is pinned by its defining properties instead).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as sps

# --------------------------------------------------------------------------
# Sec. 1 / Sec. 2.1: Green's function, Nystrom weights, discrete LS operator
# --------------------------------------------------------------------------


def green(d: int, omega: float, r):
    """Free-space Helmholtz Green's function G(x), |x| = r > 0 (Sec. 1):
    (i/4) H_0^(1)(omega r) in 2D, exp(i omega r) / (4 pi r) in 3D."""
    r = np.asarray(r, dtype=np.float64)
    if d == 2:
        return 0.25j * sps.hankel1(0, omega * r)
    return np.exp(1j * omega * r) / (4.0 * math.pi * r)


def cell_integral_G(d: int, omega: float, h: float, nq: int = 48) -> complex:
    """READING of k_0 (Sec. 2.1, Sec. 3.1): integral of G over the cell [-h/2,h/2]^d.

    2D, in polar coordinates about the singular point:
        int_0^R H_0(omega r) r dr = R H_1(omega R)/omega + 2i/(pi omega^2),
    so  k_0 = (i/(4 omega)) int_0^{2pi} R(t) H_1(omega R(t)) dt - 1/omega^2,
    R(t) = (h/2)/max(|cos t|, |sin t|), integrated over one of the 8 congruent
    sectors [0, pi/4] with Gauss-Legendre.
    3D:  int_0^R e^{i omega r} r dr = e^{i omega R}(R/(i omega) + 1/omega^2) - 1/omega^2,
    integrated over the 6 faces of the cube with the solid-angle element
    (h/2) dy dz / R^3, tensor Gauss-Legendre on each face.
    """
    x, wq = np.polynomial.legendre.leggauss(nq)
    if d == 2:
        a, b = 0.0, math.pi / 4
        t = 0.5 * (b - a) * x + 0.5 * (b + a)
        w = 0.5 * (b - a) * wq
        R = (0.5 * h) / np.cos(t)
        ang = np.sum(w * R * sps.hankel1(1, omega * R)) * 8.0
        return complex(1j / (4.0 * omega) * ang - 1.0 / omega ** 2)
    a = 0.5 * h
    y = a * x
    wy = a * wq
    Y, Z = np.meshgrid(y, y, indexing="ij")
    W = np.outer(wy, wy)
    R = np.sqrt(a * a + Y * Y + Z * Z)
    F = np.exp(1j * omega * R) * (R / (1j * omega) + 1.0 / omega ** 2) - 1.0 / omega ** 2
    face = np.sum(W * F * a / R ** 3)
    return complex(6.0 * face / (4.0 * math.pi))


def nystrom_weights(d: int, n: int, omega: float, span: int) -> np.ndarray:
    """k_j = G(p_j) h^d for j != 0 and k_0 from cell_integral_G (Sec. 2.1),
    for j in {-span..span}^d.  Returned array is indexed [j1+span, j2+span, ...]."""
    h = 1.0 / (n + 1)
    ax = np.arange(-span, span + 1, dtype=np.float64)
    grids = np.meshgrid(*([ax] * d), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids)) * h
    k = np.zeros(r.shape, dtype=np.complex128)
    nz = r > 0
    k[nz] = green(d, omega, r[nz]) * h ** d
    k[(span,) * d] = cell_integral_G(d, omega, h)
    return k


def ls_apply(u: np.ndarray, m: np.ndarray, omega: float, kw: np.ndarray) -> np.ndarray:
    """(I + omega^2 K M) u on I (Eq. LS_d_c), the convolution sum_{j in I}
    k_{i-j} m_j u_j evaluated with a zero-padded FFT (Sec. 2.1).  kw must span
    at least n-1; any FFT length >= 2n-1 gives the same linear convolution."""
    n = u.shape[0]
    d = u.ndim
    span = (kw.shape[0] - 1) // 2
    L = 2 * n
    kc = np.zeros((L,) * d, dtype=np.complex128)
    idx = np.arange(-(n - 1), n)
    sl = tuple(np.ix_(*([idx % L] * d)))
    src = tuple(np.ix_(*([idx + span] * d)))
    kc[sl] = kw[src]
    v = np.zeros((L,) * d, dtype=np.complex128)
    v[(slice(0, n),) * d] = m * u
    conv = np.fft.ifftn(np.fft.fftn(kc) * np.fft.fftn(v))[(slice(0, n),) * d]
    return u + omega ** 2 * conv


def ls_apply_direct(u, m, omega, kw):
    """The same operator by direct O(N^2) summation (pin for ls_apply)."""
    n = u.shape[0]
    d = u.ndim
    span = (kw.shape[0] - 1) // 2
    pts = np.array(np.meshgrid(*([np.arange(n)] * d), indexing="ij")).reshape(d, -1).T
    mu = (m * u).reshape(-1)
    out = np.zeros(n ** d, dtype=np.complex128)
    for a, pi in enumerate(pts):
        off = pi[None, :] - pts + span
        out[a] = np.sum(kw[tuple(off.T)] * mu)
    return u + omega ** 2 * out.reshape(u.shape)


def ls_apply_transpose(v, m, omega, kw):
    """A^T v = v + omega^2 M K v (K is symmetric since k is even)."""
    z = ls_apply(v, np.ones_like(m), omega, kw) - v      # omega^2 K v
    return v + m * z


def plane_wave(n: int, omega: float, direction) -> np.ndarray:
    """[u_I]_j = exp(i omega d . p_j) on I (Sec. 2.1)."""
    xs = np.meshgrid(*([np.arange(1, n + 1) / (n + 1.0)] * len(direction)), indexing="ij")
    ph = sum(float(direction[a]) * xs[a] for a in range(len(direction)))
    return np.exp(1j * omega * ph)


def ls_rhs(m, omega, kw, direction) -> np.ndarray:
    """g_i = -omega^2 sum_{j in I} k_{i-j} m_j [u_I]_j (Sec. 2.1)."""
    uI = plane_wave(m.shape[0], omega, direction)
    return -(ls_apply(uI, m, omega, kw) - uI)


# --------------------------------------------------------------------------
# Sec. 2.2.1: interior stencils alpha, beta
# --------------------------------------------------------------------------


def neighbourhood_offsets(d: int) -> np.ndarray:
    """mu = {j : ||j||_inf <= 1}, listed in lexicographic order (x1 slowest)."""
    ax = [-1, 0, 1]
    return np.array(np.meshgrid(*([ax] * d), indexing="ij")).reshape(d, -1).T


def interior_stencils(d: int, n: int, omega: float):
    """alpha = argmin_{||alpha||=1} ||alpha^* K_{mu,mu^c}|| (Eq. alpha) and
    beta^* = alpha^* K_{mu,mu} (Eq. beta), with mu^c = {-n..n}^d minus mu.

    alpha is the left singular vector of the smallest singular value.
    Returns (alpha, beta, sigma) with sigma the singular values (descending).
    """
    mu = neighbourhood_offsets(d)
    kw = nystrom_weights(d, n, omega, n + 1)
    span = n + 1
    ax = np.arange(-n, n + 1)
    cols = np.array(np.meshgrid(*([ax] * d), indexing="ij")).reshape(d, -1).T
    in_mu = np.all(np.abs(cols) <= 1, axis=1)
    cols = cols[~in_mu]
    K_c = np.empty((len(mu), len(cols)), dtype=np.complex128)
    for a, o in enumerate(mu):
        off = o[None, :] - cols + span
        K_c[a] = kw[tuple(off.T)]
    U, s, _ = np.linalg.svd(K_c, full_matrices=False)
    alpha = U[:, -1]
    c = alpha[len(mu) // 2]
    alpha = alpha * (abs(c) / c)
    alpha[len(mu) // 2] = abs(c)
    K_mm = np.empty((len(mu), len(mu)), dtype=np.complex128)
    for a, o in enumerate(mu):
        K_mm[a] = kw[tuple((o[None, :] - mu + span).T)]
    beta = (alpha.conj() @ K_mm).conj()
    return alpha, beta, s


# --------------------------------------------------------------------------
# Sec. 2.2.2: PML profile and PML stencils gamma
# --------------------------------------------------------------------------


def pml_sigma(idx, n: int, b: int, C: float, omega: float):
    """sigma(x) at x = idx * h (Sec. 2.2.2, eta = b h): -(C/omega)((x+h)/eta)^2
    left of -h, 0 on (-h, 1+h), (C/omega)((x-1-h)/eta)^2 right of 1+h.
    READING: the Dirichlet layer (idx = -b-1 or n+2+b) takes the same formula."""
    idx = np.asarray(idx, dtype=np.float64)
    left = np.where(idx <= -1, -(C / omega) * ((idx + 1.0) / b) ** 2, 0.0)
    right = np.where(idx >= n + 2, (C / omega) * ((idx - n - 2.0) / b) ** 2, 0.0)
    return left + right


def pml_directions(d: int) -> np.ndarray:
    """R: the 8 (2D) or 26 (3D) directions toward the neighbours, normalised."""
    mu = neighbourhood_offsets(d)
    mu = mu[np.any(mu != 0, axis=1)].astype(np.float64)
    return mu / np.linalg.norm(mu, axis=1)[:, None]


def pml_stencil(omega_loc: float, h: float, sig: list[np.ndarray]) -> np.ndarray:
    """gamma with gamma^* F^sigma_{mu_i,R} = 0, ||gamma|| = 1 (Eq. gamma).

    sig[a] = sigma at the three positions (offset -1, 0, +1) along axis a.
    Column r of F is exp(i omega_loc r . (p_j^sigma - p_i^sigma)) over j in mu_i.
    gamma spans the orthogonal complement of range(F): the last column of the
    complete QR factor of F.  Returns the row coefficients conj(gamma), with
    the centre entry real positive.
    """
    d = len(sig)
    mu = neighbourhood_offsets(d)
    R = pml_directions(d)
    dz = np.zeros((len(mu), d), dtype=np.complex128)
    for a in range(d):
        s = np.asarray(sig[a])
        dz[:, a] = mu[:, a] * h + 1j * (s[mu[:, a] + 1] - s[1])
    F = np.exp(1j * omega_loc * (dz @ R.T))
    Q, _ = np.linalg.qr(F, mode="complete")
    gamma = Q[:, -1]
    c = gamma[len(mu) // 2]
    gamma = gamma * (abs(c) / c)
    gamma[len(mu) // 2] = abs(c)
    return gamma.conj()


def frequency_samples(m: np.ndarray, omega: float, n_s: int) -> np.ndarray:
    """Samples of the squared-frequency range [omega^2(1-max m), omega^2(1-min m)]
    (Sec. 2.3).  READING: endpoints included, 0 joins the range (PML points)."""
    mmax = max(float(np.max(m)), 0.0)
    mmin = min(float(np.min(m)), 0.0)
    if mmax == mmin:
        return np.array([omega ** 2 * (1.0 - mmax)])
    return np.linspace(omega ** 2 * (1.0 - mmax), omega ** 2 * (1.0 - mmin), n_s)


def nearest_sample(samples: np.ndarray, value: float) -> int:
    """Index of the sample closest to value; ties go to the lower index."""
    return int(np.argmin(np.abs(samples - value)))


# --------------------------------------------------------------------------
# Sec. 2.2.3, 2.3, 2.4: sparse system H, slabs, moving-PML subproblems, sweep
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Params:
    b_pml: int = 12
    b_slab: int = 4
    b_aux: int | None = None      # READING: defaults to b_pml (Sec. 2.3 uses b for both)
    C: float = 10.0
    n_samples: int | None = None  # defaults to n (Sec. 2.3)
    fronts: int = 1               # 2: two sweeping fronts meeting in the middle slab (Sec. 2.4 remark 1)
    recursive: bool = False       # 3D: slab subproblems swept along x2 (the recursive approach, Sec. 3.1)


class _TwoFronts:
    """The sweep with two fronts (Sec. 2.4 remark 1, the setting of Sec. 2.5):
    the slabs left of the middle slab c = (l-1)//2 carry their moving PML on
    the left (as in Algorithm 2), the slabs right of it on the right, and c
    is padded with auxiliary PML on both sides.  Both fronts eliminate toward
    c, c is solved with the couplings from both neighbours, then both fronts
    substitute back toward the boundaries.  With the exact Schur inverses
    this is block Gaussian elimination from both ends, i.e. H^{-1}."""

    def aux_sides(self, i: int):
        """(auxiliary layers on the left, on the right) of slab i's subproblem."""
        nl = self.n_slabs
        if self.p.fronts != 2:
            return i > 0, False
        c = (nl - 1) // 2
        return (0 < i <= c), (c <= i < nl - 1)

    def right_sigma(self, e: int, a1: int):
        """sigma along x1 at a1 - 1, a1, a1 + 1 for the auxiliary PML right of
        D_i's last layer e: the right PML profile of width b_aux translated so
        that layer e plays the role of index n + 1 (the mirror image of the
        left auxiliary profile)."""
        return pml_sigma(np.array([a1 - 1, a1, a1 + 1]) - e + self.n + 1, self.n, self.b_aux, self.p.C,
                         self.omega)

    def sweep_two_fronts(self, f, T=None):
        T = T or self.T
        nl = self.n_slabs
        c = (nl - 1) // 2
        u = [None] * nl
        for i in range(0, c):                              # left front, toward c
            v = self.slab_view(f, i).copy()
            if i > 0:
                v[0] -= self.couple_left(i, u[i - 1][-1])
            u[i] = T(i, v)
        for i in range(nl - 1, c, -1):                     # right front, toward c
            v = self.slab_view(f, i).copy()
            if i < nl - 1:
                v[-1] -= self.couple_right(i, u[i + 1][0])
            u[i] = T(i, v)
        v = self.slab_view(f, c).copy()                    # the middle slab
        if c > 0:
            v[0] -= self.couple_left(c, u[c - 1][-1])
        if c < nl - 1:
            v[-1] -= self.couple_right(c, u[c + 1][0])
        u[c] = T(c, v)
        for i in range(c - 1, -1, -1):                     # back toward the left boundary
            w = np.zeros_like(u[i])
            w[-1] = self.couple_right(i, u[i + 1][0])
            u[i] = u[i] - T(i, w)
        for i in range(c + 1, nl):                         # back toward the right boundary
            w = np.zeros_like(u[i])
            w[0] = self.couple_left(i, u[i - 1][-1])
            u[i] = u[i] - T(i, w)
        return np.concatenate(u, axis=0)

    def exact_T_ops_two_fronts(self):
        """The exact Schur inverses of the two-front elimination: restrictions
        to D_i of H_{[0:i]}^{-1} (slabs left of c), H_{[i:l]}^{-1} (slabs right
        of c) and H^{-1} (the middle slab c)."""
        H = self.assemble_H().toarray()
        per = self.n_tot ** (self.m.ndim - 1)
        b, nl = self.b, self.n_slabs
        c = (nl - 1) // 2
        starts = [(self.slab_first[i] + b) * per for i in range(nl)]
        ends = [(self.slab_last[i] + b + 1) * per for i in range(nl)]
        inv = []
        for i in range(nl):
            if i < c:
                lo, hi = 0, ends[i]
            elif i > c:
                lo, hi = starts[i], H.shape[0]
            else:
                lo, hi = 0, H.shape[0]
            Hi = np.linalg.inv(H[lo:hi, lo:hi])
            inv.append(Hi[starts[i] - lo:ends[i] - lo, starts[i] - lo:ends[i] - lo])

        def T(i, v):
            return (inv[i] @ v.reshape(-1)).reshape(v.shape)
        return T


class Problem2D(_TwoFronts):
    """The 2D sparsified system and its sweeping preconditioner.

    Index convention: grid index (i1, i2) with i in I^{h+eta} = {-b..n+1+b}^2
    (b = b_pml); arrays over that set are stored at [i1+b, i2+b].  Vectors on
    I = {1..n}^2 are (n, n) arrays at [i1-1, i2-1].
    """

    def __init__(self, n: int, omega: float, m: np.ndarray, params: Params | None = None):
        self.p = params or Params()
        self.n, self.omega, self.m = n, float(omega), np.asarray(m, dtype=np.float64)
        self.h = 1.0 / (n + 1)
        self.b = self.p.b_pml
        self.b_aux = self.p.b_aux if self.p.b_aux is not None else self.b
        self.n_tot = n + 2 + 2 * self.b
        self.kw = nystrom_weights(2, n, omega, n)
        self.alpha, self.beta, self.sv = interior_stencils(2, n, omega)
        ns = self.p.n_samples if self.p.n_samples is not None else n
        self.samples = frequency_samples(self.m, self.omega, ns)
        self._gcache: dict = {}
        self._slabs()
        self._factor()

    # ---- sizes and coefficients -------------------------------------------------
    def m_at(self, i1: int, i2: int) -> float:
        n = self.n
        if 1 <= i1 <= n and 1 <= i2 <= n:
            return float(self.m[i1 - 1, i2 - 1])
        return 0.0

    def sigma(self, idx):
        return pml_sigma(idx, self.n, self.b, self.p.C, self.omega)

    def _gamma(self, key, omega_loc, s1, s2):
        g = self._gcache.get(key)
        if g is None:
            g = pml_stencil(omega_loc, self.h, [np.asarray(s1), np.asarray(s2)]).reshape(3, 3)
            self._gcache[key] = g
        return g

    def row(self, i1: int, i2: int) -> np.ndarray:
        """Coefficients c[da+1, db+1] of the row of H at (i1, i2) (Eq. sp_stc):
        on I^h:  conj(alpha_o) + omega^2 conj(beta_o) m_{i+o};
        on the PML points:  conj(gamma_i)  (global omega, physical sigma)."""
        n = self.n
        if 0 <= i1 <= n + 1 and 0 <= i2 <= n + 1:
            c = np.empty(9, dtype=np.complex128)
            for a, o in enumerate(neighbourhood_offsets(2)):
                c[a] = np.conj(self.alpha[a]) + self.omega ** 2 * np.conj(self.beta[a]) * \
                    self.m_at(i1 + o[0], i2 + o[1])
            return c.reshape(3, 3)
        s1 = self.sigma([i1 - 1, i1, i1 + 1])
        s2 = self.sigma([i2 - 1, i2, i2 + 1])
        return self._gamma(("phys", tuple(s1), tuple(s2)), self.omega, s1, s2)

    def aux_row(self, s: int, t: int, i2: int) -> np.ndarray:
        """Row of an auxiliary PML point t = 1..b_aux layers left of D_i (first
        layer s), at true position (s-t, i2) (Sec. 2.3, Eq. Hwv_approx).
        sigma along x1 is the left PML profile translated so that layer s plays
        the role of layer 0; sigma along x2 is the physical one; the local
        frequency is the sample nearest to omega^2 (1 - m(s-t, i2)).  The x1
        profile has the auxiliary width b_aux (eta = b_aux h)."""
        a1 = s - t
        s1 = pml_sigma(np.array([a1 - 1, a1, a1 + 1]) - s, self.n, self.b_aux, self.p.C, self.omega)
        s2 = self.sigma([i2 - 1, i2, i2 + 1])
        k = nearest_sample(self.samples, self.omega ** 2 * (1.0 - self.m_at(a1, i2)))
        return self._gamma(("aux", k, tuple(s1), tuple(s2)), math.sqrt(self.samples[k]), s1, s2)

    def aux_row_right(self, e: int, t: int, i2: int) -> np.ndarray:
        """Row of the auxiliary PML point t = 1..b_aux layers right of D_i's last
        layer e (two fronts), at true position (e+t, i2): the mirrored profile
        along x1, the physical sigma along x2, the sample nearest
        omega^2 (1 - m(e+t, i2))."""
        a1 = e + t
        s1 = self.right_sigma(e, a1)
        s2 = self.sigma([i2 - 1, i2, i2 + 1])
        k = nearest_sample(self.samples, self.omega ** 2 * (1.0 - self.m_at(a1, i2)))
        return self._gamma(("auxr", k, tuple(s1), tuple(s2)), math.sqrt(self.samples[k]), s1, s2)

    # ---- assembled H and f = Q r -------------------------------------------------
    def assemble_H(self) -> sp.csr_matrix:
        """H on I^{h+eta}, zero Dirichlet values on its boundary dropped (Eq. Huf)."""
        b, nt = self.b, self.n_tot
        rows, cols, vals = [], [], []
        for i1 in range(-b, self.n + 2 + b):
            for i2 in range(-b, self.n + 2 + b):
                c = self.row(i1, i2)
                r = (i1 + b) * nt + (i2 + b)
                for da in (-1, 0, 1):
                    for db in (-1, 0, 1):
                        j1, j2 = i1 + da, i2 + db
                        if -b <= j1 <= self.n + 1 + b and -b <= j2 <= self.n + 1 + b:
                            rows.append(r)
                            cols.append((j1 + b) * nt + (j2 + b))
                            vals.append(c[da + 1, db + 1])
        return sp.csr_matrix((vals, (rows, cols)), shape=(nt * nt, nt * nt))

    def sparsify_rhs(self, r: np.ndarray) -> np.ndarray:
        """f = Q r on I^{h+eta}: f_i = alpha^* r_{mu_i} on I^h, 0 on the PML
        (Eq. Huf; Algorithm 2 step 1), r zero-padded outside I."""
        n, b, nt = self.n, self.b, self.n_tot
        rp = np.zeros((n + 4, n + 4), dtype=np.complex128)     # indices -1..n+2
        rp[2:n + 2, 2:n + 2] = r
        f = np.zeros((nt, nt), dtype=np.complex128)
        ac = np.conj(self.alpha).reshape(3, 3)
        for da in (-1, 0, 1):
            for db in (-1, 0, 1):
                f[b:b + n + 2, b:b + n + 2] += ac[da + 1, db + 1] * \
                    rp[1 + da:n + 3 + da, 1 + db:n + 3 + db]
        return f

    # ---- slabs and subproblems ---------------------------------------------------
    def _slabs(self):
        """Slabs along x1 (Sec. 2.3): slab 1 = left PML + b_slab normal layers,
        middle slabs b_slab layers, the last slab the remaining normal layers +
        right PML.  READING: the remainder goes to the last slab."""
        n, b, bs = self.n, self.b, self.p.b_slab
        nl = -(-(n + 2) // bs)
        self.n_slabs = nl
        self.slab_first, self.slab_last = [], []
        for i in range(nl):
            lo = -b if i == 0 else i * bs
            hi = n + 1 + b if i == nl - 1 else (i + 1) * bs - 1
            self.slab_first.append(lo)
            self.slab_last.append(hi)

    def subproblem(self, i: int):
        """Matrix of the subproblem of slab i (0-based), Eq. (Hwv_approx).

        Unknowns: b_aux virtual auxiliary layers (x1 = s-b_aux..s-1) then the
        layers of D_i; for i = 0 there are no auxiliary layers (T~_1 = T_1).
        With two fronts the slabs from the middle one rightward take their
        b_aux auxiliary layers (x1 = e+1..e+b_aux) on the right instead (the
        middle slab on both sides).  Couplings leaving the layer set are
        dropped (zero Dirichlet values).  Returns (matrix, x1 list of layers,
        offset of D_i within the layers).
        """
        b, nt = self.b, self.n_tot
        s, e = self.slab_first[i], self.slab_last[i]
        left, right = self.aux_sides(i)
        aux = list(range(s - self.b_aux, s)) if left else []
        aux_r = list(range(e + 1, e + 1 + self.b_aux)) if right else []
        layers = aux + list(range(s, e + 1)) + aux_r
        pos = {x1: a for a, x1 in enumerate(layers)}
        rows, cols, vals = [], [], []
        for a, x1 in enumerate(layers):
            for i2 in range(-b, self.n + 2 + b):
                if x1 < s:
                    c = self.aux_row(s, s - x1, i2)
                elif x1 > e:
                    c = self.aux_row_right(e, x1 - e, i2)
                else:
                    c = self.row(x1, i2)
                r = a * nt + (i2 + b)
                for da in (-1, 0, 1):
                    ja = pos.get(x1 + da)
                    if ja is None:
                        continue
                    for db in (-1, 0, 1):
                        j2 = i2 + db
                        if -b <= j2 <= self.n + 1 + b:
                            rows.append(r)
                            cols.append(ja * nt + (j2 + b))
                            vals.append(c[da + 1, db + 1])
        M = sp.csr_matrix((vals, (rows, cols)), shape=(len(layers) * nt, len(layers) * nt))
        return M, layers, len(aux)

    def _factor(self):
        """Algorithm 1 steps 5-8: LU of every subproblem (sparse LU, partial pivoting)."""
        self.lu, self.n_aux, self.n_layers = [], [], []
        for i in range(self.n_slabs):
            M, layers, na = self.subproblem(i)
            self.lu.append(spla.splu(M.tocsc()))
            self.n_aux.append(na)
            self.n_layers.append(len(layers))

    def _T(self, i, v, trans):
        nt = self.n_tot
        na, nd = self.n_aux[i], v.shape[0]
        rhs = np.zeros((self.n_layers[i] * nt,), dtype=np.complex128)
        rhs[na * nt:(na + nd) * nt] = v.reshape(-1)
        w = self.lu[i].solve(rhs, trans=trans)
        return w[na * nt:(na + nd) * nt].reshape(v.shape)

    def T(self, i: int, v: np.ndarray) -> np.ndarray:
        """T~_i v: pad v (layers of D_i x n_tot) with zeros on the auxiliary
        layers, solve the subproblem, restrict to D_i (Eq. Hwv_approx)."""
        return self._T(i, v, "N")

    def T_transpose(self, i: int, v: np.ndarray) -> np.ndarray:
        return self._T(i, v, "T")

    def couple_left(self, i: int, u_prev_last: np.ndarray) -> np.ndarray:
        """H_{[i,i-1]} u_{[i-1]}: rows of D_i's first layer, x1-offset -1."""
        b, nt = self.b, self.n_tot
        s = self.slab_first[i]
        out = np.zeros(nt, dtype=np.complex128)
        for i2 in range(-b, self.n + 2 + b):
            c = self.row(s, i2)
            for db in (-1, 0, 1):
                j2 = i2 + db
                if -b <= j2 <= self.n + 1 + b:
                    out[i2 + b] += c[0, db + 1] * u_prev_last[j2 + b]
        return out

    def couple_right(self, i: int, u_next_first: np.ndarray) -> np.ndarray:
        """H_{[i,i+1]} u_{[i+1]}: rows of D_i's last layer, x1-offset +1."""
        b, nt = self.b, self.n_tot
        e = self.slab_last[i]
        out = np.zeros(nt, dtype=np.complex128)
        for i2 in range(-b, self.n + 2 + b):
            c = self.row(e, i2)
            for db in (-1, 0, 1):
                j2 = i2 + db
                if -b <= j2 <= self.n + 1 + b:
                    out[i2 + b] += c[2, db + 1] * u_next_first[j2 + b]
        return out

    def slab_view(self, f: np.ndarray, i: int) -> np.ndarray:
        b = self.b
        return f[self.slab_first[i] + b:self.slab_last[i] + b + 1]

    def sweep(self, f: np.ndarray, T=None) -> np.ndarray:
        """Algorithm 2 steps 3-9: forward then backward sweep with T~_i."""
        if self.p.fronts == 2:
            return self.sweep_two_fronts(f, T)
        T = T or self.T
        nl = self.n_slabs
        u = [None] * nl
        u[0] = T(0, self.slab_view(f, 0))
        for i in range(1, nl):
            v = self.slab_view(f, i).copy()
            v[0] -= self.couple_left(i, u[i - 1][-1])
            u[i] = T(i, v)
        for i in range(nl - 2, -1, -1):
            v = np.zeros_like(u[i])
            v[-1] = self.couple_right(i, u[i + 1][0])
            u[i] = u[i] - T(i, v)
        return np.concatenate(u, axis=0)

    def extract(self, ut: np.ndarray) -> np.ndarray:
        b, n = self.b, self.n
        return ut[b + 1:b + 1 + n, b + 1:b + 1 + n]

    def precondition(self, r: np.ndarray) -> np.ndarray:
        """P r: f = Q r, sweep, extract on I (Algorithm 2)."""
        return self.extract(self.sweep(self.sparsify_rhs(r)))

    def precondition_transpose(self, y: np.ndarray) -> np.ndarray:
        """P^T y = Q^T Sweep^T E^T y, with Sweep^T the two passes in reverse:
        z_1 = v_1, z_i = v_i - H_{[i-1,i]}^T T~_{i-1}^T z_{i-1};
        x_l = T~_l^T z_l, x_i = T~_i^T (z_i - H_{[i+1,i]}^T x_{i+1}).
        Written for one sweeping front."""
        if self.p.fronts != 1:
            raise ValueError("the transposed sweep is written for one front")
        b, n, nt = self.b, self.n, self.n_tot
        v = np.zeros((nt, nt), dtype=np.complex128)
        v[b + 1:b + 1 + n, b + 1:b + 1 + n] = y
        nl = self.n_slabs
        z = [self.slab_view(v, i).copy() for i in range(nl)]
        for i in range(1, nl):
            # H_{[i,i-1]} maps slab i-1's last layer into slab i's first-layer rows;
            # its transpose maps slab i's first-layer values back onto that layer.
            t = self.T_transpose(i - 1, z[i - 1])
            z[i][0] -= self._cr_T(i - 1, t)
        x = [None] * nl
        x[nl - 1] = self.T_transpose(nl - 1, z[nl - 1])
        for i in range(nl - 2, -1, -1):
            w = z[i].copy()
            w[-1] -= self._couple_right_T_from_next(i, x[i + 1][0])
            x[i] = self.T_transpose(i, w)
        ut = np.concatenate(x, axis=0)
        return self._sparsify_T(ut)

    def _cr_T(self, i, t):
        # (H_{[i,i+1]})^T t restricted to slab i+1's first layer, from t on slab i's layers
        b, nt = self.b, self.n_tot
        e = self.slab_last[i]
        out = np.zeros(nt, dtype=np.complex128)
        for i2 in range(-b, self.n + 2 + b):
            c = self.row(e, i2)
            for db in (-1, 0, 1):
                j2 = i2 + db
                if -b <= j2 <= self.n + 1 + b:
                    out[j2 + b] += c[2, db + 1] * t[-1][i2 + b]
        return out

    def _couple_right_T_from_next(self, i, x_next_first):
        # (H_{[i+1,i]})^T x_{i+1}: rows of D_{i+1}'s first layer, offset -1, transposed
        b, nt = self.b, self.n_tot
        s = self.slab_first[i + 1]
        out = np.zeros(nt, dtype=np.complex128)
        for i2 in range(-b, self.n + 2 + b):
            c = self.row(s, i2)
            for db in (-1, 0, 1):
                j2 = i2 + db
                if -b <= j2 <= self.n + 1 + b:
                    out[j2 + b] += c[0, db + 1] * x_next_first[i2 + b]
        return out

    def _sparsify_T(self, ut):
        """Q^T: f_i = sum_o conj(alpha_o) r_{i+o}, so (Q^T w)_j = sum_o conj(alpha_o) w_{j-o}
        over j in I."""
        b, n = self.b, self.n
        ac = np.conj(self.alpha).reshape(3, 3)
        out = np.zeros((n, n), dtype=np.complex128)
        for da in (-1, 0, 1):
            for db in (-1, 0, 1):
                out += ac[da + 1, db + 1] * ut[b + 1 - da:b + 1 + n - da, b + 1 - db:b + 1 + n - db]
        return out

    # ---- the exact Schur recursion (for pins) ----------------------------------
    def exact_T_ops(self):
        """T_[i] as the restriction of H_{[1:i,1:i]}^{-1} to D_i (Eq. Hwv), dense."""
        H = self.assemble_H().toarray()
        b, nt = self.b, self.n_tot
        ends = [(self.slab_last[i] + b + 1) * nt for i in range(self.n_slabs)]
        starts = [(self.slab_first[i] + b) * nt for i in range(self.n_slabs)]
        inv = []
        for i in range(self.n_slabs):
            Hi = H[:ends[i], :ends[i]]
            Ti = np.linalg.inv(Hi)[starts[i]:, starts[i]:]
            inv.append(Ti)

        def T(i, v):
            return (inv[i] @ v.reshape(-1)).reshape(v.shape)
        return T


# --------------------------------------------------------------------------
# Sec. 3.1: the same construction in 3D (27-point stencils, 26 directions)
# --------------------------------------------------------------------------


class Problem3D(_TwoFronts):
    """The 3D sparsified system and its non-recursive sweeping preconditioner
    (Sec. 3.1): alpha/beta on the 27-point neighbourhood, gamma annihilating the
    26 normalised directions of {-1,0,1}^3 minus 0, slabs of x1-layers (each a
    quasi-2D problem) swept exactly as in Algorithm 2.  Each slab subproblem is
    factored here by a sparse LU (partial pivoting); the paper's nested
    dissection is a different direct solver for the same subproblem.

    Index convention: grid index (i1, i2, i3) in I^{h+eta} = {-b..n+1+b}^3,
    stored at [i1+b, i2+b, i3+b]; vectors on I are (n, n, n) arrays at
    [i1-1, i2-1, i3-1].  A layer is the (n_tot, n_tot) plane of fixed x1.
    """

    def __init__(self, n: int, omega: float, m: np.ndarray, params: Params | None = None):
        self.p = params or Params()
        self.n, self.omega, self.m = n, float(omega), np.asarray(m, dtype=np.float64)
        self.h = 1.0 / (n + 1)
        self.b = self.p.b_pml
        self.b_aux = self.p.b_aux if self.p.b_aux is not None else self.b
        self.n_tot = n + 2 + 2 * self.b
        self.kw = nystrom_weights(3, n, omega, n)
        self.alpha, self.beta, self.sv = interior_stencils(3, n, omega)
        ns = self.p.n_samples if self.p.n_samples is not None else n
        self.samples = frequency_samples(self.m, self.omega, ns)
        self._gcache: dict = {}
        self._slabs()
        self._factor()
        if self.p.recursive:
            self._inner_factor()

    def m_at(self, i1: int, i2: int, i3: int) -> float:
        n = self.n
        if 1 <= i1 <= n and 1 <= i2 <= n and 1 <= i3 <= n:
            return float(self.m[i1 - 1, i2 - 1, i3 - 1])
        return 0.0

    def sigma(self, idx):
        return pml_sigma(idx, self.n, self.b, self.p.C, self.omega)

    def _gamma(self, key, omega_loc, s1, s2, s3):
        g = self._gcache.get(key)
        if g is None:
            g = pml_stencil(omega_loc, self.h, [np.asarray(s1), np.asarray(s2), np.asarray(s3)]).reshape(3, 3, 3)
            self._gcache[key] = g
        return g

    def row(self, i1: int, i2: int, i3: int) -> np.ndarray:
        """Coefficients c[d1+1, d2+1, d3+1] of H's row at (i1, i2, i3): on I^h
        conj(alpha_o) + omega^2 conj(beta_o) m_{i+o}; on the PML conj(gamma_i)."""
        n = self.n
        if 0 <= i1 <= n + 1 and 0 <= i2 <= n + 1 and 0 <= i3 <= n + 1:
            c = np.empty(27, dtype=np.complex128)
            for a, o in enumerate(neighbourhood_offsets(3)):
                c[a] = np.conj(self.alpha[a]) + self.omega ** 2 * np.conj(self.beta[a]) * \
                    self.m_at(i1 + o[0], i2 + o[1], i3 + o[2])
            return c.reshape(3, 3, 3)
        s1 = self.sigma([i1 - 1, i1, i1 + 1])
        s2 = self.sigma([i2 - 1, i2, i2 + 1])
        s3 = self.sigma([i3 - 1, i3, i3 + 1])
        return self._gamma(("phys", tuple(s1), tuple(s2), tuple(s3)), self.omega, s1, s2, s3)

    def aux_row(self, s: int, t: int, i2: int, i3: int) -> np.ndarray:
        """Row of the auxiliary PML point t layers left of D_i (first layer s),
        at true position (s-t, i2, i3): x1 profile of the left PML of width
        b_aux translated to end at layer s, physical sigma along x2 and x3,
        local frequency the sample nearest omega^2 (1 - m(s-t, i2, i3))."""
        a1 = s - t
        s1 = pml_sigma(np.array([a1 - 1, a1, a1 + 1]) - s, self.n, self.b_aux, self.p.C, self.omega)
        s2 = self.sigma([i2 - 1, i2, i2 + 1])
        s3 = self.sigma([i3 - 1, i3, i3 + 1])
        k = nearest_sample(self.samples, self.omega ** 2 * (1.0 - self.m_at(a1, i2, i3)))
        return self._gamma(("aux", k, tuple(s1), tuple(s2), tuple(s3)), math.sqrt(self.samples[k]), s1, s2, s3)

    def aux_row_right(self, e: int, t: int, i2: int, i3: int) -> np.ndarray:
        """Row of the auxiliary PML point t layers right of D_i's last layer e
        (two fronts): the mirrored profile along x1."""
        a1 = e + t
        s1 = self.right_sigma(e, a1)
        s2 = self.sigma([i2 - 1, i2, i2 + 1])
        s3 = self.sigma([i3 - 1, i3, i3 + 1])
        k = nearest_sample(self.samples, self.omega ** 2 * (1.0 - self.m_at(a1, i2, i3)))
        return self._gamma(("auxr", k, tuple(s1), tuple(s2), tuple(s3)), math.sqrt(self.samples[k]), s1, s2,
                           s3)

    def _range(self):
        return range(-self.b, self.n + 2 + self.b)

    def assemble_H(self) -> sp.csr_matrix:
        """H on I^{h+eta}, zero Dirichlet values on its boundary dropped."""
        b, nt, lo, hi = self.b, self.n_tot, -self.b, self.n + 1 + self.b
        rows, cols, vals = [], [], []
        for i1 in self._range():
            for i2 in self._range():
                for i3 in self._range():
                    c = self.row(i1, i2, i3)
                    r = ((i1 + b) * nt + (i2 + b)) * nt + (i3 + b)
                    for o in neighbourhood_offsets(3):
                        j = (i1 + o[0], i2 + o[1], i3 + o[2])
                        if all(lo <= v <= hi for v in j):
                            rows.append(r)
                            cols.append(((j[0] + b) * nt + (j[1] + b)) * nt + (j[2] + b))
                            vals.append(c[o[0] + 1, o[1] + 1, o[2] + 1])
        return sp.csr_matrix((vals, (rows, cols)), shape=(nt ** 3, nt ** 3))

    def sparsify_rhs(self, r: np.ndarray) -> np.ndarray:
        """f = Q r: f_i = alpha^* r_{mu_i} on I^h, 0 on the PML, r zero off I."""
        n, b, nt = self.n, self.b, self.n_tot
        rp = np.zeros((n + 4,) * 3, dtype=np.complex128)     # indices -1..n+2
        rp[2:n + 2, 2:n + 2, 2:n + 2] = r
        f = np.zeros((nt,) * 3, dtype=np.complex128)
        ac = np.conj(self.alpha).reshape(3, 3, 3)
        for o in neighbourhood_offsets(3):
            f[b:b + n + 2, b:b + n + 2, b:b + n + 2] += ac[o[0] + 1, o[1] + 1, o[2] + 1] * \
                rp[1 + o[0]:n + 3 + o[0], 1 + o[1]:n + 3 + o[1], 1 + o[2]:n + 3 + o[2]]
        return f

    def _slabs(self):
        """Slabs of x1-layers, exactly as in 2D (Sec. 3.1, Sec. 2.3)."""
        n, b, bs = self.n, self.b, self.p.b_slab
        nl = -(-(n + 2) // bs)
        self.n_slabs = nl
        self.slab_first, self.slab_last = [], []
        for i in range(nl):
            self.slab_first.append(-b if i == 0 else i * bs)
            self.slab_last.append(n + 1 + b if i == nl - 1 else (i + 1) * bs - 1)

    def subproblem(self, i: int):
        """Matrix of slab i's subproblem (Eq. Hwv_approx in 3D): b_aux virtual
        auxiliary layers then D_i's layers (none for the first slab), and with
        two fronts the right-side auxiliary layers of the slabs from the middle
        one rightward; couplings leaving the layer set are dropped.  Returns
        (matrix, layers, n_aux)."""
        b, nt, lo, hi = self.b, self.n_tot, -self.b, self.n + 1 + self.b
        s, e = self.slab_first[i], self.slab_last[i]
        left, right = self.aux_sides(i)
        aux = list(range(s - self.b_aux, s)) if left else []
        aux_r = list(range(e + 1, e + 1 + self.b_aux)) if right else []
        layers = aux + list(range(s, e + 1)) + aux_r
        pos = {x1: a for a, x1 in enumerate(layers)}
        rows, cols, vals = [], [], []
        for a, x1 in enumerate(layers):
            for i2 in self._range():
                for i3 in self._range():
                    if x1 < s:
                        c = self.aux_row(s, s - x1, i2, i3)
                    elif x1 > e:
                        c = self.aux_row_right(e, x1 - e, i2, i3)
                    else:
                        c = self.row(x1, i2, i3)
                    r = (a * nt + (i2 + b)) * nt + (i3 + b)
                    for o in neighbourhood_offsets(3):
                        ja = pos.get(x1 + o[0])
                        j2, j3 = i2 + o[1], i3 + o[2]
                        if ja is None or not (lo <= j2 <= hi and lo <= j3 <= hi):
                            continue
                        rows.append(r)
                        cols.append((ja * nt + (j2 + b)) * nt + (j3 + b))
                        vals.append(c[o[0] + 1, o[1] + 1, o[2] + 1])
        sz = len(layers) * nt * nt
        return sp.csr_matrix((vals, (rows, cols)), shape=(sz, sz)), layers, len(aux)

    def _factor(self):
        """Algorithm 1 in 3D: an LU of every slab subproblem (not needed by the
        recursive approach, which sweeps each subproblem instead)."""
        self.lu, self.n_aux, self.n_layers, self.slab_layers = [], [], [], []
        for i in range(self.n_slabs):
            M, layers, na = self.subproblem(i)
            self.lu.append(None if self.p.recursive else spla.splu(M.tocsc()))
            self.n_aux.append(na)
            self.n_layers.append(len(layers))
            self.slab_layers.append(layers)

    def _T(self, i, v, trans):
        nt2 = self.n_tot ** 2
        na, nd = self.n_aux[i], v.shape[0]
        rhs = np.zeros((self.n_layers[i] * nt2,), dtype=np.complex128)
        rhs[na * nt2:(na + nd) * nt2] = v.reshape(-1)
        w = self.lu[i].solve(rhs, trans=trans)
        return w[na * nt2:(na + nd) * nt2].reshape(v.shape)

    def T(self, i: int, v: np.ndarray) -> np.ndarray:
        """T~_i v: zero auxiliary layers, solve, restrict to D_i (with the
        recursive approach the solve is the inner sweep along x2)."""
        if self.p.recursive:
            return self.T_recursive(i, v)
        return self._T(i, v, "N")

    def T_transpose(self, i: int, v: np.ndarray) -> np.ndarray:
        if self.p.recursive:
            raise ValueError("the transposed sweep is written for the non-recursive approach")
        return self._T(i, v, "T")

    # ---- the recursive approach (Sec. 3.1): each quasi-2D slab subproblem S_i
    # swept along x2 into quasi-1D sub-slab subproblems, padded with auxiliary
    # PML along x2 exactly as the slabs are along x1.  The sub-slabs E_j use the
    # same partition of x2 as the slabs D_i use of x1.
    def sigma1_of(self, i: int, x1: int) -> np.ndarray:
        """sigma along x1 at x1-1, x1, x1+1 for a layer of slab i's subproblem:
        the auxiliary profile on its auxiliary layers, else the physical one."""
        s, e = self.slab_first[i], self.slab_last[i]
        idx = np.array([x1 - 1, x1, x1 + 1])
        if x1 < s:
            return pml_sigma(idx - s, self.n, self.b_aux, self.p.C, self.omega)
        if x1 > e:
            return self.right_sigma(e, x1)
        return self.sigma(idx)

    def slab_row(self, i: int, x1: int, i2: int, i3: int) -> np.ndarray:
        """Row of slab i's subproblem S_i at (x1, i2, i3)."""
        s, e = self.slab_first[i], self.slab_last[i]
        if x1 < s:
            return self.aux_row(s, s - x1, i2, i3)
        if x1 > e:
            return self.aux_row_right(e, x1 - e, i2, i3)
        return self.row(x1, i2, i3)

    def inner_aux_row(self, i: int, x1: int, f: int, t: int, i3: int) -> np.ndarray:
        """Row of an inner auxiliary point t = 1..b_aux x2-layers before the
        first x2-layer f of a sub-slab, at (x1, f-t, i3) of slab i's
        subproblem: along x2 the left profile of width b_aux translated so that
        f plays the role of index 0, along x1 the layer's own profile, along x3
        the physical one; local frequency the sample nearest omega^2 (1 - m)."""
        a2 = f - t
        s1 = self.sigma1_of(i, x1)
        s2 = pml_sigma(np.array([a2 - 1, a2, a2 + 1]) - f, self.n, self.b_aux, self.p.C, self.omega)
        s3 = self.sigma([i3 - 1, i3, i3 + 1])
        k = nearest_sample(self.samples, self.omega ** 2 * (1.0 - self.m_at(x1, a2, i3)))
        return self._gamma(("aux2", k, tuple(s1), tuple(s2), tuple(s3)), math.sqrt(self.samples[k]), s1, s2, s3)

    def inner_subproblem(self, i: int, j: int):
        """Matrix of sub-slab j of slab i: x1 over slab i's subproblem layers,
        x2 over b_aux auxiliary layers (none for j = 0) then E_j, x3 over the
        whole range; rows on E_j are S_i's, rows on the auxiliary layers are
        inner_aux_row's; couplings leaving the set are dropped.  Unknown order
        (x1 layer, x2 layer, x3).  Returns (matrix, x2 list, n_aux2)."""
        b, nt, lo, hi = self.b, self.n_tot, -self.b, self.n + 1 + self.b
        layers1 = self.slab_layers[i]
        f, e2 = self.slab_first[j], self.slab_last[j]
        aux2 = list(range(f - self.b_aux, f)) if j > 0 else []
        x2s = aux2 + list(range(f, e2 + 1))
        p1 = {x: a for a, x in enumerate(layers1)}
        p2 = {x: a for a, x in enumerate(x2s)}
        n2 = len(x2s)
        rows, cols, vals = [], [], []
        for a1, x1 in enumerate(layers1):
            for a2, x2 in enumerate(x2s):
                for i3 in self._range():
                    c = self.inner_aux_row(i, x1, f, f - x2, i3) if x2 < f else self.slab_row(i, x1, x2, i3)
                    r = (a1 * n2 + a2) * nt + (i3 + b)
                    for o in neighbourhood_offsets(3):
                        j1, j2, j3 = p1.get(x1 + o[0]), p2.get(x2 + o[1]), i3 + o[2]
                        if j1 is None or j2 is None or not (lo <= j3 <= hi):
                            continue
                        rows.append(r)
                        cols.append((j1 * n2 + j2) * nt + (j3 + b))
                        vals.append(c[o[0] + 1, o[1] + 1, o[2] + 1])
        sz = len(layers1) * n2 * nt
        return sp.csr_matrix((vals, (rows, cols)), shape=(sz, sz)), x2s, len(aux2)

    def _inner_factor(self):
        """A sparse LU of every sub-slab subproblem, and each slab's S_i (for the
        couplings between its sub-slabs)."""
        self.inner_lu, self.inner_na = [], []
        self.S = []
        for i in range(self.n_slabs):
            self.S.append(self.subproblem(i)[0].tocsr())
            lus, nas = [], []
            for j in range(self.n_slabs):
                M, x2s, na2 = self.inner_subproblem(i, j)
                lus.append(spla.splu(M.tocsc()))
                nas.append(na2)
            self.inner_lu.append(lus)
            self.inner_na.append(nas)

    def _Tinner(self, i: int, j: int, v: np.ndarray) -> np.ndarray:
        """T~_{i,j} v: v on (x1 layers of S_i, E_j, x3), zero on the auxiliary
        x2-layers, solve, restrict to E_j."""
        L1, nd, nt = v.shape
        na2 = self.inner_na[i][j]
        rhs = np.zeros((L1, na2 + nd, nt), dtype=np.complex128)
        rhs[:, na2:] = v
        w = self.inner_lu[i][j].solve(rhs.reshape(-1)).reshape(rhs.shape)
        return w[:, na2:]

    def _inner_couple(self, i: int, j: int, side: int, plane: np.ndarray) -> np.ndarray:
        """S_i's coupling of sub-slab j's first (side -1) or last (side +1)
        x2-layer with the neighbouring x2-layer, applied to that layer's values
        plane (x1 layers of S_i, x3)."""
        b, nt = self.b, self.n_tot
        L1 = len(self.slab_layers[i])
        x2r = self.slab_first[j] if side < 0 else self.slab_last[j]
        x2c = x2r + side
        a1 = np.arange(L1)[:, None]
        i3 = np.arange(nt)[None, :]
        r_idx = ((a1 * nt + (x2r + b)) * nt + i3).reshape(-1)
        c_idx = ((a1 * nt + (x2c + b)) * nt + i3).reshape(-1)
        return (self.S[i][r_idx][:, c_idx] @ plane.reshape(-1)).reshape(L1, nt)

    def inner_sweep(self, i: int, V: np.ndarray, T=None) -> np.ndarray:
        """Algorithm 2 along x2 on slab i's subproblem: V on (x1 layers of S_i,
        x2, x3); forward then backward over the sub-slabs with T~_{i,j}."""
        T = T or (lambda j, v: self._Tinner(i, j, v))
        b = self.b
        nl = self.n_slabs
        E = [slice(self.slab_first[j] + b, self.slab_last[j] + b + 1) for j in range(nl)]
        u = [None] * nl
        for j in range(nl):
            v = V[:, E[j], :].copy()
            if j > 0:
                v[:, 0, :] -= self._inner_couple(i, j, -1, u[j - 1][:, -1, :])
            u[j] = T(j, v)
        for j in range(nl - 2, -1, -1):
            w = np.zeros_like(u[j])
            w[:, -1, :] = self._inner_couple(i, j, +1, u[j + 1][:, 0, :])
            u[j] = u[j] - T(j, w)
        return np.concatenate(u, axis=1)

    def T_recursive(self, i: int, v: np.ndarray, T=None) -> np.ndarray:
        """The recursive approach's T~_i v: pad v with zeros on the auxiliary
        x1-layers, apply the inner sweep, restrict to D_i."""
        nt = self.n_tot
        na, nd = self.n_aux[i], v.shape[0]
        V = np.zeros((self.n_layers[i], nt, nt), dtype=np.complex128)
        V[na:na + nd] = v
        return self.inner_sweep(i, V, T)[na:na + nd]

    def exact_inner_ops(self, i: int):
        """The exact Schur inverses of slab i's inner elimination: restrictions
        to E_j of (S_i restricted to x2 <= last x2-layer of E_j)^{-1}."""
        b, nt = self.b, self.n_tot
        S = self.S[i].toarray()
        L1 = len(self.slab_layers[i])
        ops = []
        for j in range(self.n_slabs):
            keep = np.array([(a1 * nt + x2) * nt + x3 for a1 in range(L1) for x2 in range(self.slab_last[j] + b + 1)
                             for x3 in range(nt)])
            Sinv = np.linalg.inv(S[np.ix_(keep, keep)])
            x2j = range(self.slab_first[j] + b, self.slab_last[j] + b + 1)
            pos = {k: q for q, k in enumerate(keep)}
            sel = np.array([pos[(a1 * nt + x2) * nt + x3] for a1 in range(L1) for x2 in x2j for x3 in range(nt)])
            ops.append(Sinv[np.ix_(sel, sel)])

        def T(j, v):
            return (ops[j] @ v.reshape(-1)).reshape(v.shape)
        return T

    def _layer_coupling(self, x1: int, plane: np.ndarray, side: int, transpose: bool) -> np.ndarray:
        """Apply the x1-offset `side` (-1 or +1) part of the rows of layer x1 to
        the neighbouring layer's values `plane` (or its transpose)."""
        b, nt, lo, hi = self.b, self.n_tot, -self.b, self.n + 1 + self.b
        out = np.zeros((nt, nt), dtype=np.complex128)
        for i2 in self._range():
            for i3 in self._range():
                c = self.row(x1, i2, i3)[side + 1]
                for d2 in (-1, 0, 1):
                    for d3 in (-1, 0, 1):
                        j2, j3 = i2 + d2, i3 + d3
                        if lo <= j2 <= hi and lo <= j3 <= hi:
                            if transpose:
                                out[j2 + b, j3 + b] += c[d2 + 1, d3 + 1] * plane[i2 + b, i3 + b]
                            else:
                                out[i2 + b, i3 + b] += c[d2 + 1, d3 + 1] * plane[j2 + b, j3 + b]
        return out

    def couple_left(self, i, u_prev_last):
        """H_{[i,i-1]} u_{[i-1]}: rows of D_i's first layer, x1-offset -1."""
        return self._layer_coupling(self.slab_first[i], u_prev_last, -1, False)

    def couple_right(self, i, u_next_first):
        """H_{[i,i+1]} u_{[i+1]}: rows of D_i's last layer, x1-offset +1."""
        return self._layer_coupling(self.slab_last[i], u_next_first, +1, False)

    def slab_view(self, f, i):
        b = self.b
        return f[self.slab_first[i] + b:self.slab_last[i] + b + 1]

    def sweep(self, f, T=None):
        """Algorithm 2 (forward then backward sweep) on 3D slabs."""
        if self.p.fronts == 2:
            return self.sweep_two_fronts(f, T)
        T = T or self.T
        nl = self.n_slabs
        u = [None] * nl
        u[0] = T(0, self.slab_view(f, 0))
        for i in range(1, nl):
            v = self.slab_view(f, i).copy()
            v[0] -= self.couple_left(i, u[i - 1][-1])
            u[i] = T(i, v)
        for i in range(nl - 2, -1, -1):
            v = np.zeros_like(u[i])
            v[-1] = self.couple_right(i, u[i + 1][0])
            u[i] = u[i] - T(i, v)
        return np.concatenate(u, axis=0)

    def extract(self, ut):
        b, n = self.b, self.n
        return ut[b + 1:b + 1 + n, b + 1:b + 1 + n, b + 1:b + 1 + n]

    def precondition(self, r):
        """P r: f = Q r, sweep, extract on I."""
        return self.extract(self.sweep(self.sparsify_rhs(r)))

    def precondition_transpose(self, y):
        """P^T y = Q^T Sweep^T E^T y, the two passes of the sweep transposed
        and taken in reverse (as in 2D).  Written for one sweeping front."""
        if self.p.fronts != 1:
            raise ValueError("the transposed sweep is written for one front")
        b, n, nt = self.b, self.n, self.n_tot
        v = np.zeros((nt,) * 3, dtype=np.complex128)
        v[b + 1:b + 1 + n, b + 1:b + 1 + n, b + 1:b + 1 + n] = y
        nl = self.n_slabs
        z = [self.slab_view(v, i).copy() for i in range(nl)]
        for i in range(1, nl):
            # H_{[i-1,i]}^T: slab i-1's last-layer rows (x1-offset +1), transposed
            t = self.T_transpose(i - 1, z[i - 1])
            z[i][0] -= self._layer_coupling(self.slab_last[i - 1], t[-1], +1, True)
        x = [None] * nl
        x[nl - 1] = self.T_transpose(nl - 1, z[nl - 1])
        for i in range(nl - 2, -1, -1):
            # H_{[i+1,i]}^T: slab i+1's first-layer rows (x1-offset -1), transposed
            w = z[i].copy()
            w[-1] -= self._layer_coupling(self.slab_first[i + 1], x[i + 1][0], -1, True)
            x[i] = self.T_transpose(i, w)
        ut = np.concatenate(x, axis=0)
        ac = np.conj(self.alpha).reshape(3, 3, 3)
        out = np.zeros((n, n, n), dtype=np.complex128)
        for o in neighbourhood_offsets(3):
            out += ac[o[0] + 1, o[1] + 1, o[2] + 1] * \
                ut[b + 1 - o[0]:b + 1 + n - o[0], b + 1 - o[1]:b + 1 + n - o[1], b + 1 - o[2]:b + 1 + n - o[2]]
        return out

    def exact_T_ops(self):
        """T_[i] as the restriction of H_{[1:i,1:i]}^{-1} to D_i (Eq. Hwv), dense."""
        H = self.assemble_H().toarray()
        b, nt2 = self.b, self.n_tot ** 2
        inv = []
        for i in range(self.n_slabs):
            e = (self.slab_last[i] + b + 1) * nt2
            s0 = (self.slab_first[i] + b) * nt2
            inv.append(np.linalg.inv(H[:e, :e])[s0:, s0:])

        def T(i, v):
            return (inv[i] @ v.reshape(-1)).reshape(v.shape)
        return T


# --------------------------------------------------------------------------
# GMRES (Sec. 2.5: standard restarted GMRES, relative tolerance)
# --------------------------------------------------------------------------


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    relres_est: float
    history: list


def gmres(apply_A, apply_P, g: np.ndarray, restart: int = 30, tol: float = 1e-8,
          max_iter: int = 500) -> GmresResult:
    """Right-preconditioned restarted GMRES, MGS Arnoldi, Givens rotations.
    x0 = 0; stops when the Givens residual |rho_{j+1}| <= tol ||g||.
    The iteration count is the total number of Arnoldi steps."""
    shape = g.shape
    b = g.reshape(-1)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return GmresResult(x.reshape(shape), 0, 0.0, [])
    r = b.copy()
    total = 0
    hist = []
    while True:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, b.size), dtype=np.complex128)
        Hm = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        rho = np.zeros(restart + 1, dtype=np.complex128)
        rho[0] = beta
        V[0] = r / beta
        k = 0
        done = False
        for j in range(restart):
            w = apply_A(apply_P(V[j].reshape(shape))).reshape(-1)
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -np.conj(sn[i]) * Hm[i, j] + np.conj(cs[i]) * Hm[i + 1, j]
                Hm[i, j] = t
            a_, b_ = Hm[j, j], Hm[j + 1, j]
            den = math.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            cs[j] = a_ / den if den != 0 else 1.0
            sn[j] = b_ / den if den != 0 else 0.0
            # rotation [[c, s], [-conj(s), conj(c)]] with c = a/den, s = b/den
            cs[j], sn[j] = np.conj(cs[j]), np.conj(sn[j])
            Hm[j, j] = cs[j] * a_ + sn[j] * b_
            Hm[j + 1, j] = 0.0
            rho[j + 1] = -np.conj(sn[j]) * rho[j]
            rho[j] = cs[j] * rho[j]
            total += 1
            k = j + 1
            hist.append(abs(rho[j + 1]) / bnorm)
            if abs(rho[j + 1]) <= tol * bnorm or total >= max_iter:
                done = True
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (rho[i] - Hm[i, i + 1:k] @ y[i + 1:k]) / Hm[i, i]
        x = x + apply_P((y @ V[:k]).reshape(shape)).reshape(-1)
        if done:
            break
        r = b - apply_A(x.reshape(shape)).reshape(-1)
    return GmresResult(x.reshape(shape), total, hist[-1] if hist else 0.0, hist)


# --------------------------------------------------------------------------
# End-to-end solve (Algorithms 1 and 2 + GMRES)
# --------------------------------------------------------------------------


def make_problem(n, omega, m, params: Params | None = None):
    """Problem2D or Problem3D by the dimension of m."""
    m = np.asarray(m)
    return (Problem3D if m.ndim == 3 else Problem2D)(n, omega, m, params)


def solve(n, omega, m, direction, params: Params | None = None, restart=30, tol=1e-8,
          max_iter=500, problem=None):
    """Scattered field u on I for one incident plane wave."""
    pb = problem or make_problem(n, omega, m, params)
    g = ls_rhs(m, omega, pb.kw, direction)
    A = lambda u: ls_apply(u, m, omega, pb.kw)  # noqa: E731
    res = gmres(A, pb.precondition, g, restart, tol, max_iter)
    gn = np.linalg.norm(g)
    relres = np.linalg.norm(g - A(res.x)) / gn if gn > 0 else 0.0
    return res, relres, pb, g


def dense_ls_matrix(n, omega, m, kw):
    """I + omega^2 K M as a dense matrix (pins on tiny grids)."""
    shape = np.asarray(m).shape
    N = int(np.prod(shape))
    A = np.zeros((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        A[:, j] = ls_apply(e.reshape(shape), m, omega, kw).reshape(-1)
    return A


# --------------------------------------------------------------------------
# Gradient of a receiver misfit with respect to m (adjoint of Eq. LS_d)
# --------------------------------------------------------------------------


def misfit(n, omega, m, dirs, receivers, data, kw=None):
    """L = 1/2 sum_s sum_r |u_s(receiver r) - d_{s,r}|^2, u_s the scattered field
    of the plane wave with direction dirs[s], solved densely (tiny grids).
    receivers: integer grid indices into the (n,)*d arrays, shape (n_rcv, d)."""
    kw = kw if kw is not None else nystrom_weights(np.asarray(m).ndim, n, omega, n)
    A = dense_ls_matrix(n, omega, m, kw)
    idx = tuple(np.asarray(receivers).T)
    L = 0.0
    for s, d in enumerate(dirs):
        g = ls_rhs(m, omega, kw, d)
        u = np.linalg.solve(A, g.reshape(-1)).reshape(g.shape)
        L += 0.5 * float(np.sum(np.abs(u[idx] - data[s]) ** 2))
    return L


def misfit_gradient_dense(n, omega, m, dirs, receivers, data, kw=None):
    """dL/dm by the dense adjoint: with A = I + omega^2 K M and g = -omega^2 K M u_I
    (Eq. LS_d), A du/dm_x = -omega^2 K e_x (u + u_I)_x; so with
    A^T lambda = R^T conj(u(receivers) - d) (R = restriction to the receivers),
    dL/dm_x = Re(-omega^2 (K lambda)_x (u + u_I)_x), summed over the waves."""
    m = np.asarray(m, dtype=np.float64)
    kw = kw if kw is not None else nystrom_weights(m.ndim, n, omega, n)
    A = dense_ls_matrix(n, omega, m, kw)
    idx = tuple(np.asarray(receivers).T)
    grad = np.zeros(m.shape)
    one = np.ones_like(m)
    for s, d in enumerate(dirs):
        uI = plane_wave(n, omega, d)
        g = ls_rhs(m, omega, kw, d)
        u = np.linalg.solve(A, g.reshape(-1)).reshape(g.shape)
        rt = np.zeros(m.shape, dtype=np.complex128)
        np.add.at(rt, idx, np.conj(u[idx] - data[s]))
        lam = np.linalg.solve(A.T, rt.reshape(-1)).reshape(m.shape)
        Klam_w2 = ls_apply(lam, one, omega, kw) - lam           # omega^2 K lambda
        grad += np.real(-Klam_w2 * (u + uI))
    return grad


# --------------------------------------------------------------------------
# Sec. 4: the sparsifying scheme as a direct discretization of Helmholtz
# --------------------------------------------------------------------------


def helmholtz_rhs(pb, f):
    """F = beta^* f_{mu_i} on I^h, 0 on the PML, f zero off I (Sec. 4: the
    right-hand side of alpha^* u_{mu_i} = beta^* f_{mu_i}).  2D grid (n_tot, n_tot)."""
    n, b, nt = pb.n, pb.b, pb.n_tot
    fp = np.zeros((n + 4, n + 4), dtype=np.complex128)     # indices -1..n+2
    fp[2:n + 2, 2:n + 2] = f
    F = np.zeros((nt, nt), dtype=np.complex128)
    bc = np.conj(pb.beta).reshape(3, 3)
    for da in (-1, 0, 1):
        for db in (-1, 0, 1):
            F[b:b + n + 2, b:b + n + 2] += bc[da + 1, db + 1] * fp[1 + da:n + 3 + da, 1 + db:n + 3 + db]
    return F


def helmholtz_direct(pb, f):
    """Solve the sparsified system H u~ = beta^* f (Sec. 4) exactly (sparse LU)
    for a source f on I; H has the alpha rows (with the medium's beta terms,
    so a medium m gives the heterogeneous equation) and the PML rows.
    Returns u on I and the full grid solution."""
    H = pb.assemble_H().tocsc()
    F = helmholtz_rhs(pb, f)
    ut = spla.spsolve(H, F.reshape(-1)).reshape(F.shape)
    return pb.extract(ut), ut


def delta_source(n, point):
    """Discrete delta of unit mass at the grid point `point` (indices 1..n):
    f = 1/h^2 there, 0 elsewhere."""
    h = 1.0 / (n + 1)
    f = np.zeros((n, n), dtype=np.complex128)
    f[point[0] - 1, point[1] - 1] = 1.0 / (h * h)
    return f
