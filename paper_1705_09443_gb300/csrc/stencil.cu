// PML stencils gamma (Sec. 2.2.2, Eq. gamma), assembly of the slab
// subproblems (Sec. 2.2.3, Sec. 2.3, Eq. Hwv_approx) and the sparsifying map
// f = Q r (Eq. Huf; Algorithm 2 step 1).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

struct StencilArgs {
    double2 a_conj[9];   // conj(alpha_o)
    double2 b_conj[9];   // conj(beta_o)
};

// sigma at grid index q of the physical profile (eta = b h): left of -1 the
// quadratic -(C/omega)((q+1)/b)^2, right of n+2 the mirror (C/omega)((q-n-2)/b)^2,
// zero in between; the Dirichlet layers take the same formula.
__device__ __forceinline__ double sigma_phys(int q, int n, int b, double Cw) {
    if (q <= -1) { const double t = (q + 1.0) / b; return -Cw * t * t; }
    if (q >= n + 2) { const double t = (q - n - 2.0) / b; return Cw * t * t; }
    return 0.0;
}

// Null vector of F^T for a 9 x 8 complex F (gamma^* F = 0): last column of the
// unitary factor of a Householder QR of F.  Returns conj(gamma), unit norm,
// centre entry real positive.  R: working precision (double, or float for the
// moving-PML stencils of the single-precision preconditioner).
template <typename R>
__device__ void gamma_from_F(cx<R> F[9][8], double2 out[9]) {
    using C = cx<R>;
    R vn2[8];
    for (int k = 0; k < 8; ++k) {
        R nx = 0;
        for (int i = k; i < 9; ++i) nx += cabs2(F[i][k]);
        nx = sqrt(nx);
        const C fkk = F[k][k];
        const R afk = sqrt(cabs2(fkk));
        const C ph = afk > 0 ? mk(fkk.x / afk, fkk.y / afk) : mk(R(1), R(0));
        const C alpha = mk(-ph.x * nx, -ph.y * nx);
        F[k][k] = fkk - alpha;  // v stored in column k, rows k..8
        R v2 = 0;
        for (int i = k; i < 9; ++i) v2 += cabs2(F[i][k]);
        vn2[k] = v2;
        if (v2 == 0) continue;
        for (int j = k + 1; j < 8; ++j) {
            C dot = czero<C>();
            for (int i = k; i < 9; ++i) dot = cfma_conj(F[i][k], F[i][j], dot);
            const R sc = R(2) / v2;
            for (int i = k; i < 9; ++i) F[i][j] = F[i][j] - (sc * dot) * F[i][k];
        }
    }
    C q[9];
    for (int i = 0; i < 9; ++i) q[i] = czero<C>();
    q[8] = mk(R(1), R(0));
    for (int k = 7; k >= 0; --k) {
        if (vn2[k] == 0) continue;
        C dot = czero<C>();
        for (int i = k; i < 9; ++i) dot = cfma_conj(F[i][k], q[i], dot);
        const R sc = R(2) / vn2[k];
        for (int i = k; i < 9; ++i) q[i] = q[i] - (sc * dot) * F[i][k];
    }
    R nq = 0;
    for (int i = 0; i < 9; ++i) nq += cabs2(q[i]);
    nq = sqrt(nq);
    const R a4 = sqrt(cabs2(q[4]));
    const C ph = mk(q[4].x / a4, -q[4].y / a4);  // |q4| / q4
    for (int i = 0; i < 9; ++i) {
        C g = (R(1) / nq) * (q[i] * ph);
        if (i == 4) g = mk(a4 / nq, R(0));
        out[i] = mk((double)g.x, -(double)g.y);   // conj(gamma)
    }
}

// Stencil for stretch triples s1, s2 (sigma at offsets -1, 0, +1 along x1, x2)
// and local frequency w: F[o][r] = exp(i w r.(dp_o + i dsigma_o)) over the
// 8 normalised neighbour directions r.  The exponential factors into an x1
// and an x2 part, E1(da, sc ra) E2(db, sc rb) with E(d, v) = exp(i w v (d h +
// i dsigma_d)), and E(d, -v) has the conjugate phase and the reciprocal
// modulus of E(d, v): 2 x 3 x 2 complex exponentials give all 72 entries.
template <typename R>
__device__ void pml_stencil(const double s1[3], const double s2[3], double w, double h, double2 out[9]) {
    using C = cx<R>;
    const R is2 = R(0.70710678118654752440);
    // E[axis][d + 1][scale][sign]: scale 0 -> v = 1, 1 -> v = 1/sqrt(2); sign 0 -> +v, 1 -> -v
    C E[2][3][2][2];
    for (int ax = 0; ax < 2; ++ax) {
        const double* sg = ax == 0 ? s1 : s2;
        for (int d = -1; d <= 1; ++d) {
            const R re = R(d * h), im = R(sg[d + 1] - sg[1]);
            for (int sc = 0; sc < 2; ++sc) {
                const R v = sc ? is2 : R(1);
                R sn, cs;
                sincos(R(w) * v * re, &sn, &cs);
                const R mag = exp(-R(w) * v * im);
                const R inv = R(1) / mag;
                E[ax][d + 1][sc][0] = mk(mag * cs, mag * sn);
                E[ax][d + 1][sc][1] = mk(inv * cs, -inv * sn);
            }
        }
    }
    C F[9][8];
    for (int o = 0; o < 9; ++o) {
        const int da = o / 3 - 1, db = o % 3 - 1;
        int col = 0;
        for (int ra = -1; ra <= 1; ++ra)
            for (int rb = -1; rb <= 1; ++rb) {
                if (ra == 0 && rb == 0) continue;
                const int sc = (ra != 0 && rb != 0) ? 1 : 0;
                const C e1 = ra == 0 ? mk(R(1), R(0)) : E[0][da + 1][sc][ra < 0];
                const C e2 = rb == 0 ? mk(R(1), R(0)) : E[1][db + 1][sc][rb < 0];
                F[o][col++] = e1 * e2;
            }
    }
    gamma_from_F<R>(F, out);
}

// Class of a grid index along one axis: 0 interior (all three sigmas zero),
// 1..b left PML (index -b..-1), b+1..2b right PML (index n+2..n+1+b).
__device__ __forceinline__ int pml_class(int q, int n, int b) {
    if (q <= -1) return q + b + 1;
    if (q >= n + 2) return b + 1 + (q - n - 2);
    return 0;
}
__device__ __forceinline__ int class_index(int cl, int n, int b) {
    if (cl == 0) return 0;
    if (cl <= b) return cl - b - 1;
    return n + 2 + (cl - b - 1);
}

// Physical PML stencils: one per (class x1, class x2), global omega.
__global__ void gamma_phys_kernel(double2* out, int n, int b, double Cw, double omega, double h) {
    const int nc = 2 * b + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc * nc) return;
    const int c1 = e / nc, c2 = e % nc;
    double2 g[9];
    if (c1 == 0 && c2 == 0) {
        for (int o = 0; o < 9; ++o) g[o] = mk(0.0, 0.0);
    } else {
        const int q1 = class_index(c1, n, b), q2 = class_index(c2, n, b);
        double s1[3], s2[3];
        for (int t = 0; t < 3; ++t) {
            s1[t] = sigma_phys(q1 - 1 + t, n, b, Cw);
            s2[t] = sigma_phys(q2 - 1 + t, n, b, Cw);
        }
        pml_stencil<double>(s1, s2, omega, h, g);
    }
    for (int o = 0; o < 9; ++o) out[(size_t)e * 9 + o] = g[o];
}

// Auxiliary (moving) PML stencils: per frequency sample k, auxiliary layer
// t = 1..b_aux (distance from D_i) and x2 class.  Along x1 the left profile of
// width b_aux translated so that D_i's first layer plays the role of index 0
// (right = 0), or, for the auxiliary PML right of D_i (two fronts, right = 1),
// the right profile translated so that D_i's last layer plays the role of
// index n + 1.  R = float for the single-precision preconditioner (these
// stencils enter only the slab subproblems, which it factors in single
// precision).
template <typename R>
__global__ void gamma_aux_kernel(double2* out, int n, int b, int baux, int ns, double s_lo, double s_hi,
                                 double Cw, double h, int right) {
    const int nc = 2 * b + 1;
    const long long tot = (long long)ns * baux * nc;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const int c2 = (int)(e % nc);
    const int t = (int)((e / nc) % baux) + 1;
    const int k = (int)(e / ((long long)nc * baux));
    double sk = (ns == 1) ? s_lo : (k == ns - 1 ? s_hi : s_lo + k * ((s_hi - s_lo) / (ns - 1)));
    const double w = sqrt(sk);
    double s1[3], s2[3];
    const int q2 = class_index(c2, n, b);
    for (int u = 0; u < 3; ++u) {
        double v = 0;
        if (!right) {   // offset q1 from D_i's first layer
            const int q1 = -t - 1 + u;
            if (q1 <= -1) { const double tt = (q1 + 1.0) / baux; v = -Cw * tt * tt; }
        } else {        // offset d from D_i's last layer
            const int d = t - 1 + u;
            if (d >= 1) { const double tt = (d - 1.0) / baux; v = Cw * tt * tt; }
        }
        s1[u] = v;
        s2[u] = sigma_phys(q2 - 1 + u, n, b, Cw);
    }
    double2 g[9];
    pml_stencil<R>(s1, s2, w, h, g);
    for (int o = 0; o < 9; ++o) out[(size_t)e * 9 + o] = g[o];
}

__device__ __forceinline__ double m_at(const double* m, int n, int i1, int i2) {
    return (i1 >= 1 && i1 <= n && i2 >= 1 && i2 <= n) ? m[(size_t)(i1 - 1) * n + (i2 - 1)] : 0.0;
}

// Row coefficients of every slab subproblem: coef[off + k*cstride + la*9 + o].
__global__ void assemble_kernel(const SlabDev* __restrict__ slabs, int n_slabs, const double* __restrict__ m,
                                const double2* __restrict__ gphys, const double2* __restrict__ gaux,
                                const double2* __restrict__ gaux_r, StencilArgs st, double2* __restrict__ coef, int n, int b, int baux, int n_tot,
                                int ns, double s_lo, double s_hi, double omega) {
    const int i = blockIdx.y;
    if (i >= n_slabs) return;
    const SlabDev sd = slabs[i];
    const int tot = sd.w * n_tot;
    const int nc = 2 * b + 1;
    const double w2 = omega * omega;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        const int k = e / sd.w, la = e % sd.w;
        const int x1 = sd.s - sd.na + la, i2 = k - b;
        double2* out = coef + sd.coef_off + (long long)k * sd.cstride + la * 9;
        if (la < sd.na || la > sd.ll) {   // auxiliary layer t left of D_i, or right of it
            const bool rgt = la > sd.ll;
            const int t = rgt ? la - sd.ll : sd.na - la;
            const double v = w2 * (1.0 - m_at(m, n, x1, i2));
            int kk = 0;
            if (ns > 1) {
                const double x = (v - s_lo) / ((s_hi - s_lo) / (ns - 1));
                kk = (int)ceil(x - 0.5);  // nearest sample, ties to the lower one
                kk = kk < 0 ? 0 : (kk > ns - 1 ? ns - 1 : kk);
            }
            const double2* g = (rgt ? gaux_r : gaux) + (((size_t)kk * baux + (t - 1)) * nc + pml_class(i2, n, b)) * 9;
            for (int o = 0; o < 9; ++o) out[o] = g[o];
        } else if (x1 >= 0 && x1 <= n + 1 && i2 >= 0 && i2 <= n + 1) {
            for (int o = 0; o < 9; ++o) {
                const double mm = m_at(m, n, x1 + o / 3 - 1, i2 + o % 3 - 1);
                out[o] = st.a_conj[o] + (w2 * mm) * st.b_conj[o];
            }
        } else {
            const double2* g = gphys + ((size_t)pml_class(x1, n, b) * nc + pml_class(i2, n, b)) * 9;
            for (int o = 0; o < 9; ++o) out[o] = g[o];
        }
    }
}

// f = Q r: f_i = sum_o conj(alpha_o) r_{i+o} on I^h = {0..n+1}^2, zero on the
// PML; r is zero outside I.  Layout f[r][a2][a1] over the n_tot^2 grid (x2
// slowest, so a slab solve reads one block row's layers contiguously).
template <typename C>
__global__ void sparsify_kernel(const double2* __restrict__ r, C* __restrict__ f, StencilArgs st, int n, int b,
                                int n_tot) {
    const long long tot = (long long)n_tot * n_tot;
    const int rr = blockIdx.y;
    const double2* rv = r + (long long)rr * n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i2 = (int)(e / n_tot) - b, i1 = (int)(e % n_tot) - b;   // x2 slowest
        double2 acc = mk(0.0, 0.0);
        if (i1 >= 0 && i1 <= n + 1 && i2 >= 0 && i2 <= n + 1) {
            for (int o = 0; o < 9; ++o) {
                const int j1 = i1 + o / 3 - 1, j2 = i2 + o % 3 - 1;
                if (j1 >= 1 && j1 <= n && j2 >= 1 && j2 <= n)
                    acc = cfma(st.a_conj[o], rv[(long long)(j1 - 1) * n + (j2 - 1)], acc);
            }
        }
        f[(long long)rr * tot + e] = to_c<C>(acc);
    }
}

// The same f = Q r by 32 x 32 tiles of the output: r (x1 slowest) is read
// into shared memory along x2 and f (x2 slowest) written along x1, so both
// sides are coalesced (the plain kernel reads r across rows).  The stencil
// arithmetic runs in the working precision C of f: FP32 for the
// single-precision sweep, whose input f is rounded to FP32 anyway (nine FP64
// complex FMAs per point would make the kernel FP64-bound on this GPU).
// grid (tiles along x1, tiles along x2, R), 256 threads.
template <typename C>
__global__ void __launch_bounds__(256) sparsify_tiled_kernel(const double2* __restrict__ r, C* __restrict__ f,
                                                             StencilArgs st, int n, int b, int n_tot) {
    __shared__ C P[34][35];
    const int rr = blockIdx.z;
    const double2* rv = r + (long long)rr * n * n;
    const int a1_0 = blockIdx.x * 32, a2_0 = blockIdx.y * 32;     // grid indices of the tile's corner
    const int i1_0 = a1_0 - b, i2_0 = a2_0 - b;
    for (int e = threadIdx.x; e < 34 * 34; e += blockDim.x) {
        const int p1 = e / 34, p2 = e % 34;
        const int j1 = i1_0 - 1 + p1, j2 = i2_0 - 1 + p2;
        P[p1][p2] = (j1 >= 1 && j1 <= n && j2 >= 1 && j2 <= n) ? to_c<C>(rv[(long long)(j1 - 1) * n + (j2 - 1)])
                                                               : czero<C>();
    }
    C a[9];
#pragma unroll
    for (int o = 0; o < 9; ++o) a[o] = to_c<C>(st.a_conj[o]);
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int a1 = a1_0 + tx, i1 = a1 - b;
    for (int q = ty; q < 32; q += 8) {
        const int a2 = a2_0 + q, i2 = a2 - b;
        if (a1 >= n_tot || a2 >= n_tot) continue;
        C acc = czero<C>();
        if (i1 >= 0 && i1 <= n + 1 && i2 >= 0 && i2 <= n + 1)
#pragma unroll
            for (int o = 0; o < 9; ++o) acc = cfma(a[o], P[tx + o / 3][q + o % 3], acc);
        f[(long long)rr * n_tot * n_tot + (long long)a2 * n_tot + a1] = acc;
    }
}

// Q^T (Eq. Huf transposed): r_j = sum_o conj(alpha_o) X_{j-o} for j in I, X on the
// grid rows of I^h (x2 slowest, like the sparsified right-hand side).
template <typename C>
__global__ void sparsify_t_kernel(const C* __restrict__ X, double2* __restrict__ r, StencilArgs st, int n, int b,
                                  int n_tot) {
    const long long N = (long long)n * n, tot = (long long)n_tot * n_tot;
    const int rr = blockIdx.y;
    const C* xv = X + (long long)rr * tot;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int j1 = (int)(e / n) + 1, j2 = (int)(e % n) + 1;
        double2 acc = mk(0.0, 0.0);
        for (int o = 0; o < 9; ++o) {
            const int i1 = j1 - (o / 3 - 1), i2 = j2 - (o % 3 - 1);   // in 0..n+1
            acc = cfma(st.a_conj[o], to_d(xv[(long long)(i2 + b) * n_tot + (i1 + b)]), acc);
        }
        r[rr * N + e] = acc;
    }
}

// dL/dm = Re((-omega^2 K mu) . (u + u_I)) summed over the right-hand sides, with
// u_I = exp(i omega d.p) recomputed from the directions.
__global__ void gradient_kernel(const double2* __restrict__ Kmu, const double2* __restrict__ u,
                                const double* __restrict__ dirs, double* __restrict__ grad, int n, int R, double omega,
                                double h) {
    const long long N = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e / n), col = (int)(e % n);
        double acc = 0.0;
        for (int r = 0; r < R; ++r) {
            const double ph = omega * (dirs[2 * r] * (row + 1) * h + dirs[2 * r + 1] * (col + 1) * h);
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double2 ut = u[r * N + e] + mk(cs, sn);
            const double2 k = Kmu[r * N + e];
            acc += k.x * ut.x - k.y * ut.y;
        }
        grad[e] = acc;
    }
}

// y = H x on the n_tot^2 grid (x2 slowest): every point's row from the
// subproblem table of the slab whose D_i holds it (those rows are H's rows,
// Eq. Hwv_approx), FP64; neighbours outside the grid are the zero Dirichlet
// values.
__global__ void apply_H_kernel(const SlabDev* __restrict__ slabs, int n_slabs, const double2* __restrict__ coef,
                               const double2* __restrict__ x, double2* __restrict__ y, int n_tot, int b, int bs) {
    const long long tot = (long long)n_tot * n_tot;
    const int rr = blockIdx.y;
    const double2* xv = x + rr * tot;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int X2 = (int)(e / n_tot), X1 = (int)(e % n_tot);
        const int x1 = X1 - b;
        int i = x1 < 0 ? 0 : x1 / bs;
        if (i > n_slabs - 1) i = n_slabs - 1;
        const SlabDev sd = slabs[i];
        const double2* row = coef + sd.coef_off + (long long)X2 * sd.cstride + (sd.na + (x1 - sd.s)) * 9;
        double2 acc = mk(0.0, 0.0);
        for (int o = 0; o < 9; ++o) {
            const int Y1 = X1 + o / 3 - 1, Y2 = X2 + o % 3 - 1;
            if (Y1 >= 0 && Y1 < n_tot && Y2 >= 0 && Y2 < n_tot) acc = cfma(row[o], xv[(long long)Y2 * n_tot + Y1], acc);
        }
        y[rr * tot + e] = acc;
    }
}

// u on I from a grid vector (x2 slowest).
__global__ void extract_grid_kernel(const double2* __restrict__ U, double2* __restrict__ u, int n, int b, int n_tot) {
    const long long N = (long long)n * n, tot = (long long)n_tot * n_tot;
    const int rr = blockIdx.y;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(e / n) + 1, i2 = (int)(e % n) + 1;
        u[rr * N + e] = U[rr * tot + (long long)(i2 + b) * n_tot + (i1 + b)];
    }
}

StencilArgs stencil_args(const lss_ctx* c) {
    StencilArgs st;
    for (int o = 0; o < 9; ++o) {
        st.a_conj[o] = make_double2(c->alpha[o].real(), -c->alpha[o].imag());
        st.b_conj[o] = make_double2(c->beta[o].real(), -c->beta[o].imag());
    }
    return st;
}

}  // namespace

int lss_build_gamma_phys(lss_ctx* c, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_SETUP, 1);
    const int nc = 2 * c->b + 1;
    const double Cw = c->pml.C / c->omega;
    gamma_phys_kernel<<<(nc * nc + 127) / 128, 128, 0, s>>>(c->gam_phys, c->n, c->b, Cw, c->omega, c->h);
    return lss_check_cuda(c, cudaGetLastError(), "gamma tables");
}

int lss_build_gamma_aux(lss_ctx* c, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_SETUP, 1);
    const int nc = 2 * c->b + 1;
    const double Cw = c->pml.C / c->omega;
    const long long tot = (long long)c->ns_eff * c->b_aux * nc;
    const unsigned grid = (unsigned)((tot + 127) / 128);
    for (int right = 0; right < (c->fronts == 2 ? 2 : 1); ++right) {
        double2* out = right ? c->gam_aux_r : c->gam_aux;
        if (c->prec == LSS_FP64)
            gamma_aux_kernel<double><<<grid, 128, 0, s>>>(out, c->n, c->b, c->b_aux, c->ns_eff, c->s_lo, c->s_hi, Cw,
                                                          c->h, right);
        else
            gamma_aux_kernel<float><<<grid, 128, 0, s>>>(out, c->n, c->b, c->b_aux, c->ns_eff, c->s_lo, c->s_hi, Cw,
                                                         c->h, right);
    }
    return lss_check_cuda(c, cudaGetLastError(), "gamma tables");
}

int lss_assemble_slabs(lss_ctx* c, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_SETUP, 1);
    const int per = std::max(1, (c->n_tot * LSS_WMAX + 255) / 256);
    assemble_kernel<<<dim3(std::min(per, 64), c->n_slabs), 256, 0, s>>>(
        c->d_slabs, c->n_slabs, c->m, c->gam_phys, c->gam_aux, c->gam_aux_r, stencil_args(c), c->coef64, c->n, c->b, c->b_aux,
        c->n_tot, c->ns_eff, c->s_lo, c->s_hi, c->omega);
    return lss_check_cuda(c, cudaGetLastError(), "assemble");
}

int lss_sparsify(lss_ctx* c, const double2* r, void* f, int R, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_SPARSIFY, 1);
    const int tiles = (c->n_tot + 31) / 32;
    const dim3 grid(tiles, tiles, R);
    if (c->prec == LSS_FP64)
        sparsify_tiled_kernel<double2><<<grid, 256, 0, s>>>(r, (double2*)f, stencil_args(c), c->n, c->b, c->n_tot);
    else
        sparsify_tiled_kernel<float2><<<grid, 256, 0, s>>>(r, (float2*)f, stencil_args(c), c->n, c->b, c->n_tot);
    return lss_check_cuda(c, cudaGetLastError(), "sparsify");
}

// F = beta^* f on I^h (Sec. 4), FP64, grid layout of the sparsified right-hand side.
int lss_sparsify_beta(lss_ctx* c, const double2* f, double2* F, int R, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_SPARSIFY, 1);
    const long long tot = (long long)c->n_tot * c->n_tot;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 4LL * c->num_sms);
    StencilArgs st = stencil_args(c);
    for (int o = 0; o < 9; ++o) st.a_conj[o] = st.b_conj[o];
    sparsify_kernel<double2><<<dim3(blocks, R), 256, 0, s>>>(f, F, st, c->n, c->b, c->n_tot);
    return lss_check_cuda(c, cudaGetLastError(), "sparsify beta");
}

int lss_apply_H(lss_ctx* c, const double2* x, double2* y, int R, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_MATVEC, 1);
    const long long tot = (long long)c->n_tot * c->n_tot;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 4LL * c->num_sms);
    apply_H_kernel<<<dim3(blocks, R), 256, 0, s>>>(c->d_slabs, c->n_slabs, c->coef64, x, y, c->n_tot, c->b,
                                                   c->slab.b_slab);
    return lss_check_cuda(c, cudaGetLastError(), "apply H");
}

int lss_extract_grid(lss_ctx* c, const double2* U, double2* u, int R, cudaStream_t s) {
    const long long N = (long long)c->n * c->n;
    const int blocks = (int)std::min<long long>((N + 255) / 256, 4LL * c->num_sms);
    extract_grid_kernel<<<dim3(blocks, R), 256, 0, s>>>(U, u, c->n, c->b, c->n_tot);
    return lss_check_cuda(c, cudaGetLastError(), "extract");
}

int lss_sparsify_t(lss_ctx* c, const void* X, double2* r, int R, cudaStream_t s) {
    ProfScope ps(c, s, LSS_PROF_SPARSIFY, 1);
    const long long N = (long long)c->n * c->n;
    const int blocks = (int)std::min<long long>((N + 255) / 256, 4096);
    if (c->prec == LSS_FP64)
        sparsify_t_kernel<double2><<<dim3(blocks, R), 256, 0, s>>>((const double2*)X, r, stencil_args(c), c->n, c->b,
                                                                    c->n_tot);
    else
        sparsify_t_kernel<float2><<<dim3(blocks, R), 256, 0, s>>>((const float2*)X, r, stencil_args(c), c->n, c->b,
                                                                   c->n_tot);
    return lss_check_cuda(c, cudaGetLastError(), "sparsify transpose");
}

int lss_gradient_m(lss_ctx* c, const double2* Kmu, const double2* u, const double* dirs_dev, double* grad, int R,
                   cudaStream_t s) {
    const long long N = (long long)c->n * c->n;
    const int blocks = (int)std::min<long long>((N + 255) / 256, 4096);
    gradient_kernel<<<blocks, 256, 0, s>>>(Kmu, u, dirs_dev, grad, c->n, R, c->omega, c->h);
    return lss_check_cuda(c, cudaGetLastError(), "gradient");
}
