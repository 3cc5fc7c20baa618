// The 3D path (Sec. 3.1): Nystrom weights and their FFT on the L^3 grid, the
// 27-point interior stencils, the 26-direction PML stencils, slabs of
// x1-layers whose subproblems are block tridiagonal along x2 with dense
// blocks of w * n_tot unknowns (layer a, x3 index c), their factorization by
// block Gaussian elimination with every pivot block inverted by blocked
// Gauss-Jordan elimination with partial pivoting, and the sweep of
// Algorithm 2 as one persistent grid-synchronised kernel.
//
// Layouts (complex entries):
//  - vectors on I: n^3, x1 slowest;  grid vectors on I^{h+eta}: n_tot^3,
//    [X1][X2][X3] with X = x + b.
//  - slab i's coefficient table: block row k (X2 = k), part p = d2+1
//    (0: coupling to block k-1, 1: the block itself, 2: block k+1), row
//    q = a * n_tot + c (a = layer of the subproblem, c = X3), 9 entries
//    (d1+1)*3 + (d3+1):  ((k*3 + p) * M + q) * 9 + ...,  M = w * n_tot.
//  - factors: per slab and block row k the dense M x M inverse of the pivot
//    block D_k, row-major.
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <type_traits>
#include <vector>

#include "fft_line.cuh"
#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"
#include "stencil3.cuh"

using cd = std::complex<double>;

namespace {

constexpr int kMaxBlock3 = 1760;      // largest pivot block M = w * n_tot (panel kernel shared memory: M x 128 B)
constexpr int kNB64 = 8;              // Gauss-Jordan panel width, FP64
constexpr int kNB32 = 16;             // Gauss-Jordan panel width, FP32
constexpr int kNO = 64;               // outer panel width of the tensor-core path
constexpr int kSweepThreads = 512;
constexpr int kSweepRB = 4;           // right-hand sides per sweep launch

int line_threads3(int L) { return L / 4 < 32 ? 32 : L / 4; }
int col_group3(int L) { return L >= 1024 ? 1 : (L >= 256 ? 2 : 4); }

// ---------------------------------------------------------------- kernel table (Sec. 2.1 in 3D)

// k_j = G(|p_j|) h^3 = h^3 exp(i omega r) / (4 pi r)
__device__ __forceinline__ double2 k_weight_3d(double r, double omega, double h3) {
    double sn, cs;
    sincos(omega * r, &sn, &cs);
    const double s = h3 / (4.0 * M_PI * r);
    return mk(s * cs, s * sn);
}

// Circular L^3 table: offsets |o_a| <= n-1 at o_a mod L, zero elsewhere; [j1][j2][j3].
__global__ void k3_table_circ(double2* kc, int n, int L, double omega, double h, double2 k0) {
    const long long tot = (long long)L * L * L;
    const double h3 = h * h * h;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int j1 = (int)(e / ((long long)L * L)), j2 = (int)((e / L) % L), j3 = (int)(e % L);
        const int o1 = j1 < L / 2 ? j1 : j1 - L, o2 = j2 < L / 2 ? j2 : j2 - L, o3 = j3 < L / 2 ? j3 : j3 - L;
        double2 v = mk(0.0, 0.0);
        if (abs(o1) <= n - 1 && abs(o2) <= n - 1 && abs(o3) <= n - 1) {
            if (o1 == 0 && o2 == 0 && o3 == 0) v = k0;
            else v = k_weight_3d(h * sqrt((double)o1 * o1 + (double)o2 * o2 + (double)o3 * o3), omega, h3);
        }
        kc[e] = v;
    }
}

// Offsets {-(n+1)..n+1}^3, index ((o1+n+1)*S + o2+n+1)*S + o3+n+1, S = 2n+3.
__global__ void k3_table_ext(double2* kx, int n, double omega, double h, double2 k0) {
    const int S = 2 * n + 3;
    const long long tot = (long long)S * S * S;
    const double h3 = h * h * h;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int o1 = (int)(e / ((long long)S * S)) - (n + 1), o2 = (int)((e / S) % S) - (n + 1),
                  o3 = (int)(e % S) - (n + 1);
        kx[e] = (o1 == 0 && o2 == 0 && o3 == 0)
                    ? k0
                    : k_weight_3d(h * sqrt((double)o1 * o1 + (double)o2 * o2 + (double)o3 * o3), omega, h3);
    }
}

// Gram matrix of K_{mu,mu^c} (Eq. alpha in 3D): G_ab = sum_{j in mu^c} k_{o_a-j} conj(k_{o_b-j}),
// mu^c = {-n..n}^3 minus mu; pairs a <= b of the 27 offsets; block partial sums.
__global__ void gram3_partial(const double2* __restrict__ kx, int n, double2* __restrict__ part) {
    __shared__ double2 red[256];
    int pair = blockIdx.y, a = 0;
    while (pair >= 27 - a) { pair -= 27 - a; ++a; }
    const int b = a + pair;
    const int a1 = a / 9 - 1, a2 = (a / 3) % 3 - 1, a3 = a % 3 - 1;
    const int b1 = b / 9 - 1, b2 = (b / 3) % 3 - 1, b3 = b % 3 - 1;
    const long long S = 2 * n + 3, Mw = 2 * n + 1;
    const long long tot = Mw * Mw * Mw;
    double2 acc = mk(0.0, 0.0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int j1 = (int)(e / (Mw * Mw)) - n, j2 = (int)((e / Mw) % Mw) - n, j3 = (int)(e % Mw) - n;
        if (abs(j1) <= 1 && abs(j2) <= 1 && abs(j3) <= 1) continue;
        const double2 ka = kx[((a1 - j1 + n + 1) * S + (a2 - j2 + n + 1)) * S + (a3 - j3 + n + 1)];
        const double2 kb = kx[((b1 - j1 + n + 1) * S + (b2 - j2 + n + 1)) * S + (b3 - j3 + n + 1)];
        acc = cfma(ka, conjc(kb), acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// ---------------------------------------------------------------- LS operator in 3D (pruned FFT convolution)

// Pass over contiguous x3 lines.  Forward: grid (n^2 or L^2 lines, R); line
// (i1, i2) of the input (m.*u, u, m.*u_I, or a raw L-line) -> buf[r][line][L].
template <int IN>
__global__ void mv3_rows_fwd(const double2* __restrict__ x, const double* __restrict__ m,
                             const double* __restrict__ dirs, double2* __restrict__ uI, double2* __restrict__ buf,
                             const double2* __restrict__ tw, int n, int lines, int L, int lg, double omega,
                             double h) {
    extern __shared__ double2 sm[];
    double2* A = sm;
    double2* B = sm + L;
    const int line = blockIdx.x, r = blockIdx.y, t = threadIdx.x, nt = blockDim.x;
    const long long N = (long long)n * n * n;
    for (int j = t; j < L; j += nt) {
        double2 v = mk(0.0, 0.0);
        if (IN == MV_IN_RAW) {
            v = x[(long long)line * L + j];
        } else if (j < n) {
            const long long e = (long long)line * n + j;
            if (IN == MV_IN_MU) {
                v = m[e] * x[r * N + e];
            } else if (IN == MV_IN_U) {
                v = x[r * N + e];
            } else {   // u_I = exp(i omega d.p), p = ((i1+1) h, (i2+1) h, (j+1) h)
                const int i1 = line / n, i2 = line % n;
                const double* d = dirs + 3 * r;
                const double ph = omega * h * (d[0] * (i1 + 1) + d[1] * (i2 + 1) + d[2] * (j + 1));
                double sn, cs;
                sincos(ph, &sn, &cs);
                if (uI) uI[r * N + e] = mk(cs, sn);
                v = m[e] * mk(cs, sn);
            }
        }
        A[j] = v;
    }
    __syncthreads();
    double2* res = fft_line<false>(A, B, L, lg, tw, t, nt);
    double2* out = buf + ((long long)r * lines + line) * L;
    for (int j = t; j < L; j += nt) out[j] = res[j];
}

// Inverse pass over contiguous x3 lines, n kept, fused epilogue.  grid (n^2, R).
template <int OUT>
__global__ void mv3_rows_inv(const double2* __restrict__ buf, const double2* __restrict__ x,
                             const double* __restrict__ m, double2* __restrict__ y, const double2* __restrict__ tw,
                             int n, int L, int lg) {
    extern __shared__ double2 sm[];
    double2* A = sm;
    double2* B = sm + L;
    const int line = blockIdx.x, r = blockIdx.y, t = threadIdx.x, nt = blockDim.x;
    const long long N = (long long)n * n * n;
    const double2* in = buf + ((long long)r * n * n + line) * L;
    for (int j = t; j < L; j += nt) A[j] = in[j];
    __syncthreads();
    double2* res = fft_line<true>(A, B, L, lg, tw, t, nt);
    for (int j = t; j < n; j += nt) {
        const long long e = (long long)line * n + j;
        const double2 v = res[j];
        if (OUT == MV_OUT_A) y[r * N + e] = x[r * N + e] + v;
        else if (OUT == MV_OUT_AT) y[r * N + e] = x[r * N + e] + m[e] * v;
        else y[r * N + e] = mk(-v.x, -v.y);
    }
}

enum { COL_FWD = 0, COL_CONV = 1, COL_INV = 2, COL_KHAT = 3 };

// Strided-line pass.  The input is viewed as [r][p][row][q] with rows_in rows
// (row stride Q); line (p, q) is FFT'd along row.  C consecutive q per CTA
// (coalesced).  grid (Q / C, P, R), block C * nt.
//  COL_FWD:  rows_in nonzero -> L rows of out[r][p][k][q]
//  COL_CONV: in place (out == in): forward, * khat[q * L + k], inverse, keep rows_out rows
//  COL_INV:  inverse of L rows, keep rows_out rows of out[r][p][row][q]
//  COL_KHAT: forward, out[q * L + k] = scale * result (kernel transform, transposed)
template <int MODE>
__global__ void mv3_cols(const double2* __restrict__ in, double2* __restrict__ out, const double2* __restrict__ khat,
                         const double2* __restrict__ tw, int P, int rows_in, int rows_out, long long Q, int L,
                         int lg, int C, double scale) {
    extern __shared__ double2 sm[];
    double2* A = sm;
    double2* B = sm + (size_t)C * L;
    const long long q0 = (long long)blockIdx.x * C;
    const int p = blockIdx.y, r = blockIdx.z;
    const int nt = blockDim.x / C, g = threadIdx.x / nt, t = threadIdx.x % nt;
    const double2* ib = in + ((long long)r * P + p) * rows_in * Q;
    for (int idx = threadIdx.x; idx < L * C; idx += blockDim.x) {
        const int row = idx / C, c = idx % C;
        A[(size_t)c * L + row] = row < rows_in ? ib[(long long)row * Q + q0 + c] : mk(0.0, 0.0);
    }
    __syncthreads();
    double2* res = (MODE == COL_INV) ? fft_line<true>(A + (size_t)g * L, B + (size_t)g * L, L, lg, tw, t, nt)
                                     : fft_line<false>(A + (size_t)g * L, B + (size_t)g * L, L, lg, tw, t, nt);
    const long long q = q0 + g;
    if (MODE == COL_KHAT) {
        for (int k = t; k < L; k += nt) out[q * L + k] = scale * res[k];
        return;
    }
    if (MODE == COL_CONV) {
        const double2* kh = khat + q * L;
        for (int k = t; k < L; k += nt) res[k] = res[k] * __ldg(&kh[k]);
        __syncthreads();
        double2* other = (res == A + (size_t)g * L) ? B + (size_t)g * L : A + (size_t)g * L;
        res = fft_line<true>(res, other, L, lg, tw, t, nt);
    }
    // every group's result sits in the same half (A or B)
    const double2* base = (res == A + (size_t)g * L) ? A : B;
    const int rows_o = (MODE == COL_FWD) ? L : rows_out;
    const int rows_tot = (MODE == COL_FWD) ? L : rows_out;
    double2* ob = out + ((long long)r * P + p) * rows_tot * Q;
    for (int idx = threadIdx.x; idx < rows_o * C; idx += blockDim.x) {
        const int row = idx / C, c = idx % C;
        ob[(long long)row * Q + q0 + c] = base[(size_t)c * L + row];
    }
}

// ---------------------------------------------------------------- PML stencils (Eq. gamma in 3D)

// Physical PML stencils: one per (class x1, class x2, class x3), global omega.
__global__ void __launch_bounds__(32 * kGamWarps) gamma3_phys_kernel(double2* out, int n, int b, double Cw,
                                                                      double omega, double h) {
    __shared__ GamSmem S[kGamWarps];
    const int nc = 2 * b + 1;
    const int wid = threadIdx.x / 32;
    const int e = blockIdx.x * kGamWarps + wid;
    if (e >= nc * nc * nc) return;
    const int c1 = e / (nc * nc), c2 = (e / nc) % nc, c3 = e % nc;
    if (c1 == 0 && c2 == 0 && c3 == 0) {
        if ((threadIdx.x & 31) < 27) out[(size_t)e * 27 + (threadIdx.x & 31)] = mk(0.0, 0.0);
        return;
    }
    double sig[3][3];
    const int q[3] = {class_index3(c1, n, b), class_index3(c2, n, b), class_index3(c3, n, b)};
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < 3; ++t) sig[a][t] = sigma_phys3(q[a] - 1 + t, n, b, Cw);
    gamma3_warp(sig, omega, h, S[wid], out + (size_t)e * 27);
}

// Moving-PML stencils: per (sample k, auxiliary layer t = 1..b_aux, class x2,
// class x3); along x1 the left profile of width b_aux translated so that D_i's
// first layer plays the role of index 0 (right = 0), or the right profile
// translated so that D_i's last layer plays the role of index n + 1 (right = 1,
// two fronts); local frequency sqrt(s_k).
__global__ void __launch_bounds__(32 * kGamWarps) gamma3_aux_kernel(double2* out, int n, int b, int baux, int ns,
                                                                     double s_lo, double s_hi, double Cw, double h,
                                                                     int right) {
    __shared__ GamSmem S[kGamWarps];
    const int nc = 2 * b + 1;
    const int wid = threadIdx.x / 32;
    const long long e = (long long)blockIdx.x * kGamWarps + wid;
    const long long tot = (long long)ns * baux * nc * nc;
    if (e >= tot) return;
    const int c3 = (int)(e % nc), c2 = (int)((e / nc) % nc);
    const int t = (int)((e / ((long long)nc * nc)) % baux) + 1;
    const int k = (int)(e / ((long long)nc * nc * baux));
    const double sk = (ns == 1) ? s_lo : (k == ns - 1 ? s_hi : s_lo + k * ((s_hi - s_lo) / (ns - 1)));
    double sig[3][3];
    const int q2 = class_index3(c2, n, b), q3 = class_index3(c3, n, b);
    for (int u = 0; u < 3; ++u) {
        double v = 0;
        if (!right) {   // offset q1 from D_i's first layer
            const int q1 = -t - 1 + u;
            if (q1 <= -1) { const double tt = (q1 + 1.0) / baux; v = -Cw * tt * tt; }
        } else {        // offset d from D_i's last layer
            const int d = t - 1 + u;
            if (d >= 1) { const double tt = (d - 1.0) / baux; v = Cw * tt * tt; }
        }
        sig[0][u] = v;
        sig[1][u] = sigma_phys3(q2 - 1 + u, n, b, Cw);
        sig[2][u] = sigma_phys3(q3 - 1 + u, n, b, Cw);
    }
    gamma3_warp(sig, sqrt(sk), h, S[wid], out + (size_t)e * 27);
}

// ---------------------------------------------------------------- assembly, Q, extraction

// Row coefficients of every slab subproblem.  grid (blocks, n_slabs); thread
// per row (k, a, c).  Layout in the file comment.
__global__ void assemble3_kernel(const Slab3* __restrict__ slabs, const double* __restrict__ m,
                                 const double2* __restrict__ gphys, const double2* __restrict__ gaux,
                                 const double2* __restrict__ gaux_r, Stencil27 st,
                                 double2* __restrict__ coef, int n, int b, int baux, int n_tot, int ns, double s_lo,
                                 double s_hi, double omega) {
    const Slab3 sd = slabs[blockIdx.y];
    const long long rows = (long long)n_tot * sd.M;
    const int nc = 2 * b + 1;
    const double w2 = omega * omega;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / sd.M), qr = (int)(e % sd.M);
        const int a = qr / n_tot, c = qr % n_tot;
        const int x1 = sd.s - sd.na + a, i2 = k - b, i3 = c - b;
        double2 row[27];
        if (a < sd.na || a > sd.ll) {   // auxiliary layer t left of D_i, or right of it
            const bool rgt = a > sd.ll;
            const int t = rgt ? a - sd.ll : sd.na - a;
            const double v = w2 * (1.0 - m3_at(m, n, x1, i2, i3));
            int kk = 0;
            if (ns > 1) {
                const double x = (v - s_lo) / ((s_hi - s_lo) / (ns - 1));
                kk = (int)ceil(x - 0.5);   // nearest sample, ties to the lower one
                kk = kk < 0 ? 0 : (kk > ns - 1 ? ns - 1 : kk);
            }
            const double2* g = (rgt ? gaux_r : gaux) +
                               ((((size_t)kk * baux + (t - 1)) * nc + pml_class3(i2, n, b)) * nc + pml_class3(i3, n, b)) *
                                   27;
            for (int o = 0; o < 27; ++o) row[o] = g[o];
        } else if (x1 >= 0 && x1 <= n + 1 && i2 >= 0 && i2 <= n + 1 && i3 >= 0 && i3 <= n + 1) {
            for (int o = 0; o < 27; ++o) {
                const double mm = m3_at(m, n, x1 + o / 9 - 1, i2 + (o / 3) % 3 - 1, i3 + o % 3 - 1);
                row[o] = st.a_conj[o] + (w2 * mm) * st.b_conj[o];
            }
        } else {
            const double2* g =
                gphys + (((size_t)pml_class3(x1, n, b) * nc + pml_class3(i2, n, b)) * nc + pml_class3(i3, n, b)) * 27;
            for (int o = 0; o < 27; ++o) row[o] = g[o];
        }
        double2* out = coef + sd.cf_off;
        for (int o = 0; o < 27; ++o) {
            const int d1 = o / 9, d2 = (o / 3) % 3, d3 = o % 3;
            out[(((long long)k * 3 + d2) * sd.M + qr) * 9 + d1 * 3 + d3] = row[o];
        }
    }
}

// f = Q r on the n_tot^3 grid: f_i = sum_o conj(alpha_o) r_{i+o} on I^h, zero on the PML.
template <typename C>
__global__ void sparsify3_kernel(const double2* __restrict__ r, C* __restrict__ f, Stencil27 st, int n, int b,
                                 int n_tot) {
    const long long tot = (long long)n_tot * n_tot * n_tot;
    const long long N = (long long)n * n * n;
    const int rr = blockIdx.y;
    const double2* rv = r + rr * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(e / ((long long)n_tot * n_tot)) - b, i2 = (int)((e / n_tot) % n_tot) - b,
                  i3 = (int)(e % n_tot) - b;
        double2 acc = mk(0.0, 0.0);
        if (i1 >= 0 && i1 <= n + 1 && i2 >= 0 && i2 <= n + 1 && i3 >= 0 && i3 <= n + 1) {
            for (int o = 0; o < 27; ++o) {
                const int j1 = i1 + o / 9 - 1, j2 = i2 + (o / 3) % 3 - 1, j3 = i3 + o % 3 - 1;
                if (j1 >= 1 && j1 <= n && j2 >= 1 && j2 <= n && j3 >= 1 && j3 <= n)
                    acc = cfma(st.a_conj[o], rv[((long long)(j1 - 1) * n + (j2 - 1)) * n + (j3 - 1)], acc);
            }
        }
        f[rr * tot + e] = to_c<C>(acc);
    }
}

// y (on I) = the sweep solution restricted to I.
template <typename C>
__global__ void extract3_kernel(const C* __restrict__ ut, double2* __restrict__ y, int n, int b, int n_tot) {
    const long long N = (long long)n * n * n, G = (long long)n_tot * n_tot * n_tot;
    const int rr = blockIdx.y;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
         e += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(e / ((long long)n * n)), i2 = (int)((e / n) % n), i3 = (int)(e % n);
        y[rr * N + e] = to_d(ut[rr * G + ((long long)(i1 + 1 + b) * n_tot + (i2 + 1 + b)) * n_tot + (i3 + 1 + b)]);
    }
}

__global__ void cast3_kernel(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// ---------------------------------------------------------------- factorization (block LU along x2)

// W = A_k: the 9-point (d1, d3) block of coefficients with d2 = 0 (in-block
// index (a, c), c < nc: for the slabs (x1 layer, x3), for the sub-slab
// problems of the recursive approach (x2 layer, x1 layer) with the block index
// along x3).
template <typename C>
__global__ void f3_init_A(const Slab3* __restrict__ slabs, const C* __restrict__ coef, C* __restrict__ W, int k) {
    const Slab3 sd = slabs[blockIdx.y];
    const int M = sd.M, n_tot = sd.nc;
    const long long MM = (long long)M * M;
    C* w = W + sd.w_off;
    const C* cf = coef + sd.cf_off + ((long long)k * 3 + 1) * M * 9;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MM;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / M), j = (int)(e % M);
        const int ai = i / n_tot, ci = i % n_tot, aj = j / n_tot, cj = j % n_tot;
        const int d1 = aj - ai, d3 = cj - ci;
        C v = czero<C>();
        if (d1 >= -1 && d1 <= 1 && d3 >= -1 && d3 <= 1) v = cf[(long long)i * 9 + (d1 + 1) * 3 + (d3 + 1)];
        w[e] = v;
    }
}

// X = D_{k-1}^{-1} B_{k-1}: X[q][j] = sum_{d1,d3} Dinv[q][p] Bc[p][(d1,d3)], p = j - (d1, d3).
template <typename C>
__global__ void f3_schur_X(const Slab3* __restrict__ slabs, const C* __restrict__ coef, const C* __restrict__ fac,
                           C* __restrict__ X, int k) {
    const Slab3 sd = slabs[blockIdx.y];
    const int M = sd.M, w = sd.w, n_tot = sd.nc;
    const long long MM = (long long)M * M;
    const C* Dinv = fac + sd.fac_off + (long long)(k - 1) * MM;
    const C* bc = coef + sd.cf_off + ((long long)(k - 1) * 3 + 2) * M * 9;
    C* x = X + sd.w_off;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MM;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / M), j = (int)(e % M);
        const int aj = j / n_tot, cj = j % n_tot;
        C acc = czero<C>();
        for (int d1 = -1; d1 <= 1; ++d1) {
            const int ap = aj - d1;
            if (ap < 0 || ap >= w) continue;
            for (int d3 = -1; d3 <= 1; ++d3) {
                const int cp = cj - d3;
                if (cp < 0 || cp >= n_tot) continue;
                const int p = ap * n_tot + cp;
                acc = cfma(Dinv[(long long)q * M + p], bc[(long long)p * 9 + (d1 + 1) * 3 + (d3 + 1)], acc);
            }
        }
        x[e] = acc;
    }
}

// W = A_k - C_k X: W[i][j] = A_k[i][j] - sum_{d1,d3} Cc[i][(d1,d3)] X[i + (d1, d3)][j].
template <typename C>
__global__ void f3_schur_D(const Slab3* __restrict__ slabs, const C* __restrict__ coef, const C* __restrict__ X,
                           C* __restrict__ W, int k) {
    const Slab3 sd = slabs[blockIdx.y];
    const int M = sd.M, w = sd.w, n_tot = sd.nc;
    const long long MM = (long long)M * M;
    const C* cc = coef + sd.cf_off + ((long long)k * 3 + 0) * M * 9;
    const C* ac = coef + sd.cf_off + ((long long)k * 3 + 1) * M * 9;
    const C* x = X + sd.w_off;
    C* wm = W + sd.w_off;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MM;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / M), j = (int)(e % M);
        const int ai = i / n_tot, ci = i % n_tot, aj = j / n_tot, cj = j % n_tot;
        C v = czero<C>();
        if (aj - ai >= -1 && aj - ai <= 1 && cj - ci >= -1 && cj - ci <= 1)
            v = ac[(long long)i * 9 + (aj - ai + 1) * 3 + (cj - ci + 1)];
        for (int d1 = -1; d1 <= 1; ++d1) {
            const int aq = ai + d1;
            if (aq < 0 || aq >= w) continue;
            for (int d3 = -1; d3 <= 1; ++d3) {
                const int cq = ci + d3;
                if (cq < 0 || cq >= n_tot) continue;
                const C cv = cc[(long long)i * 9 + (d1 + 1) * 3 + (d3 + 1)];
                const C xv = x[(long long)(aq * n_tot + cq) * M + j];
                v = v - cv * xv;
            }
        }
        wm[e] = v;
    }
}

__global__ void f3_rowid_init(const Slab3* __restrict__ slabs, int* __restrict__ rowid, int Mmax) {
    const int s = blockIdx.y;
    const int M = slabs[s].M;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x)
        rowid[(long long)s * Mmax + r] = r;
}

// Gauss-Jordan elimination of the panel columns J = [j0, j0+nbp) of W (one CTA
// per slab, the M x NB panel in shared memory, column-major so that the
// threads of a warp, which own consecutive rows, touch consecutive words).  Pivot j = j0 + jj is the
// largest |W[r][j]| over rows r >= j (ties to the lower row); rows j and r are
// swapped inside the panel (the rest of the rows later, by f3_swap_extract),
// recorded in piv and in rowid.  After the panel the columns J hold the
// eliminated values: rows R = [j0, j0+nbp) the inverse E of the pivot block,
// the other rows -P_O E.
template <typename C, int NB>
__global__ void __launch_bounds__(512) f3_panel(const Slab3* __restrict__ slabs, C* __restrict__ W, int* __restrict__ piv,
                                                int* __restrict__ rowid, int j0, int Mmax, int* err) {
    using R = decltype(C{}.x);
    extern __shared__ __align__(16) unsigned char smraw[];
    C* P = reinterpret_cast<C*>(smraw);
    __shared__ R red_v[32];
    __shared__ int red_i[32];
    __shared__ C s_pj[NB], s_oj[NB], s_d;
    __shared__ int s_pr;
    const int slab = blockIdx.x;
    const Slab3 sd = slabs[slab];
    const int M = sd.M;
    if (j0 >= M) return;
    const int nbp = min(NB, M - j0);
    C* w = W + sd.w_off;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < M * nbp; e += nt) {
        const int r = e / nbp, q = e % nbp;
        P[q * M + r] = w[(long long)r * M + j0 + q];
    }
    __syncthreads();
    const int nw = nt / 32;
    for (int jj = 0; jj < nbp; ++jj) {
        const int j = j0 + jj;
        // pivot: the largest |P[jj][r]| over rows r >= j (ties to the lower row);
        // each warp reduces its rows, then every thread reduces the warps'
        // results itself (no second barrier)
        R best = -1;
        int bi = M;
        for (int r = j + tid; r < M; r += nt) {
            const R v = cabs2(P[jj * M + r]);
            if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
        __syncthreads();
        // warp 0: the pivot over the warps' results, the pivot row (old row pr)
        // scaled by d = 1 / pivot and the old row j (which moves to position pr)
        if (tid < 32) {
            best = tid < nw ? red_v[tid] : R(-1);
            bi = tid < nw ? red_i[tid] : M;
            for (int o = 16; o > 0; o >>= 1) {
                const R ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            const bool sing = !(best > 0) || !isfinite(best) || bi >= M;
            const int pr = sing ? j : bi;
            const C d = crecip(P[jj * M + pr]);
            if (tid < nbp) {
                s_pj[tid] = (tid == jj) ? d : P[tid * M + pr] * d;
                s_oj[tid] = P[tid * M + j];
            }
            if (tid == 0) {
                if (sing) atomicOr(err, LSS_DERR_SINGULAR);
                s_pr = pr;
                s_d = d;
                piv[slab * NB + jj] = pr;
                if (pr != j) {
                    int* rid = rowid + (long long)slab * Mmax;
                    const int t = rid[j];
                    rid[j] = rid[pr];
                    rid[pr] = t;
                }
            }
        }
        __syncthreads();
        // new row j = the scaled pivot row; every other row i (row pr taking
        // the old row j's values) eliminated: x_q -= l pj_q, x_jj = -l d
        const int pr = s_pr;
        const C d = s_d;
        C pj[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) pj[q] = q < nbp ? s_pj[q] : czero<C>();
        for (int i = tid; i < M; i += nt) {
            if (i == j) {
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q < nbp) P[q * M + i] = pj[q];
                continue;
            }
            const bool sw = i == pr;
            const C l = sw ? s_oj[jj] : P[jj * M + i];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (q >= nbp) break;
                const C x = sw ? s_oj[q] : P[q * M + i];
                P[q * M + i] = (q == jj) ? czero<C>() - l * d : x - l * pj[q];
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < M * nbp; e += nt) {
        const int r = e / nbp, q = e % nbp;
        w[(long long)r * M + j0 + q] = P[q * M + r];
    }
}

// Outside the panel columns: apply the panel's row swaps; for the columns in
// [c_lo, c_hi) also move the pivot rows' entries into T (T[jj][c], zero for c
// in J) and zero them in W (the columns the following update covers).  The
// swaps touch at most 2 nbp rows; their composition (row x receives the old
// row src[x]) is worked out once per CTA, then every column is a gather: all
// loads first, then the stores.
template <typename C, int NB>
__global__ void f3_swap_extract(const Slab3* __restrict__ slabs, C* __restrict__ W, const int* __restrict__ piv,
                                C* __restrict__ T, int j0, int Tld, int c_lo, int c_hi) {
    __shared__ int rows[2 * NB], src[2 * NB], nrows_s;
    const int slab = blockIdx.y;
    const Slab3 sd = slabs[slab];
    const int M = sd.M;
    if (j0 >= M) return;
    const int nbp = min(NB, M - j0);
    if (threadIdx.x == 0) {
        int na = 0;
        for (int jj = 0; jj < nbp; ++jj) rows[na++] = j0 + jj;
        for (int jj = 0; jj < nbp; ++jj) {
            const int r = piv[slab * NB + jj];
            bool seen = false;
            for (int q = 0; q < na; ++q) seen |= rows[q] == r;
            if (!seen) rows[na++] = r;
        }
        for (int q = 0; q < na; ++q) src[q] = rows[q];
        for (int jj = 0; jj < nbp; ++jj) {
            const int r = piv[slab * NB + jj];
            int pr = 0;
            while (rows[pr] != r) ++pr;
            const int tmp = src[jj];
            src[jj] = src[pr];
            src[pr] = tmp;
        }
        nrows_s = na;
    }
    __syncthreads();
    const int na = nrows_s;
    C* w = W + sd.w_off;
    C* t = T + (long long)slab * NB * Tld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
        const bool local = c >= c_lo && c < c_hi;
        if (c >= j0 && c < j0 + nbp) {
            if (local)
                for (int jj = 0; jj < nbp; ++jj) t[(long long)jj * Tld + c] = czero<C>();
            continue;
        }
        C v[2 * NB];
#pragma unroll
        for (int q = 0; q < 2 * NB; ++q)
            if (q < na) v[q] = w[(long long)src[q] * M + c];
#pragma unroll
        for (int q = 0; q < 2 * NB; ++q) {
            if (q >= na) break;
            if (q < nbp && local) {
                t[(long long)q * Tld + c] = v[q];
                w[(long long)rows[q] * M + c] = czero<C>();
            } else {
                w[(long long)rows[q] * M + c] = v[q];
            }
        }
    }
}

// W[i][c] += sum_kk W[i][j0+kk] T[kk][c] for c in [c_lo, c_hi) outside J
// (CUDA cores).  64 x 64 output tiles, 256 threads, 4 x 4 entries each.
// grid (row tiles x column tiles of the range, slabs).
template <typename C, int NB>
__global__ void __launch_bounds__(256) f3_update_cc(const Slab3* __restrict__ slabs, C* __restrict__ W,
                                                    const C* __restrict__ T, int j0, int Tld, int c_lo, int c_hi) {
    __shared__ C As[64][NB];
    __shared__ C Ts[NB][64];
    const int slab = blockIdx.y;
    const Slab3 sd = slabs[slab];
    const int M = sd.M;
    if (j0 >= M) return;
    const int nbp = min(NB, M - j0);
    const int ce = min(c_hi, M);
    if (ce <= c_lo) return;
    const int tiles = (M + 63) / 64, ctiles = (ce - c_lo + 63) / 64;
    if ((int)blockIdx.x >= tiles * ctiles) return;
    const int i0 = (blockIdx.x / ctiles) * 64, c0 = c_lo + (blockIdx.x % ctiles) * 64;
    C* w = W + sd.w_off;
    const C* t = T + (long long)slab * NB * Tld;
    const int tid = threadIdx.x;
    for (int e = tid; e < 64 * NB; e += 256) {
        const int i = e / NB, q = e % NB;
        As[i][q] = (i0 + i < M && q < nbp) ? w[(long long)(i0 + i) * M + j0 + q] : czero<C>();
    }
    for (int e = tid; e < NB * 64; e += 256) {
        const int q = e / 64, c = e % 64;
        Ts[q][c] = (c0 + c < ce && q < nbp) ? t[(long long)q * Tld + c0 + c] : czero<C>();
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;
    C acc[4][4];
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) acc[u][v] = czero<C>();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        C a[4], b[4];
        for (int u = 0; u < 4; ++u) a[u] = As[ty + 16 * u][q];
        for (int v = 0; v < 4; ++v) b[v] = Ts[q][tx + 16 * v];
        for (int u = 0; u < 4; ++u)
            for (int v = 0; v < 4; ++v) acc[u][v] = cfma(a[u], b[v], acc[u][v]);
    }
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty + 16 * u;
        if (i >= M) continue;
        for (int v = 0; v < 4; ++v) {
            const int c = c0 + tx + 16 * v;
            if (c >= ce || (c >= j0 && c < j0 + nbp)) continue;
            C* p = w + (long long)i * M + c;
            *p = *p + acc[u][v];
        }
    }
}

// The outer panel [J0, J0 + nbo) is eliminated (its rows are already swapped
// everywhere): for the columns outside it move the pivot rows into T64
// (T64[kk][c], kk < nbo) and zero them in W; zero T64 inside the panel.
template <typename C>
__global__ void f3_extract_outer(const Slab3* __restrict__ slabs, C* __restrict__ W, C* __restrict__ T64, int J0,
                                 int NO, int Tld) {
    const int slab = blockIdx.y;
    const Slab3 sd = slabs[slab];
    const int M = sd.M;
    if (J0 >= M) return;
    const int nbo = min(NO, M - J0);
    C* w = W + sd.w_off;
    C* t = T64 + (long long)slab * NO * Tld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
        const bool inside = c >= J0 && c < J0 + nbo;
        for (int k0 = 0; k0 < nbo; k0 += 16) {   // 16 independent loads, then the stores
            C v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u)
                v[u] = (!inside && k0 + u < nbo) ? w[(long long)(J0 + k0 + u) * M + c] : czero<C>();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                if (k0 + u >= nbo) break;
                t[(long long)(k0 + u) * Tld + c] = v[u];
                if (!inside) w[(long long)(J0 + k0 + u) * M + c] = czero<C>();
            }
        }
    }
}

// Dinv_k[i][rowid[r]] = W[i][r]: the column permutation undoing the row
// interchanges, stored as factor block k.
template <typename C>
__global__ void f3_finalize(const Slab3* __restrict__ slabs, const C* __restrict__ W, const int* __restrict__ rowid,
                            C* __restrict__ fac, int k, int Mmax) {
    extern __shared__ int inv[];
    const int slab = blockIdx.y;
    const Slab3 sd = slabs[slab];
    const int M = sd.M;
    const int* rid = rowid + (long long)slab * Mmax;
    for (int r = threadIdx.x; r < M; r += blockDim.x) inv[rid[r]] = r;
    __syncthreads();
    const long long MM = (long long)M * M;
    const C* w = W + sd.w_off;
    C* out = fac + sd.fac_off + (long long)k * MM;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MM;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / M), j = (int)(e % M);
        out[e] = w[(long long)i * M + inv[j]];
    }
}

// ---------------------------------------------------------------- sweep (Algorithm 2, 3D slabs)

// One step of up to two slab solves that advance together: block row k of the
// block-tridiagonal solve, dir 0 = forward substitution, 1 = backward.  One
// front runs one slab solve at a time; two fronts (Sec. 2.4 remark 1) pair a
// slab of the left front with one of the right front (slab[1] = -1: none), the
// grid split in two halves.  Per slab, flags:
//   S3_FWD  the forward sweep's solve: input f_i minus the couplings, result
//           assigned; without it the backward correction: input the couplings,
//           result subtracted;
//   S3_CL   coupling H_{[i,i-1]} u_{i-1} into D_i's first layer;
//   S3_CR   coupling H_{[i,i+1]} u_{i+1} into D_i's last layer.
enum { S3_FWD = 1, S3_CL = 2, S3_CR = 4 };
struct Step3 {
    int dir, k;
    int slab[2];
    int flags[2];
};

struct Sweep3Args {
    const Slab3* slabs;
    const Step3* steps;
    int nsteps, n_tot, b, Mmax;
    const void* coef;
    const void* fac;
    const void* f;      // sparsified right-hand sides on the grid (R)
    void* ut;           // sweep solution on the grid (R)
    void* Y;            // block substitution vectors, per group of the grid: [2][r][k][Mmax]
    void* TB;           // split mode: the step input t, per group: [2][r][Mmax]
    int R;              // right-hand sides in this launch (<= kSweepRB)
    long long G;        // n_tot^3
    unsigned dcap;      // bytes of the shared-memory buffer for D_k^{-1} rows
    unsigned* bar;
    int* err;
};

// The half of the grid a CTA works in for a step: group g, its block index lb
// within the group and the group's size Gg.
struct Group3 { int g, lb, Gg; };
__device__ __forceinline__ Group3 group_of(const Step3& st, int G) {
    if (st.slab[1] < 0) return Group3{0, (int)blockIdx.x, G};
    const int h = G / 2;
    return (int)blockIdx.x < h ? Group3{0, (int)blockIdx.x, h} : Group3{1, (int)blockIdx.x - h, G - h};
}

// The coupling of layer a's rows with the neighbouring slab's layer at grid
// x1-index X1o (x1-offset slot d1 = 0 for -1, 2 for +1): sum over the 3 x 3
// (x2, x3) neighbours of block row k.
template <typename C>
__device__ __forceinline__ C layer_coupling(const Sweep3Args& A, const C* cf, int M, int k, int q, int c, int d1,
                                            int X1o, int r) {
    const C* ut = (const C*)A.ut;
    const int nt = A.n_tot, K = A.n_tot;
    const C* rowc = cf + (long long)k * 3 * M * 9;
    C v = czero<C>();
    for (int d2 = -1; d2 <= 1; ++d2) {
        const int k2 = k + d2;
        if (k2 < 0 || k2 >= K) continue;
        for (int d3 = -1; d3 <= 1; ++d3) {
            const int c3 = c + d3;
            if (c3 < 0 || c3 >= nt) continue;
            v = cfma(rowc[((long long)(d2 + 1) * M + q) * 9 + d1 * 3 + (d3 + 1)],
                     ut[r * A.G + ((long long)X1o * nt + k2) * nt + c3], v);
        }
    }
    return v;
}

// Input t_q of one step for right-hand side r, entry q = (a, c) of block k of
// the slab sd (flags fl); Yr = this right-hand side's substitution vectors.
template <typename C>
__device__ __forceinline__ C step_input(const Sweep3Args& A, const Slab3& sd, int fl, int dir, int k, int r, int q,
                                        const C* Yr) {
    const C* coef = (const C*)A.coef;
    const C* f = (const C*)A.f;
    const int nt = A.n_tot, M = sd.M, w = sd.w, na = sd.na;
    const int a = q / nt, c = q % nt;
    const int X1s = sd.s + A.b;
    const C* cf = coef + sd.cf_off;
    C v = czero<C>();
    if (dir == 0) {
        C cpl = czero<C>();
        if ((fl & S3_CL) && a == na) cpl = cpl + layer_coupling<C>(A, cf, M, k, q, c, 0, X1s - 1, r);
        if ((fl & S3_CR) && a == sd.ll) cpl = cpl + layer_coupling<C>(A, cf, M, k, q, c, 2, X1s + sd.nl, r);
        if (fl & S3_FWD) {
            if (a >= na && a <= sd.ll) v = f[r * A.G + ((long long)(X1s + a - na) * nt + k) * nt + c];
            v = v - cpl;
        } else {
            v = cpl;
        }
        if (k > 0) {                                      // - C_k y_{k-1}
            const C* cc = cf + ((long long)k * 3 + 0) * M * 9 + (long long)q * 9;
            const C* yp = Yr + (long long)(k - 1) * A.Mmax;
            for (int d1 = -1; d1 <= 1; ++d1) {
                const int a1 = a + d1;
                if (a1 < 0 || a1 >= w) continue;
                for (int d3 = -1; d3 <= 1; ++d3) {
                    const int c3 = c + d3;
                    if (c3 < 0 || c3 >= nt) continue;
                    v = v - cc[(d1 + 1) * 3 + (d3 + 1)] * yp[a1 * nt + c3];
                }
            }
        }
    } else {                                              // B_k x_{k+1}
        const C* bc = cf + ((long long)k * 3 + 2) * M * 9 + (long long)q * 9;
        const C* xn = Yr + (long long)(k + 1) * A.Mmax;
        for (int d1 = -1; d1 <= 1; ++d1) {
            const int a1 = a + d1;
            if (a1 < 0 || a1 >= w) continue;
            for (int d3 = -1; d3 <= 1; ++d3) {
                const int c3 = c + d3;
                if (c3 < 0 || c3 >= nt) continue;
                v = cfma(bc[(d1 + 1) * 3 + (d3 + 1)], xn[a1 * nt + c3], v);
            }
        }
    }
    return v;
}

// Rows [r0, r1) of D_k^{-1} of slab i that block lb of a group of Gg blocks
// owns, as a 16-byte aligned byte window [lo, lo + bytes) of the factor array;
// off = byte offset of the first row.
struct RowWin { unsigned long long lo; unsigned bytes, off; int r0, r1; };
template <typename C>
__device__ __forceinline__ RowWin row_window(const Sweep3Args& A, int i, int k, int lb, int Gg) {
    const Slab3 sd = A.slabs[i];
    const int M = sd.M;
    RowWin wdw;
    wdw.r0 = (int)((long long)lb * M / Gg);
    wdw.r1 = (int)((long long)(lb + 1) * M / Gg);
    const unsigned long long a = (unsigned long long)((const C*)A.fac + sd.fac_off + (long long)k * M * M +
                                                      (long long)wdw.r0 * M);
    const unsigned long long e = a + (unsigned long long)(wdw.r1 - wdw.r0) * M * sizeof(C);
    wdw.lo = a & ~15ull;
    wdw.bytes = (unsigned)(((e + 15ull) & ~15ull) - wdw.lo);
    wdw.off = (unsigned)(a - wdw.lo);
    return wdw;
}
template <typename C>
__device__ __forceinline__ RowWin step_window(const Sweep3Args& A, const Step3& st, int G) {
    const Group3 gr = group_of(st, G);
    return row_window<C>(A, st.slab[gr.g], st.k, gr.lb, gr.Gg);
}

// One CTA per SM, persistent, walking the host-built step table.  Each step:
// the input t of the step in shared memory, this CTA's rows of D_k^{-1} t
// (the rows arrive by a bulk copy issued before the previous step's grid
// barrier whenever they fit the buffer), the outputs, a grid barrier.
// Forward substitution y_k = D_k^{-1}(v_k - C_k y_{k-1}), backward
// x_k = y_k - D_k^{-1} B_k x_{k+1}.  A paired step runs two slab solves, one
// per half of the grid.  SPLIT: each CTA forms only its own rows of t,
// exchanged through global memory and a second grid barrier (FP64, where
// forming the whole t in every CTA would cost more arithmetic than the
// product itself); otherwise every CTA forms all of its slab's t.
template <typename C, bool SPLIT>
__global__ void __launch_bounds__(kSweepThreads) sweep3_kernel(Sweep3Args A) {
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smraw);
    unsigned char* dbuf = smraw + 128;
    C* t = reinterpret_cast<C*>(dbuf + A.dcap);            // [R][Mmax]
    C* part = t + (size_t)A.R * A.Mmax;                    // [warps][kSweepRB]
    C* ut = (C*)A.ut;
    const int nt = A.n_tot, K = A.n_tot, G = gridDim.x, tid = threadIdx.x;
    const int nwarps = blockDim.x / 32, wid = tid / 32, lane = tid & 31;
    const long long ystride = (long long)A.R * K * A.Mmax;   // one group's substitution vectors
    unsigned nbar = 0;   // grid barriers passed (the arrival counter starts at zero)
    // s_pending: thread 0 issued the bulk copy of the current step's rows
    // (decided by thread 0 alone, read by all after a barrier, so that the
    // whole CTA agrees; no copy is issued once a wait has expired)
    __shared__ int s_pending;
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        s_pending = 0;
        if (A.nsteps > 0) {
            const RowWin wn = step_window<C>(A, A.steps[0], G);
            if (wn.r1 > wn.r0 && wn.bytes <= A.dcap) {
                mbar_expect_tx(mbar, wn.bytes);
                tma_load_1d(dbuf, (const void*)wn.lo, wn.bytes, mbar);
                s_pending = 1;
            }
        }
    }
    __syncthreads();
    unsigned pcount = 0;   // bulk copies completed so far (mbarrier phase)
    for (int s = 0; s < A.nsteps; ++s) {
        const Step3 st = A.steps[s];
        const Group3 gr = group_of(st, G);
        const int slab = st.slab[gr.g], fl = st.flags[gr.g];
        const Slab3 sd = A.slabs[slab];
        const int M = sd.M, k = st.k, na = sd.na;
        const int X1s = sd.s + A.b;
        C* Y = (C*)A.Y + gr.g * ystride;
        C* TB = (C*)A.TB + (long long)gr.g * A.R * A.Mmax;
        const RowWin wn = row_window<C>(A, slab, k, gr.lb, gr.Gg);
        const int r0 = wn.r0, nrows = wn.r1 - wn.r0;
        const int P = nrows > 0 ? max(1, nwarps / nrows) : 1;
        // ---- t
        if (SPLIT) {
            for (int e = tid; e < nrows * A.R; e += blockDim.x) {
                const int r = e / nrows, q = r0 + e % nrows;
                TB[(size_t)r * A.Mmax + q] =
                    step_input<C>(A, sd, fl, st.dir, k, r, q, Y + (long long)r * K * A.Mmax);
            }
            grid_barrier_count(A.bar, (++nbar) * (unsigned)G, A.err);
            for (int e = tid; e < A.R * M; e += blockDim.x) {
                const int r = e / M, q = e % M;
                t[(size_t)r * A.Mmax + q] = TB[(size_t)r * A.Mmax + q];
            }
        } else {
            const int tot = A.R * M;
            for (int e = tid; e < tot; e += 2 * blockDim.x) {
                const int e2 = e + blockDim.x;
                const int ra = e / M, rb = e2 / M;
                const C v1 = step_input<C>(A, sd, fl, st.dir, k, ra, e % M, Y + (long long)ra * K * A.Mmax);
                C v2 = czero<C>();
                if (e2 < tot) v2 = step_input<C>(A, sd, fl, st.dir, k, rb, e2 % M, Y + (long long)rb * K * A.Mmax);
                t[(size_t)ra * A.Mmax + e % M] = v1;
                if (e2 < tot) t[(size_t)rb * A.Mmax + e2 % M] = v2;
            }
        }
        __syncthreads();
        // ---- this CTA's rows of D_k^{-1} t
        const C* Dg = (const C*)A.fac + sd.fac_off + (long long)k * M * M;
        const C* Drows = Dg + (long long)r0 * M;
        if (s_pending) {
            if (mbar_wait(mbar, pcount & 1u, A.err)) Drows = reinterpret_cast<const C*>(dbuf + wn.off);
            ++pcount;     // (expired: read the rows from global memory)
        }
        if (nrows > 0 && wid < nrows * P) {
            const int lr = wid / P, pp = wid % P;
            const int cb = (int)((long long)pp * M / P), ce = (int)((long long)(pp + 1) * M / P);
            C acc[kSweepRB];
            for (int r = 0; r < kSweepRB; ++r) acc[r] = czero<C>();
            const C* Drow = Drows + (long long)lr * M;
#pragma unroll 4
            for (int j = cb + lane; j < ce; j += 32) {
                const C dv = Drow[j];
                for (int r = 0; r < kSweepRB; ++r)
                    if (r < A.R) acc[r] = cfma(dv, t[(size_t)r * A.Mmax + j], acc[r]);
            }
            for (int r = 0; r < kSweepRB; ++r) {
                if (r >= A.R) break;
                for (int o = 16; o > 0; o >>= 1) {
                    acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
                    acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
                }
                if (lane == 0) part[(size_t)wid * kSweepRB + r] = acc[r];
            }
        }
        __syncthreads();
        // ---- the next step's rows: the buffer is free again
        if (tid == 0) {
            s_pending = 0;
            if (s + 1 < A.nsteps && !(*(volatile int*)A.err & LSS_DERR_TIMEOUT)) {
                const RowWin nx = step_window<C>(A, A.steps[s + 1], G);
                if (nx.r1 > nx.r0 && nx.bytes <= A.dcap) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(mbar, nx.bytes);
                    tma_load_1d(dbuf, (const void*)nx.lo, nx.bytes, mbar);
                    s_pending = 1;
                }
            }
        }
        // ---- outputs
        for (int e = tid; e < nrows * A.R; e += blockDim.x) {
            const int lr = e / A.R, r = e % A.R;
            const int row = r0 + lr;
            C sum = czero<C>();
            for (int pp = 0; pp < P; ++pp) sum = sum + part[(size_t)(lr * P + pp) * kSweepRB + r];
            C* yk = Y + (long long)r * K * A.Mmax + (long long)k * A.Mmax + row;
            const C val = st.dir == 0 ? sum : *yk - sum;
            *yk = val;
            const bool final_x = st.dir == 1 || k == K - 1;
            const int a = row / nt, c = row % nt;
            if (final_x && a >= na && a <= sd.ll) {
                C* up = ut + r * A.G + ((long long)(X1s + a - na) * nt + k) * nt + c;
                *up = (fl & S3_FWD) ? val : *up - val;
            }
        }
        grid_barrier_count(A.bar, (++nbar) * (unsigned)G, A.err);
    }
    if (s_pending) mbar_wait(mbar, pcount & 1u, A.err);   // nothing may stay in flight at exit
}


__global__ void f2_to_d2_kernel(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = make_double2(a[e].x, a[e].y);
}

void extract_f2_to_d2(double2* dst, const float2* src, long long n, int num_sms, cudaStream_t s) {
    f2_to_d2_kernel<<<2 * num_sms, 256, 0, s>>>(src, dst, n);
}

}  // namespace

// ---------------------------------------------------------------- host side

void lss3_free(lss_ctx* c) {
    Ctx3* d = c->d3;
    if (!d) return;
    lss3r_free(c);
    void* ptrs[] = {d->d_slabs, d->khat, d->gam_phys, d->gam_aux, d->gam_aux_r, d->coef64, d->coef == d->coef64 ? nullptr : d->coef,
                    d->fac, d->W, d->X, d->T, d->piv, d->rowid, d->f, d->ut, d->Y, d->mvA, d->mvB, d->TB,
                    d->steps_all, d->steps_one, d->T64};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete d;
    c->d3 = nullptr;
}

long long lss3_N(const lss_ctx* c) { return (long long)c->n * c->n * c->n; }

namespace {

int dalloc3(lss_ctx* c, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return lss_fail(c, LSS_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    return LSS_OK;
}

int configure3(lss_ctx* c) {
    std::lock_guard<std::mutex> lock(lss_config_mutex());
    long long& done = lss_dev_cache((const void*)&configure3, 0);
    if (done) return LSS_OK;
    const int smax = 200 * 1024;
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(mv3_rows_fwd<MV_IN_MU>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_rows_fwd<MV_IN_U>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_rows_fwd<MV_IN_PLANEWAVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_rows_fwd<MV_IN_RAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_rows_inv<MV_OUT_A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_rows_inv<MV_OUT_AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_rows_inv<MV_OUT_NEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_cols<COL_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_cols<COL_CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_cols<COL_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv3_cols<COL_KHAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    const int psm = 210 * 1024;
    const int panel = kMaxBlock3 * kNB64 * (int)sizeof(double2);   // = kMaxBlock3 * kNB32 * sizeof(float2)
    if (!e) e = cudaFuncSetAttribute(f3_panel<double2, kNB64>, cudaFuncAttributeMaxDynamicSharedMemorySize, panel);
    if (!e) e = cudaFuncSetAttribute(f3_panel<float2, kNB32>, cudaFuncAttributeMaxDynamicSharedMemorySize, panel);
    if (!e) e = cudaFuncSetAttribute(sweep3_kernel<double2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, psm);
    if (!e) e = cudaFuncSetAttribute(sweep3_kernel<float2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, psm);
    if (e) return lss_check_cuda(c, e, "3D kernel attributes");
    done = 1;
    return LSS_OK;
}

// Kernel transform: khat[(k2*L + k3)*L + k1] = omega^2/L^3 FFT3(kc)[k1][k2][k3].
int build_kernel3(lss_ctx* c, cudaStream_t s) {
    Ctx3* d = c->d3;
    const int L = c->L, lg = c->lgL;
    std::vector<double2> tw(L);
    for (int k = 0; k < L; ++k) {
        const long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)L;
        tw[k] = make_double2((double)cosl(a), (double)sinl(a));
    }
    int rc = lss_check_cuda(c, cudaMemcpyAsync(c->tw, tw.data(), L * sizeof(double2), cudaMemcpyHostToDevice, s),
                            "twiddles");
    if (rc) return rc;
    const cd k0 = lss_cell_integral_G(3, c->omega, c->h);
    const long long L3 = (long long)L * L * L;
    double2 *kc = nullptr, *tmp = nullptr;
    rc = dalloc3(c, (void**)&kc, L3 * sizeof(double2), "k table");
    if (!rc) rc = dalloc3(c, (void**)&tmp, L3 * sizeof(double2), "k table fft");
    if (rc) { if (kc) cudaFree(kc); return rc; }
    const int nt = line_threads3(L);
    const size_t sh = 2 * (size_t)L * sizeof(double2);
    const int C = col_group3(L);
    {
        ProfScope ps(c, s, LSS_PROF_SETUP, 4);
        k3_table_circ<<<4 * c->num_sms, 256, 0, s>>>(kc, c->n, L, c->omega, c->h, make_double2(k0.real(), k0.imag()));
        mv3_rows_fwd<MV_IN_RAW><<<dim3(L * L, 1), nt, sh, s>>>(kc, nullptr, nullptr, nullptr, tmp, c->tw, c->n, L * L,
                                                              L, lg, c->omega, c->h);
        // along x2: [j1][j2][k3] -> [j1][k2][k3]
        mv3_cols<COL_FWD><<<dim3(L / C, L, 1), C * nt, 2 * (size_t)C * L * sizeof(double2), s>>>(
            tmp, kc, nullptr, c->tw, L, L, L, L, L, lg, C, 1.0);
        // along x1, stored transposed and scaled
        const double scale = c->omega * c->omega / ((double)L * L * L);
        mv3_cols<COL_KHAT><<<dim3((unsigned)((long long)L * L / C), 1, 1), C * nt, 2 * (size_t)C * L * sizeof(double2),
                             s>>>(kc, d->khat, nullptr, c->tw, 1, L, L, (long long)L * L, L, lg, C, scale);
    }
    rc = lss_check_cuda(c, cudaGetLastError(), "3D kernel table");
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(kc);
    cudaFree(tmp);
    if (!rc) rc = lss_check_cuda(c, e, "3D kernel table");
    return rc;
}

// alpha (smallest eigenvector of the 27 x 27 Gram matrix of K_{mu,mu^c}) and
// beta^* = alpha^* K_{mu,mu} (Eq. alpha, Eq. beta in 3D).
int build_interior3(lss_ctx* c, cudaStream_t s) {
    Ctx3* d = c->d3;
    const int n = c->n, S = 2 * n + 3;
    const cd k0 = lss_cell_integral_G(3, c->omega, c->h);
    const int nblk = 2 * c->num_sms, npair = 27 * 28 / 2;
    double2 *kx = nullptr, *part = nullptr;
    int rc = dalloc3(c, (void**)&kx, (size_t)S * S * S * sizeof(double2), "k ext 3D");
    if (!rc) rc = dalloc3(c, (void**)&part, (size_t)npair * nblk * sizeof(double2), "gram 3D");
    if (rc) { if (kx) cudaFree(kx); return rc; }
    {
        ProfScope ps(c, s, LSS_PROF_SETUP, 2);
        k3_table_ext<<<4 * c->num_sms, 256, 0, s>>>(kx, n, c->omega, c->h, make_double2(k0.real(), k0.imag()));
        gram3_partial<<<dim3(nblk, npair), 256, 0, s>>>(kx, n, part);
    }
    std::vector<double2> hp((size_t)npair * nblk), k5(125);
    cudaError_t e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, s);
    for (int u = 0; u < 5 && !e; ++u)
        for (int v = 0; v < 5 && !e; ++v)
            e = cudaMemcpyAsync(&k5[(u * 5 + v) * 5], kx + ((size_t)(n - 1 + u) * S + (n - 1 + v)) * S + (n - 1),
                                5 * sizeof(double2), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    cudaFree(kx);
    cudaFree(part);
    if (e) return lss_check_cuda(c, e, "gram 3D");
    std::vector<cd> Gm(27 * 27);
    int pair = 0;
    for (int a = 0; a < 27; ++a)
        for (int b = a; b < 27; ++b, ++pair) {
            cd acc = 0;
            for (int q = 0; q < nblk; ++q) acc += cd(hp[(size_t)pair * nblk + q].x, hp[(size_t)pair * nblk + q].y);
            Gm[a * 27 + b] = acc;
            Gm[b * 27 + a] = std::conj(acc);
        }
    std::vector<double> A(54 * 54);
    for (int a = 0; a < 27; ++a)
        for (int b = 0; b < 27; ++b) {
            A[a * 54 + b] = Gm[a * 27 + b].real();
            A[a * 54 + 27 + b] = -Gm[a * 27 + b].imag();
            A[(27 + a) * 54 + b] = Gm[a * 27 + b].imag();
            A[(27 + a) * 54 + 27 + b] = Gm[a * 27 + b].real();
        }
    std::vector<double> ev, V;
    lss_jacobi_eigen(A, 54, ev, V);
    int imin = 0;
    for (int i = 1; i < 54; ++i)
        if (ev[i] < ev[imin]) imin = i;
    cd al[27];
    double nrm = 0;
    for (int a = 0; a < 27; ++a) {
        al[a] = cd(V[a * 54 + imin], V[(27 + a) * 54 + imin]);
        nrm += std::norm(al[a]);
    }
    nrm = std::sqrt(nrm);
    const cd ph = std::abs(al[13]) / al[13];
    for (int a = 0; a < 27; ++a) al[a] = al[a] * ph / nrm;
    al[13] = cd(std::abs(al[13]), 0.0);
    for (int b = 0; b < 27; ++b) {
        cd acc = 0;
        for (int a = 0; a < 27; ++a) {
            const int e1 = a / 9 - b / 9, e2 = (a / 3) % 3 - (b / 3) % 3, e3 = a % 3 - b % 3;
            const double2 kab = k5[((e1 + 2) * 5 + (e2 + 2)) * 5 + (e3 + 2)];
            acc += al[a] * std::conj(cd(kab.x, kab.y));   // beta_b = sum_a alpha_a conj(K_ab)
        }
        d->beta[b] = acc;
    }
    for (int a = 0; a < 27; ++a) d->alpha[a] = al[a];
    return LSS_OK;
}

Stencil27 stencil_args(const Ctx3* d, double omega) {
    (void)omega;
    Stencil27 st;
    for (int o = 0; o < 27; ++o) {
        st.a_conj[o] = make_double2(d->alpha[o].real(), -d->alpha[o].imag());
        st.b_conj[o] = make_double2(d->beta[o].real(), -d->beta[o].imag());
    }
    return st;
}

}  // namespace

int lss3_setup(lss_ctx* c, const double* m_dev, cudaStream_t s) {
    Ctx3* d = new Ctx3();
    c->d3 = d;
    const int n = c->n, b = c->b, bs = c->slab.b_slab;
    const int nl = (n + 2 + bs - 1) / bs;
    c->n_slabs = nl;
    long long cf = 0, fo = 0, wo = 0;
    d->Mmax = 0;
    c->mid = (nl - 1) / 2;
    for (int i = 0; i < nl; ++i) {
        Slab3 sd{};
        if (i == 0) {
            sd.s = -b;
            sd.nl = (nl == 1) ? c->n_tot : b + bs;
        } else {
            sd.s = i * bs;
            sd.nl = (i == nl - 1) ? (n + 2 - i * bs) + b : bs;
        }
        // one front: every slab but the first padded on the left; two fronts:
        // left of the middle slab on the left, right of it on the right, the
        // middle slab on both sides
        const bool left = c->fronts == 2 ? (i > 0 && i <= c->mid) : i > 0;
        const bool right = c->fronts == 2 && i >= c->mid && i < nl - 1;
        sd.na = left ? c->b_aux : 0;
        sd.nr = right ? c->b_aux : 0;
        sd.ll = sd.na + sd.nl - 1;
        sd.w = sd.na + sd.nl + sd.nr;
        sd.nc = c->n_tot;
        sd.oi = i;
        sd.M = sd.w * c->n_tot;
        if (sd.M > kMaxBlock3 && !c->slab.recursive)
            return lss_fail(c, LSS_ERR_UNSUPPORTED, "3D: a slab block (layers x n_tot) exceeds 1760 unknowns");
        sd.cf_off = cf;
        sd.fac_off = fo;
        sd.w_off = wo;
        cf += (long long)c->n_tot * 3 * sd.M * 9;
        fo += (long long)c->n_tot * sd.M * sd.M;
        wo += (long long)sd.M * sd.M;
        d->Mmax = std::max(d->Mmax, sd.M);
        d->slabs.push_back(sd);
    }
    d->coef_len = cf;
    d->fac_len = fo;
    d->w_len = wo;
    const int nc = 2 * b + 1;
    const size_t cs = c->csize();
    const long long L3 = (long long)c->L * c->L * c->L;
    const int NB = c->prec == LSS_FP64 ? kNB64 : kNB32;
    int rc = LSS_OK;
    rc = rc ? rc : dalloc3(c, (void**)&c->m, (size_t)lss3_N(c) * sizeof(double), "m");
    rc = rc ? rc : dalloc3(c, (void**)&c->tw, (size_t)c->L * sizeof(double2), "twiddles");
    rc = rc ? rc : dalloc3(c, (void**)&d->khat, (size_t)L3 * sizeof(double2), "kernel transform");
    rc = rc ? rc : dalloc3(c, (void**)&d->gam_phys, (size_t)nc * nc * nc * 27 * sizeof(double2), "gamma");
    rc = rc ? rc : dalloc3(c, (void**)&d->gam_aux, (size_t)c->n_samples * c->b_aux * nc * nc * 27 * sizeof(double2),
                           "gamma aux");
    if (c->fronts == 2)
        rc = rc ? rc : dalloc3(c, (void**)&d->gam_aux_r,
                               (size_t)c->n_samples * c->b_aux * nc * nc * 27 * sizeof(double2), "gamma aux right");
    rc = rc ? rc : dalloc3(c, (void**)&d->coef64, (size_t)cf * sizeof(double2), "coefficients");
    if (!rc) {
        if (c->prec == LSS_FP64) d->coef = d->coef64;
        else rc = dalloc3(c, &d->coef, (size_t)cf * cs, "coefficients fp32");
    }
    if (!c->slab.recursive) {   // (the recursive approach factors the sub-slab problems instead)
        // 64 bytes of slack: the sweep copies 16-byte aligned windows of rows that
        // may end up to 15 bytes past the last factor entry
        rc = rc ? rc : dalloc3(c, &d->fac, (size_t)fo * cs + 64, "slab factors");
        rc = rc ? rc : dalloc3(c, &d->W, (size_t)wo * cs, "pivot blocks");
        rc = rc ? rc : dalloc3(c, &d->X, (size_t)wo * cs, "Schur scratch");
        rc = rc ? rc : dalloc3(c, &d->T, (size_t)nl * NB * d->Mmax * cs, "panel rows");
        if (c->prec == LSS_MIXED)
            rc = rc ? rc : dalloc3(c, &d->T64, (size_t)nl * kNO * d->Mmax * cs, "outer panel rows");
        rc = rc ? rc : dalloc3(c, (void**)&d->piv, (size_t)nl * NB * sizeof(int), "pivots");
        rc = rc ? rc : dalloc3(c, (void**)&d->rowid, (size_t)nl * d->Mmax * sizeof(int), "row ids");
    }
    rc = rc ? rc : dalloc3(c, (void**)&d->d_slabs, nl * sizeof(Slab3), "slabs");
    rc = rc ? rc : dalloc3(c, (void**)&c->d_err, sizeof(int), "status");
    rc = rc ? rc : dalloc3(c, (void**)&c->d_bar, 2 * sizeof(unsigned), "barrier");
    if (rc) return rc;
    cudaMemcpyAsync(d->d_slabs, d->slabs.data(), nl * sizeof(Slab3), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), s);
    cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), s);
    rc = configure3(c);
    if (!rc) rc = build_kernel3(c, s);
    if (!rc) rc = build_interior3(c, s);
    if (!rc && c->slab.recursive) rc = lss3r_setup(c, s);
    if (!rc) {
        ProfScope ps(c, s, LSS_PROF_SETUP, 1);
        const int tot = nc * nc * nc;
        gamma3_phys_kernel<<<(tot + kGamWarps - 1) / kGamWarps, 32 * kGamWarps, 0, s>>>(
            d->gam_phys, n, b, c->pml.C / c->omega, c->omega, c->h);
        rc = lss_check_cuda(c, cudaGetLastError(), "gamma 3D");
    }
    return rc;
}

// Medium-dependent part (after the sample range is set): moving-PML stencils,
// slab coefficients (and their single-precision copy).
int lss3_set_medium(lss_ctx* c, cudaStream_t s) {
    Ctx3* d = c->d3;
    const int n = c->n, b = c->b, nc = 2 * b + 1;
    const long long tot = (long long)c->ns_eff * c->b_aux * nc * nc;
    const int nside = c->fronts == 2 ? 2 : 1;
    ProfScope ps(c, s, LSS_PROF_SETUP, (c->prec == LSS_MIXED ? 2 : 1) + nside);
    for (int right = 0; right < nside; ++right)
        gamma3_aux_kernel<<<(unsigned)((tot + kGamWarps - 1) / kGamWarps), 32 * kGamWarps, 0, s>>>(
            right ? d->gam_aux_r : d->gam_aux, n, b, c->b_aux, c->ns_eff, c->s_lo, c->s_hi, c->pml.C / c->omega, c->h,
            right);
    const Stencil27 st = stencil_args(d, c->omega);
    assemble3_kernel<<<dim3(2 * c->num_sms, c->n_slabs), 256, 0, s>>>(d->d_slabs, c->m, d->gam_phys, d->gam_aux,
                                                                     d->gam_aux_r, st,
                                                                     d->coef64, n, b, c->b_aux, c->n_tot, c->ns_eff,
                                                                     c->s_lo, c->s_hi, c->omega);
    if (c->prec == LSS_MIXED)
        cast3_kernel<<<4 * c->num_sms, 256, 0, s>>>(d->coef64, (float2*)d->coef, d->coef_len);
    int rc = lss_check_cuda(c, cudaGetLastError(), "3D set_medium");
    if (!rc && d->rec) rc = lss3r_set_medium(c, s);
    return rc;
}

namespace {

template <typename C, int NB>
int factor_set_t(lss_ctx* c, const FactorSet3& fs, cudaStream_t s) {
    const int K = c->n_tot, nl = fs.count, Mmax = fs.Mmax;
    const Slab3* slabs = fs.d_slabs;
    const C* coef = (const C*)fs.coef;
    C* fac = (C*)fs.fac;
    C* W = (C*)fs.W;
    C* X = (C*)fs.X;
    C* T = (C*)fs.T;
    const long long MM = (long long)Mmax * Mmax;
    const int ew_blocks = (int)std::min<long long>(8LL * c->num_sms / std::max(1, nl) + 1, (MM + 255) / 256);
    const int tiles = (Mmax + 63) / 64;
    const int npanel = (Mmax + NB - 1) / NB;
    const size_t psm = (size_t)Mmax * NB * sizeof(C);
    bool use_tc = false;
    if constexpr (std::is_same<C, float2>::value) use_tc = fs.tc && lss3_use_tc();
    ProfScope ps(c, s, LSS_PROF_FACTOR, 0);
    for (int k = 0; k < K; ++k) {
        if (k == 0) {
            f3_init_A<C><<<dim3(ew_blocks, nl), 256, 0, s>>>(slabs, coef, W, 0);
            c->launches[LSS_PROF_FACTOR] += 1;
        } else {
            f3_schur_X<C><<<dim3(ew_blocks, nl), 256, 0, s>>>(slabs, coef, fac, X, k);
            f3_schur_D<C><<<dim3(ew_blocks, nl), 256, 0, s>>>(slabs, coef, X, W, k);
            c->launches[LSS_PROF_FACTOR] += 2;
        }
        f3_rowid_init<<<dim3(1, nl), 256, 0, s>>>(slabs, fs.rowid, Mmax);
        if (!use_tc) {
            for (int p = 0; p < npanel; ++p) {
                const int j0 = p * NB;
                f3_panel<C, NB><<<nl, 512, psm, s>>>(slabs, W, fs.piv, fs.rowid, j0, Mmax, c->d_err);
                f3_swap_extract<C, NB><<<dim3((Mmax + 255) / 256, nl), 256, 0, s>>>(slabs, W, fs.piv, T, j0, Mmax,
                                                                                   0, Mmax);
                f3_update_cc<C, NB><<<dim3(tiles * tiles, nl), 256, 0, s>>>(slabs, W, T, j0, Mmax, 0, Mmax);
            }
            c->launches[LSS_PROF_FACTOR] += 3LL * npanel;
        } else if constexpr (std::is_same<C, float2>::value) {
            // outer panels of kNO columns: four NB-wide Gauss-Jordan sub-panels,
            // each applying its row swaps to every column and its update to the
            // outer panel's columns only, then one rank-kNO update of all other
            // columns on the tensor cores
            const int nouter = (Mmax + kNO - 1) / kNO;
            const int otiles = (kNO + 63) / 64;
            for (int P = 0; P < nouter; ++P) {
                const int J0 = P * kNO;
                for (int q = 0; q < kNO / NB; ++q) {
                    const int j0 = J0 + q * NB;
                    if (j0 >= Mmax) break;
                    f3_panel<C, NB><<<nl, 512, psm, s>>>(slabs, W, fs.piv, fs.rowid, j0, Mmax, c->d_err);
                    f3_swap_extract<C, NB><<<dim3((Mmax + 255) / 256, nl), 256, 0, s>>>(slabs, W, fs.piv, T, j0,
                                                                                       Mmax, J0, J0 + kNO);
                    f3_update_cc<C, NB><<<dim3(tiles * otiles, nl), 256, 0, s>>>(slabs, W, T, j0, Mmax, J0,
                                                                               J0 + kNO);
                    c->launches[LSS_PROF_FACTOR] += 3;
                }
                f3_extract_outer<C><<<dim3((Mmax + 255) / 256, nl), 256, 0, s>>>(slabs, W, (C*)fs.T64, J0, kNO,
                                                                                Mmax);
                const int rc = lss3_update_tc(c, (float2*)W, (const float2*)fs.T64, J0, kNO, s);
                if (rc) return rc;
                c->launches[LSS_PROF_FACTOR] += 2;
            }
        }
        f3_finalize<C><<<dim3(ew_blocks, nl), 256, Mmax * sizeof(int), s>>>(slabs, W, fs.rowid, fac, k, Mmax);
        c->launches[LSS_PROF_FACTOR] += 2;
        const int rc = lss_check_cuda(c, cudaGetLastError(), "3D factorization launch");
        if (rc) return rc;
    }
    return LSS_OK;
}

// Step table of the whole sweep (only < 0) or of one slab solve (its forward
// solve alone, no couplings).  One front: forward solves of slabs 0..l-1
// (coupled to the left neighbour), backward corrections of l-2..0 (coupled to
// the right neighbour).  Two fronts: the forward solves of the left front
// (0..c-1) paired with those of the right front (l-1..c+1), the middle slab c
// with both couplings, then the backward corrections of both fronts paired
// (c-1..0 with c+1..l-1).
std::vector<Step3> step_table(int n_slabs, int K, int only, int fronts) {
    std::vector<Step3> v;
    auto solves = [&](int i0, int f0, int i1, int f1) {
        for (int k = 0; k < K; ++k) v.push_back({0, k, {i0, i1}, {f0, f1}});
        for (int k = K - 2; k >= 0; --k) v.push_back({1, k, {i0, i1}, {f0, f1}});
    };
    if (only >= 0) {
        solves(only, S3_FWD, -1, 0);
        return v;
    }
    if (fronts != 2) {
        for (int i = 0; i < n_slabs; ++i) solves(i, S3_FWD | (i > 0 ? S3_CL : 0), -1, 0);
        for (int i = n_slabs - 2; i >= 0; --i) solves(i, S3_CR, -1, 0);
        return v;
    }
    const int c = (n_slabs - 1) / 2;
    // pairs p of (left-front slab, right-front slab); either may be absent
    auto paired = [&](int nL, int nR, auto left, auto right) {
        for (int p = 0; p < std::max(nL, nR); ++p) {
            int iL = -1, fL = 0, iR = -1, fR = 0;
            if (p < nL) left(p, iL, fL);
            if (p < nR) right(p, iR, fR);
            if (iL < 0) { iL = iR; fL = fR; iR = -1; fR = 0; }
            solves(iL, fL, iR, fR);
        }
    };
    paired(c, n_slabs - 1 - c,
           [&](int p, int& i, int& f) { i = p; f = S3_FWD | (p > 0 ? S3_CL : 0); },
           [&](int p, int& i, int& f) { i = n_slabs - 1 - p; f = S3_FWD | (p > 0 ? S3_CR : 0); });
    solves(c, S3_FWD | (c > 0 ? S3_CL : 0) | (c < n_slabs - 1 ? S3_CR : 0), -1, 0);
    paired(c, n_slabs - 1 - c,
           [&](int p, int& i, int& f) { i = c - 1 - p; f = S3_CR; },
           [&](int p, int& i, int& f) { i = c + 1 + p; f = S3_CL; });
    return v;
}

// The sweep's grid right-hand sides for Rc vectors: f = Q r (r on I), or,
// for lss_apply_slab (fin), the slab's layers of fin's vectors r0.. given
// directly and zero elsewhere.
template <typename C>
void grid_in_t(lss_ctx* c, const double2* r, const double2* fin, int only, int r0, void* f, int Rc, cudaStream_t s) {
    Ctx3* d = c->d3;
    const long long G = (long long)c->n_tot * c->n_tot * c->n_tot;
    ProfScope ps(c, s, LSS_PROF_SPARSIFY, 1);
    if (!fin) {
        sparsify3_kernel<C><<<dim3(2 * c->num_sms, Rc), 256, 0, s>>>(r, (C*)f, stencil_args(d, c->omega), c->n, c->b,
                                                                    c->n_tot);
        return;
    }
    cudaMemsetAsync(f, 0, (size_t)Rc * G * sizeof(C), s);
    // v (nl layers x n_tot^2 per right-hand side) into the slab's layers of f
    const Slab3& sd = d->slabs[only];
    const long long per = (long long)sd.nl * c->n_tot * c->n_tot;
    const long long X1 = sd.s + c->b;
    for (int q = 0; q < Rc; ++q) {
        if (sizeof(C) == sizeof(double2)) {
            cudaMemcpyAsync((C*)f + q * G + X1 * c->n_tot * c->n_tot, fin + (r0 + q) * per, per * sizeof(double2),
                            cudaMemcpyDeviceToDevice, s);
        } else {
            cast3_kernel<<<2 * c->num_sms, 256, 0, s>>>(fin + (r0 + q) * per,
                                                       (float2*)f + q * G + X1 * c->n_tot * c->n_tot, per);
        }
    }
}

// The sweep's output for vectors r0..r0+Rc-1: ut restricted to I, or the
// slab's layers (lss_apply_slab).
template <typename C>
void grid_out_t(lss_ctx* c, const void* ut, double2* y, int only, bool fin, int r0, int Rc, cudaStream_t s) {
    Ctx3* d = c->d3;
    const long long G = (long long)c->n_tot * c->n_tot * c->n_tot;
    if (!fin) {
        ProfScope ps(c, s, LSS_PROF_SPARSIFY, 1);
        extract3_kernel<C><<<dim3(2 * c->num_sms, Rc), 256, 0, s>>>((const C*)ut, y + r0 * lss3_N(c), c->n, c->b,
                                                                    c->n_tot);
        return;
    }
    const Slab3& sd = d->slabs[only];
    const long long per = (long long)sd.nl * c->n_tot * c->n_tot;
    const long long X1 = sd.s + c->b;
    for (int q = 0; q < Rc; ++q) {
        if (sizeof(C) == sizeof(double2)) {
            cudaMemcpyAsync(y + (r0 + q) * per, (const C*)ut + q * G + X1 * c->n_tot * c->n_tot,
                            per * sizeof(double2), cudaMemcpyDeviceToDevice, s);
        } else {
            extract_f2_to_d2(y + (r0 + q) * per, (const float2*)ut + q * G + X1 * c->n_tot * c->n_tot, per,
                             c->num_sms, s);
        }
    }
}

template <typename C>
int sweep3_t(lss_ctx* c, const double2* r, double2* y, int R, int only, const double2* fin, cudaStream_t s) {
    Ctx3* d = c->d3;
    constexpr bool kSplit = std::is_same<C, double2>::value;
    const long long G = (long long)c->n_tot * c->n_tot * c->n_tot;
    const size_t cs = sizeof(C);
    const int RB = std::min(R, kSweepRB);
    int rc = lss_grow(c, &d->f, &d->f_cap, (size_t)RB * G * cs);
    if (!rc) rc = lss_grow(c, &d->ut, &d->ut_cap, (size_t)RB * G * cs);
    // per group of the grid (two when two fronts pair slab solves)
    if (!rc) rc = lss_grow(c, &d->Y, &d->Y_cap, 2 * (size_t)RB * c->n_tot * d->Mmax * cs);
    if (!rc && kSplit) rc = lss_grow(c, &d->TB, &d->TB_cap, 2 * (size_t)RB * d->Mmax * cs);
    if (rc) return rc;
    // step tables (device, cached: the whole sweep and the last single slab asked for)
    const std::vector<Step3> tab = step_table(c->n_slabs, c->n_tot, only, c->fronts);
    void** tab_dev = only < 0 ? &d->steps_all : &d->steps_one;
    size_t* tab_cap = only < 0 ? &d->steps_all_cap : &d->steps_one_cap;
    int* tab_key = only < 0 ? &d->steps_all_key : &d->steps_one_key;
    if (*tab_key != only || !*tab_dev) {
        rc = lss_grow(c, tab_dev, tab_cap, tab.size() * sizeof(Step3));
        if (!rc) rc = lss_check_cuda(c, cudaMemcpyAsync(*tab_dev, tab.data(), tab.size() * sizeof(Step3),
                                                        cudaMemcpyHostToDevice, s), "step table");
        if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "step table");
        if (rc) return rc;
        *tab_key = only;
    }
    const long long N = lss3_N(c);
    const int grid = c->num_sms;
    // shared memory: mbarrier (128 B), the D_k^{-1} row buffer, t (RB x Mmax), warp partials
    const size_t fixed = 128 + ((size_t)RB * d->Mmax + (size_t)(kSweepThreads / 32) * kSweepRB) * cs;
    size_t want = 0;
    for (const Slab3& sd : d->slabs) {
        const int gs = c->fronts == 2 ? grid / 2 : grid;   // CTAs per slab solve (paired steps: half the grid)
        const size_t rows = ((size_t)sd.M + gs - 1) / gs + 1;
        want = std::max(want, rows * sd.M * cs + 32);
    }
    const size_t budget = 210 * 1024;
    const size_t dcap = fixed >= budget ? 0 : (std::min(want, budget - fixed) & ~(size_t)15);
    const size_t smem = fixed + dcap;
    {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep3_kernel<C, kSplit>, kSweepThreads, smem);
        if (per < 1) return lss_fail(c, LSS_ERR_UNSUPPORTED, "3D sweep kernel does not fit on an SM");
    }
    for (int r0 = 0; r0 < R; r0 += RB) {
        const int Rc = std::min(RB, R - r0);
        grid_in_t<C>(c, r ? r + r0 * N : nullptr, fin, only, r0, d->f, Rc, s);
        cudaMemsetAsync(d->ut, 0, (size_t)Rc * G * cs, s);
        cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), s);   // arrival counter of the grid barriers
        Sweep3Args a{};
        a.slabs = d->d_slabs;
        a.steps = (const Step3*)*tab_dev;
        a.nsteps = (int)tab.size();
        a.n_tot = c->n_tot;
        a.b = c->b;
        a.Mmax = d->Mmax;
        a.coef = d->coef;
        a.fac = d->fac;
        a.f = d->f;
        a.ut = d->ut;
        a.Y = d->Y;
        a.TB = d->TB;
        a.R = Rc;
        a.G = G;
        a.dcap = (unsigned)dcap;
        a.bar = c->d_bar;
        a.err = c->d_err;
        void* args[] = {&a};
        {
            ProfScope ps(c, s, LSS_PROF_SLAB_A, 1);
            cudaError_t e = cudaLaunchCooperativeKernel((const void*)sweep3_kernel<C, kSplit>, dim3(grid),
                                                        dim3(kSweepThreads), args, smem, s);
            if (e) return lss_check_cuda(c, e, "3D sweep launch");
        }
        grid_out_t<C>(c, d->ut, y, only, fin != nullptr, r0, Rc, s);
    }
    return lss_check_cuda(c, cudaGetLastError(), "3D sweep");
}

}  // namespace

int lss3_factor_set(lss_ctx* c, const FactorSet3& fs, cudaStream_t s) {
    if (c->prec == LSS_FP64) return factor_set_t<double2, kNB64>(c, fs, s);
    return factor_set_t<float2, kNB32>(c, fs, s);
}

int lss3_dalloc(lss_ctx* c, void** p, size_t bytes, const char* what) { return dalloc3(c, p, bytes, what); }

void lss3_grid_in(lss_ctx* c, const double2* r, const double2* fin, int only, int r0, void* f, int Rc,
                  cudaStream_t s) {
    if (c->prec == LSS_FP64) grid_in_t<double2>(c, r, fin, only, r0, f, Rc, s);
    else grid_in_t<float2>(c, r, fin, only, r0, f, Rc, s);
}

void lss3_grid_out(lss_ctx* c, const void* ut, double2* y, int only, bool fin, int r0, int Rc, cudaStream_t s) {
    if (c->prec == LSS_FP64) grid_out_t<double2>(c, ut, y, only, fin, r0, Rc, s);
    else grid_out_t<float2>(c, ut, y, only, fin, r0, Rc, s);
}

int lss3_factor(lss_ctx* c, cudaStream_t s) {
    Ctx3* d = c->d3;
    if (d->rec) return lss3r_factor(c, s);
    FactorSet3 fs{d->d_slabs, c->n_slabs, d->Mmax, d->coef, d->fac, d->W, d->X, d->T, d->T64, d->piv, d->rowid, true};
    return lss3_factor_set(c, fs, s);
}

int lss3_sweep(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s) {
    if (c->d3->rec) return lss3r_sweep(c, r, y, R, -1, nullptr, s);
    if (c->prec == LSS_FP64) return sweep3_t<double2>(c, r, y, R, -1, nullptr, s);
    return sweep3_t<float2>(c, r, y, R, -1, nullptr, s);
}

int lss3_slab_apply(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s) {
    if (c->d3->rec) return lss3r_sweep(c, nullptr, w, R, slab, v, s);
    if (c->prec == LSS_FP64) return sweep3_t<double2>(c, nullptr, w, R, slab, v, s);
    return sweep3_t<float2>(c, nullptr, w, R, slab, v, s);
}

int lss3_matvec(lss_ctx* c, const double2* x, double2* y, int R, int in_mode, int out_mode, const double* dirs_dev,
                double2* uI, cudaStream_t s) {
    Ctx3* d = c->d3;
    const int n = c->n, L = c->L, lg = c->lgL;
    int rc = lss_grow(c, (void**)&d->mvA, &d->mvA_cap, (size_t)n * n * L * R * sizeof(double2));
    if (!rc) rc = lss_grow(c, (void**)&d->mvB, &d->mvB_cap, (size_t)n * L * L * R * sizeof(double2));
    if (rc) return rc;
    const int nt = line_threads3(L);
    const size_t sh = 2 * (size_t)L * sizeof(double2);
    const int C = col_group3(L);
    const size_t sh2 = 2 * (size_t)C * L * sizeof(double2);
    dim3 g1(n * n, R);
    ProfScope ps(c, s, LSS_PROF_MATVEC, 5);
    switch (in_mode) {
        case MV_IN_MU:
            mv3_rows_fwd<MV_IN_MU><<<g1, nt, sh, s>>>(x, c->m, nullptr, nullptr, d->mvA, c->tw, n, n * n, L, lg,
                                                    c->omega, c->h);
            break;
        case MV_IN_U:
            mv3_rows_fwd<MV_IN_U><<<g1, nt, sh, s>>>(x, c->m, nullptr, nullptr, d->mvA, c->tw, n, n * n, L, lg,
                                                   c->omega, c->h);
            break;
        case MV_IN_PLANEWAVE:
            mv3_rows_fwd<MV_IN_PLANEWAVE><<<g1, nt, sh, s>>>(x, c->m, dirs_dev, uI, d->mvA, c->tw, n, n * n, L, lg,
                                                           c->omega, c->h);
            break;
        default:
            return lss_fail(c, LSS_ERR_ARG, "matvec: bad input mode");
    }
    // x2: A[r][i1][i2][k3] (n rows) -> B[r][i1][k2][k3] (L rows)
    mv3_cols<COL_FWD><<<dim3(L / C, n, R), C * nt, sh2, s>>>(d->mvA, d->mvB, nullptr, c->tw, n, n, L, L, L, lg, C, 1.0);
    // x1: B[r][i1][(k2,k3)] in place, n rows kept
    mv3_cols<COL_CONV><<<dim3((unsigned)((long long)L * L / C), 1, R), C * nt, sh2, s>>>(
        d->mvB, d->mvB, d->khat, c->tw, 1, n, n, (long long)L * L, L, lg, C, 1.0);
    // x2 inverse: B[r][i1][k2][k3] (L rows) -> A[r][i1][i2][k3] (n rows)
    mv3_cols<COL_INV><<<dim3(L / C, n, R), C * nt, sh2, s>>>(d->mvB, d->mvA, nullptr, c->tw, n, L, n, L, L, lg, C, 1.0);
    switch (out_mode) {
        case MV_OUT_A:
            mv3_rows_inv<MV_OUT_A><<<g1, nt, sh, s>>>(d->mvA, x, c->m, y, c->tw, n, L, lg);
            break;
        case MV_OUT_AT:
            mv3_rows_inv<MV_OUT_AT><<<g1, nt, sh, s>>>(d->mvA, x, c->m, y, c->tw, n, L, lg);
            break;
        default:
            mv3_rows_inv<MV_OUT_NEG><<<g1, nt, sh, s>>>(d->mvA, x, c->m, y, c->tw, n, L, lg);
            break;
    }
    return lss_check_cuda(c, cudaGetLastError(), "3D matvec launch");
}

int lss3_get_stencils(const lss_ctx* c, double* alpha, double* beta) {
    const Ctx3* d = c->d3;
    for (int o = 0; o < 27; ++o) {
        alpha[2 * o] = d->alpha[o].real();
        alpha[2 * o + 1] = d->alpha[o].imag();
        beta[2 * o] = d->beta[o].real();
        beta[2 * o + 1] = d->beta[o].imag();
    }
    return LSS_OK;
}
