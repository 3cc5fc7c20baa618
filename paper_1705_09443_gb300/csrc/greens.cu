// Nystrom weights of the Green's function (Sec. 2.1), the FFT of the kernel for
// the LS operator, and the interior stencils alpha, beta (Sec. 2.2.1).
#include <cmath>
#include <complex>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"

using cd = std::complex<double>;

// ---------------------------------------------------------------- host quadrature
namespace {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

cd hankel1(int nu, double x) { return cd(std::cyl_bessel_j((double)nu, x), std::cyl_neumann((double)nu, x)); }

}  // namespace

// k_0 = integral of G over the cell [-h/2, h/2]^d (the diagonal weight; the
// paper's Duan-Rokhlin correction weights are not given, Sec. 2.1).
// 2D: in polar coordinates about the singular point, int_0^R H0(w r) r dr =
// R H1(w R)/w + 2i/(pi w^2); the angular integral over the square uses its
// 8 congruent sectors theta in [0, pi/4], R = (h/2)/cos(theta).
// 3D: int_0^R e^{i w r} r dr = e^{i w R}(R/(i w) + 1/w^2) - 1/w^2 over the 6
// faces, solid-angle element (h/2) dy dz / R^3.
cd lss_cell_integral_G(int d, double omega, double h) {
    const int nq = 48;
    std::vector<double> x, w;
    gauss_legendre(nq, x, w);
    if (d == 2) {
        cd acc = 0;
        for (int q = 0; q < nq; ++q) {
            const double th = 0.5 * (M_PI / 4) * (x[q] + 1.0);
            const double R = 0.5 * h / std::cos(th);
            acc += 0.5 * (M_PI / 4) * w[q] * R * hankel1(1, omega * R);
        }
        return cd(0, 1) / (4.0 * omega) * (8.0 * acc) - 1.0 / (omega * omega);
    }
    const double a = 0.5 * h;
    cd face = 0;
    for (int p = 0; p < nq; ++p)
        for (int q = 0; q < nq; ++q) {
            const double y = a * x[p], z = a * x[q];
            const double R = std::sqrt(a * a + y * y + z * z);
            const cd F = std::exp(cd(0, omega * R)) * (R / cd(0, omega) + 1.0 / (omega * omega)) -
                         1.0 / (omega * omega);
            face += a * w[p] * a * w[q] * F * a / (R * R * R);
        }
    return 6.0 * face / (4.0 * M_PI);
}

namespace {

// (J0(x), Y0(x)) for x > 0 to about 1e-16 absolute, over the whole range of
// arguments a table reaches (omega r up to several hundred), from two
// published methods:
//  x < 25: Miller's backward recurrence J_{k-1} = (2k/x) J_k - J_{k+1} from an
//   even order N >= x + 40 (where J_N is negligible), normalised by
//   J0 + 2 sum_{k>=1} J_{2k} = 1; Y0 from Neumann's series
//   Y0 = (2/pi)(ln(x/2) + gamma) J0 - (4/pi) sum_{k>=1} (-1)^k J_{2k} / k;
//  x >= 25: Hankel's asymptotic expansion
//   H0(x) = J0 + i Y0 = sqrt(2/(pi x)) e^{i(x - pi/4)} sum_k a_k (i/x)^k,
//   a_0 = 1, a_k = -a_{k-1} (2k-1)^2 / (8k), summed until a term is below
//   1e-17 (about 20 terms at x = 25; the least term, near k = 2x, is far
//   below that).
__device__ double2 bessel_j0_y0(double x) {
    if (x < 25.0) {
        const int N = 2 * (int)((x + 40.0) * 0.5) + 2;
        double jp = 0.0, jc = 1e-30, norm = 0.0, ys = 0.0;
        for (int k = N; k > 0; --k) {
            const double jm = (2.0 * k / x) * jc - jp;   // J_{k-1}
            jp = jc;
            jc = jm;
            const int km = k - 1;
            if (km > 0 && (km & 1) == 0) {
                const int h = km >> 1;
                norm += 2.0 * jc;
                ys += ((h & 1) ? -jc : jc) / h;
            }
            if (fabs(jc) > 1e200) {   // rescale against overflow at small x
                jp *= 1e-200;
                jc *= 1e-200;
                norm *= 1e-200;
                ys *= 1e-200;
            }
        }
        norm += jc;
        const double J0 = jc / norm;
        const double euler_gamma = 0.57721566490153286061;
        const double Y0 = (2.0 / M_PI) * (log(0.5 * x) + euler_gamma) * J0 - (4.0 / M_PI) * (ys / norm);
        return mk(J0, Y0);
    }
    double tr = 1.0, ti = 0.0, sr = 1.0, si = 0.0;   // term and sum of the series
    for (int k = 1; k < 64; ++k) {
        const double f = -(double)((2 * k - 1) * (2 * k - 1)) / (8.0 * k * x);
        const double nr = -ti * f, ni = tr * f;   // term *= f * i
        tr = nr;
        ti = ni;
        sr += tr;
        si += ti;
        if (fabs(tr) + fabs(ti) < 1e-17) break;
    }
    double sn, cs;
    sincos(x, &sn, &cs);
    const double a = sqrt(2.0 / (M_PI * x)) * M_SQRT1_2;   // e^{-i pi/4} = (1 - i)/sqrt(2)
    const double er = a * (cs + sn), ei = a * (sn - cs);
    return mk(er * sr - ei * si, er * si + ei * sr);
}

// G(r) h^2 = h^2 (i/4) (J0 + i Y0)(omega r) for r > 0 (2D).
__device__ __forceinline__ double2 k_weight_2d(double r, double omega, double h2) {
    const double2 jy = bessel_j0_y0(omega * r);
    return mk(-0.25 * jy.y * h2, 0.25 * jy.x * h2);
}

// Circular L x L table for the zero-padded convolution: offsets |o_a| <= n-1
// at index o_a mod L, zero elsewhere.
__global__ void k_table_circ(double2* kc, int n, int L, double omega, double h, double2 k0) {
    const long long tot = (long long)L * L;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int j1 = (int)(e / L), j2 = (int)(e % L);
        const int o1 = j1 < L / 2 ? j1 : j1 - L;
        const int o2 = j2 < L / 2 ? j2 : j2 - L;
        double2 v = mk(0.0, 0.0);
        if (abs(o1) <= n - 1 && abs(o2) <= n - 1) {
            if (o1 == 0 && o2 == 0) v = k0;
            else v = k_weight_2d(h * sqrt((double)o1 * o1 + (double)o2 * o2), omega, h * h);
        }
        kc[e] = v;
    }
}

// Offsets {-(n+1)..n+1}^2, index (o1+n+1)*(2n+3) + o2+n+1.
__global__ void k_table_ext(double2* kx, int n, double omega, double h, double2 k0) {
    const int S = 2 * n + 3;
    const long long tot = (long long)S * S;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int o1 = (int)(e / S) - (n + 1), o2 = (int)(e % S) - (n + 1);
        kx[e] = (o1 == 0 && o2 == 0) ? k0
                                     : k_weight_2d(h * sqrt((double)o1 * o1 + (double)o2 * o2), omega, h * h);
    }
}

// Gram matrix of K_{mu,mu^c} (Eq. alpha): G_ab = sum_{j in mu^c} k_{o_a-j} conj(k_{o_b-j}),
// mu^c = {-n..n}^2 minus mu; one block row of partial sums per (block, pair).
__global__ void gram_partial(const double2* __restrict__ kx, int n, double2* __restrict__ part) {
    __shared__ double2 red[256];
    const int pair = blockIdx.y;  // 0..44 over a <= b
    int a = 0, b = pair;
    while (b >= 9 - a) { b -= 9 - a; ++a; }
    b += a;
    const int a1 = a / 3 - 1, a2 = a % 3 - 1, b1 = b / 3 - 1, b2 = b % 3 - 1;
    const int S = 2 * n + 3, M = 2 * n + 1;
    const long long tot = (long long)M * M;
    double2 acc = mk(0.0, 0.0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int j1 = (int)(e / M) - n, j2 = (int)(e % M) - n;
        if (abs(j1) <= 1 && abs(j2) <= 1) continue;
        const double2 ka = kx[(long long)(a1 - j1 + n + 1) * S + (a2 - j2 + n + 1)];
        const double2 kb = kx[(long long)(b1 - j1 + n + 1) * S + (b2 - j2 + n + 1)];
        acc = cfma(ka, conjc(kb), acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)pair * gridDim.x + blockIdx.x] = red[0];
}

}  // namespace

// Cyclic Jacobi eigen-decomposition of a real symmetric matrix (n x n,
// row-major); returns eigenvalues in d and eigenvectors as columns of V.
void lss_jacobi_eigen(std::vector<double> A, int n, std::vector<double>& d, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-34 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {  // A <- A J  (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = cs * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A  (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = cs * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    d.resize(n);
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
}

// k table, twiddles, FFT of the kernel.
int lss_build_kernel(lss_ctx* c, cudaStream_t s) {
    const int L = c->L;
    std::vector<double2> tw(L);
    for (int k = 0; k < L; ++k) {
        const long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)L;
        tw[k] = make_double2((double)cosl(a), (double)sinl(a));
    }
    int rc = lss_check_cuda(c, cudaMemcpyAsync(c->tw, tw.data(), L * sizeof(double2), cudaMemcpyHostToDevice, s),
                            "twiddles");
    if (rc) return rc;
    const cd k0 = lss_cell_integral_G(2, c->omega, c->h);
    double2* kc = nullptr;
    rc = lss_check_cuda(c, cudaMallocAsync((void**)&kc, (size_t)L * L * sizeof(double2), s), "k table");
    if (rc) return lss_fail(c, LSS_ERR_OOM, "k table allocation");
    {
        ProfScope ps(c, s, LSS_PROF_SETUP, 1);
        k_table_circ<<<4 * c->num_sms, 256, 0, s>>>(kc, c->n, L, c->omega, c->h, make_double2(k0.real(), k0.imag()));
    }
    rc = lss_fft_kernel_table(c, kc, s);
    cudaFreeAsync(kc, s);
    if (rc) return rc;
    return lss_check_cuda(c, cudaGetLastError(), "k table");
}

// alpha = unit left singular vector of K_{mu,mu^c} for the smallest singular
// value (Eq. alpha), i.e. the eigenvector of the Gram matrix K K^* for its
// smallest eigenvalue; beta^* = alpha^* K_{mu,mu} (Eq. beta).  The Hermitian
// 9x9 eigenproblem is solved through its real 18x18 symmetric embedding.
int lss_build_interior_stencils(lss_ctx* c, cudaStream_t s) {
    const int n = c->n, S = 2 * n + 3;
    const cd k0 = lss_cell_integral_G(2, c->omega, c->h);
    double2* kx = nullptr;
    double2* part = nullptr;
    const int nblk = 2 * c->num_sms;
    int rc = lss_check_cuda(c, cudaMallocAsync((void**)&kx, (size_t)S * S * sizeof(double2), s), "k ext");
    if (rc) return lss_fail(c, LSS_ERR_OOM, "k ext allocation");
    rc = lss_check_cuda(c, cudaMallocAsync((void**)&part, (size_t)45 * nblk * sizeof(double2), s), "gram");
    if (rc) { cudaFreeAsync(kx, s); return lss_fail(c, LSS_ERR_OOM, "gram allocation"); }
    {
        ProfScope ps(c, s, LSS_PROF_SETUP, 2);
        k_table_ext<<<4 * c->num_sms, 256, 0, s>>>(kx, n, c->omega, c->h, make_double2(k0.real(), k0.imag()));
        gram_partial<<<dim3(nblk, 45), 256, 0, s>>>(kx, n, part);
    }
    std::vector<double2> hp((size_t)45 * nblk), kc5(25);
    cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, s);
    for (int r = 0; r < 5; ++r)
        cudaMemcpyAsync(&kc5[r * 5], kx + (size_t)(n - 1 + r) * S + (n - 1), 5 * sizeof(double2),
                        cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFreeAsync(kx, s);
    cudaFreeAsync(part, s);
    if (e) return lss_check_cuda(c, e, "gram");

    cd Gm[9][9];
    int pair = 0;
    for (int a = 0; a < 9; ++a)
        for (int b = a; b < 9; ++b, ++pair) {
            cd acc = 0;
            for (int k = 0; k < nblk; ++k) acc += cd(hp[(size_t)pair * nblk + k].x, hp[(size_t)pair * nblk + k].y);
            Gm[a][b] = acc;
            Gm[b][a] = std::conj(acc);
        }
    // real embedding [[Re, -Im], [Im, Re]]
    std::vector<double> A(18 * 18);
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            A[a * 18 + b] = Gm[a][b].real();
            A[a * 18 + 9 + b] = -Gm[a][b].imag();
            A[(9 + a) * 18 + b] = Gm[a][b].imag();
            A[(9 + a) * 18 + 9 + b] = Gm[a][b].real();
        }
    std::vector<double> d, V;
    lss_jacobi_eigen(A, 18, d, V);
    int imin = 0;
    for (int i = 1; i < 18; ++i)
        if (d[i] < d[imin]) imin = i;
    cd al[9];
    double nrm = 0;
    for (int a = 0; a < 9; ++a) {
        al[a] = cd(V[a * 18 + imin], V[(9 + a) * 18 + imin]);
        nrm += std::norm(al[a]);
    }
    nrm = std::sqrt(nrm);
    const cd ph = std::abs(al[4]) / al[4];
    for (int a = 0; a < 9; ++a) al[a] = al[a] * ph / nrm;
    al[4] = cd(std::abs(al[4]), 0.0);
    // K_{mu,mu}: entry (a, b) = k_{o_a - o_b}; kc5 holds offsets -2..2.
    for (int b = 0; b < 9; ++b) {
        cd acc = 0;
        for (int a = 0; a < 9; ++a) {
            const int d1 = (a / 3) - (b / 3), d2 = (a % 3) - (b % 3);
            const double2 kab = kc5[(d1 + 2) * 5 + (d2 + 2)];
            acc += al[a] * std::conj(cd(kab.x, kab.y));  // beta_b = sum_a alpha_a conj(K_ab)
        }
        c->beta[b] = acc;
    }
    for (int a = 0; a < 9; ++a) c->alpha[a] = al[a];
    return LSS_OK;
}
