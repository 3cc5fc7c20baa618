// Flexible restarted GMRES (Sec. 2.5 uses standard restarted GMRES; flexible
// GMRES equals it for a fixed linear preconditioner and stays valid when the
// preconditioner is applied in reduced precision).  Right preconditioning,
// x0 = 0, classical Gram-Schmidt with one re-orthogonalisation (CGS2), Givens
// rotations on the host, all vector work in FP64 kernels, R right-hand sides
// advanced together with independent Hessenberg matrices.  The kernels of one
// iteration (preconditioner, operator, both Gram-Schmidt passes) are replayed
// from a CUDA graph per basis index once the workspaces exist.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

using cd = std::complex<double>;

namespace {

constexpr int kRedThreads = 256;

// part[(i*R + r)*nblk + blk] = sum over this block's x of conj(V_i[r][x]) w[r][x]
__global__ void __launch_bounds__(kRedThreads) dots_kernel(const double2* __restrict__ V, long long vstride,
                                                           const double2* __restrict__ w, long long N, int R,
                                                           double2* __restrict__ part) {
    __shared__ double2 red[kRedThreads];
    const int r = blockIdx.y, i = blockIdx.z, nblk = gridDim.x;
    const double2* vi = V + (long long)i * vstride + (long long)r * N;
    const double2* wr = w + (long long)r * N;
    double2 acc = mk(0.0, 0.0);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)nblk * blockDim.x)
        acc = cfma_conj(vi[x], wr[x], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[((long long)i * R + r) * nblk + blockIdx.x] = red[0];
}

// h[e] (+)= sum_blk part[e * nblk + blk], e = i*R + r: one CTA per e, strided
// partial sums then a fixed tree (deterministic: the same order every call)
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const double2* __restrict__ part, int nblk,
                                                             double2* __restrict__ h, int accumulate) {
    __shared__ double2 red[kRedThreads];
    const int e = blockIdx.x;
    double2 acc = mk(0.0, 0.0);
    for (int b = threadIdx.x; b < nblk; b += kRedThreads) acc = acc + part[(long long)e * nblk + b];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[e] = accumulate ? h[e] + red[0] : red[0];
}

// w[r][x] += sign * sum_{i<J} h[i*R + r] V_i[r][x]
__global__ void update_kernel(const double2* __restrict__ V, long long vstride, const double2* __restrict__ h,
                              int J, double2* __restrict__ w, long long N, int R, double sign) {
    const int r = blockIdx.y;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        double2 acc = mk(0.0, 0.0);
        for (int i = 0; i < J; ++i) acc = cfma(h[i * R + r], V[(long long)i * vstride + (long long)r * N + x], acc);
        double2 wv = w[(long long)r * N + x];
        w[(long long)r * N + x] = mk(wv.x + sign * acc.x, wv.y + sign * acc.y);
    }
}

// y[r] = x[r] * scale[r]  (scale = 0 leaves zeros)
__global__ void scale_kernel(const double2* __restrict__ x, double2* __restrict__ y, const double* __restrict__ sc,
                             long long N) {
    const int r = blockIdx.y;
    const double s = sc[r];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
        y[(long long)r * N + e] = s * x[(long long)r * N + e];
}

// y = a - b
__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ y,
                           long long tot) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
        y[e] = a[e] - b[e];
}

struct Krylov {
    lss_ctx* c;
    cudaStream_t s;
    long long N;
    int R, nblk;
    double2* part;   // partial sums
    double2* hdev;   // (m+1) x R: first Gram-Schmidt pass, later the solution coefficients
    double2* h2dev;  // (m+1) x R: second pass
    double2* hnorm;  // R: ||w||^2
    double* scdev;   // R scales
    int grid1d;
};

// h[0..J) for every r = V_i^H w  (accumulate: h += ...)
void dots(Krylov& K, const double2* V, long long vstride, int J, const double2* w, double2* h, int accumulate) {
    ProfScope ps(K.c, K.s, LSS_PROF_KRYLOV, 2);
    dots_kernel<<<dim3(K.nblk, K.R, J), kRedThreads, 0, K.s>>>(V, vstride, w, K.N, K.R, K.part);
    const int JR = J * K.R;
    reduce_kernel<<<JR, kRedThreads, 0, K.s>>>(K.part, K.nblk, h, accumulate);
}

}  // namespace

int lss_fgmres(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
               cudaStream_t s, int transpose) {
    // transpose: solve A^T x = g (A^T = I + omega^2 M K) preconditioned by P^T
    const int mv_in = transpose ? MV_IN_U : MV_IN_MU, mv_out = transpose ? MV_OUT_AT : MV_OUT_A;
    const long long N = c->npts();
    const int m = o->restart;
    const double tol = o->tol;
    const int maxit = o->max_iter;
    const long long RN = (long long)R * N;
    // storage: V (m+1), Z (m), w, r
    const size_t nvec = (size_t)(m + 1) + m + 2;
    int rc = lss_grow(c, (void**)&c->kr_buf, &c->kr_cap, nvec * RN * sizeof(double2));
    if (rc) return rc;
    double2* V = c->kr_buf;
    double2* Z = V + (size_t)(m + 1) * RN;
    double2* w = Z + (size_t)m * RN;
    double2* rv = w + RN;
    Krylov K{c, s, N, R, 0, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    // grids sized for the whole batch: about two CTAs per SM over all right-hand sides
    K.nblk = std::max(1, std::min(2 * c->num_sms / R, (int)((N + kRedThreads - 1) / kRedThreads)));
    const size_t red_bytes = (size_t)(m + 1) * R * K.nblk * sizeof(double2) +
                             (size_t)(2 * (m + 1) + 1) * R * sizeof(double2) + (size_t)R * sizeof(double) + 64;
    rc = lss_grow(c, (void**)&c->red_buf, &c->red_cap, red_bytes);
    if (rc) return rc;
    K.part = c->red_buf;
    K.hdev = K.part + (size_t)(m + 1) * R * K.nblk;
    K.h2dev = K.hdev + (size_t)(m + 1) * R;
    K.hnorm = K.h2dev + (size_t)(m + 1) * R;
    K.scdev = reinterpret_cast<double*>(K.hnorm + R);
    const int g1 = std::max(1, std::min(4 * c->num_sms / R, (int)((N + 255) / 256)));
    const int gs = std::max(1, std::min(4 * c->num_sms, (int)((RN + 255) / 256)));

    double2* hnorm = K.hnorm;
    if (transpose && (rc = lss_prepare_sweep_t(c, s))) return rc;

    // Iteration body for basis vector j on stream bs: Z_j = P V_j, w = A Z_j,
    // two Gram-Schmidt passes against V_0..V_j, ||w||^2.
    auto body = [&](int j, cudaStream_t bs) -> int {
        Krylov Kb = K;
        Kb.s = bs;
        const double2* Vj = V + (size_t)j * RN;
        double2* Zj = Z + (size_t)j * RN;
        int r = transpose ? lss_sweep_t(c, Vj, Zj, R, bs) : lss_sweep(c, Vj, Zj, R, bs);
        if (!r) r = lss_matvec(c, Zj, w, R, mv_in, mv_out, nullptr, nullptr, bs);
        if (r) return r;
        dots(Kb, V, RN, j + 1, w, K.hdev, 0);
        { ProfScope ps_(c, bs, LSS_PROF_KRYLOV, 1); update_kernel<<<dim3(g1, R), 256, 0, bs>>>(V, RN, K.hdev, j + 1, w, N, R, -1.0); }
        dots(Kb, V, RN, j + 1, w, K.h2dev, 0);
        { ProfScope ps_(c, bs, LSS_PROF_KRYLOV, 1); update_kernel<<<dim3(g1, R), 256, 0, bs>>>(V, RN, K.h2dev, j + 1, w, N, R, -1.0); }
        dots(Kb, w, 0, 1, w, hnorm, 0);
        return lss_check_cuda(c, cudaGetLastError(), "arnoldi");
    };
    // Graphs: only once a solve with this R and transpose ran uncaptured at the
    // current workspace generation (every buffer the body touches exists), and
    // not while profiling (the profile records events around kernel groups).
    // (the 3D sweep is a cooperative grid-synchronised launch: run uncaptured)
    const bool use_graph = c->graphs_on && !c->prof_on && c->dim == 2;
    bool warm = false;
    for (const auto& k : c->graph_warm)
        warm |= k[0] == R && k[1] == transpose && (unsigned long long)k[2] == c->buf_gen;
    warm &= use_graph;
    auto graph_for = [&](int j) -> cudaGraphExec_t {
        for (const auto& g : c->graphs)
            if (g.j == j && g.R == R && g.transpose == transpose && g.gen == c->buf_gen) return g.exec;
        std::vector<lss_ctx::GraphRec> keep;   // drop graphs of older workspaces
        for (const auto& g : c->graphs) {
            if (g.gen == c->buf_gen) keep.push_back(g);
            else if (g.exec) cudaGraphExecDestroy(g.exec);
        }
        c->graphs.swap(keep);
        const unsigned long long gen0 = c->buf_gen;
        const std::string err0 = c->err;
        cudaGraphExec_t ex = nullptr;
        if (c->cap_stream || !cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) {
            cudaGraph_t gr = nullptr;
            if (!cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal)) {
                const int brc = body(j, c->cap_stream);
                cudaError_t e = cudaStreamEndCapture(c->cap_stream, &gr);
                if (!brc && !e && gr && c->buf_gen == gen0 && cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess)
                    ex = nullptr;
                if (brc || e || c->buf_gen != gen0) {
                    if (ex) cudaGraphExecDestroy(ex);
                    ex = nullptr;
                }
                if (gr) cudaGraphDestroy(gr);
            }
        }
        cudaGetLastError();   // a refused capture leaves no error behind
        c->err = err0;
        // a body that cannot be captured (e.g. the grid-synchronised recurrence)
        // is remembered as such and runs uncaptured
        c->graphs.push_back({j, R, transpose, gen0, ex});
        return ex;
    };
    auto iteration = [&](int j) -> int {
        if (warm) {
            cudaGraphExec_t ex = graph_for(j);
            if (ex) return lss_check_cuda(c, cudaGraphLaunch(ex, s), "iteration graph");
        }
        return body(j, s);
    };

    std::vector<double2> hh((size_t)(m + 2) * R);
    std::vector<double> sc(R);
    auto fetch = [&](const double2* src, size_t count) -> int {
        cudaError_t e = cudaMemcpyAsync(hh.data(), src, count * sizeof(double2), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        return lss_check_cuda(c, e, "krylov fetch");
    };
    auto set_scale = [&]() -> int {
        return lss_check_cuda(c, cudaMemcpyAsync(K.scdev, sc.data(), R * sizeof(double), cudaMemcpyHostToDevice, s),
                              "krylov scale");
    };

    // ||g||
    dots(K, g, 0, 1, g, K.hdev, 0);
    if ((rc = fetch(K.hdev, R))) return rc;
    std::vector<double> gnorm(R), beta(R);
    for (int r = 0; r < R; ++r) gnorm[r] = beta[r] = std::sqrt(std::max(0.0, hh[r].x));
    cudaMemsetAsync(u, 0, RN * sizeof(double2), s);
    cudaMemcpyAsync(rv, g, RN * sizeof(double2), cudaMemcpyDeviceToDevice, s);

    std::vector<int> iters(R, 0), done(R, 0);
    std::vector<double> est(R, 0.0);
    for (int r = 0; r < R; ++r)
        if (gnorm[r] == 0.0) done[r] = 1;
    int total = 0;
    std::vector<cd> H((size_t)(m + 1) * m * R), cs((size_t)m * R), sn((size_t)m * R), rho((size_t)(m + 1) * R);
    auto Hix = [&](int i, int j, int r) -> cd& { return H[((size_t)r * (m + 1) + i) * m + j]; };

    while (true) {
        bool all_done = true;
        for (int r = 0; r < R; ++r) all_done &= (bool)done[r];
        if (all_done || total >= maxit) break;
        std::vector<int> active(R), kr(R, 0);
        for (int r = 0; r < R; ++r) {
            active[r] = !done[r];
            sc[r] = active[r] ? 1.0 / beta[r] : 0.0;
            rho[(size_t)r * (m + 1)] = beta[r];
            for (int i = 1; i <= m; ++i) rho[(size_t)r * (m + 1) + i] = 0.0;
        }
        if ((rc = set_scale())) return rc;
        { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); scale_kernel<<<dim3(g1, R), 256, 0, s>>>(rv, V, K.scdev, N); }
        int j = 0;
        for (; j < m && total < maxit; ++j) {
            if ((rc = iteration(j))) return rc;
            // fetch h (first pass), h2 (second pass) and ||w||^2
            const size_t cnt = (size_t)(j + 1) * R;
            std::vector<double2> h1(cnt), h2v(cnt), hn(R);
            cudaError_t e = cudaMemcpyAsync(h1.data(), K.hdev, cnt * sizeof(double2), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaMemcpyAsync(h2v.data(), K.h2dev, cnt * sizeof(double2), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaMemcpyAsync(hn.data(), hnorm, R * sizeof(double2), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            if ((rc = lss_check_cuda(c, e, "arnoldi fetch"))) return rc;
            ++total;
            for (int r = 0; r < R; ++r) {
                if (!active[r]) { sc[r] = 0.0; continue; }
                for (int i = 0; i <= j; ++i)
                    Hix(i, j, r) = cd(h1[(size_t)i * R + r].x + h2v[(size_t)i * R + r].x,
                                      h1[(size_t)i * R + r].y + h2v[(size_t)i * R + r].y);
                const double hnr = std::sqrt(std::max(0.0, hn[r].x));
                Hix(j + 1, j, r) = hnr;
                sc[r] = hnr > 0 ? 1.0 / hnr : 0.0;
                for (int i = 0; i < j; ++i) {
                    const cd a = Hix(i, j, r), b = Hix(i + 1, j, r);
                    const cd cc = cs[(size_t)r * m + i], ss = sn[(size_t)r * m + i];
                    Hix(i, j, r) = cc * a + ss * b;
                    Hix(i + 1, j, r) = -std::conj(ss) * a + std::conj(cc) * b;
                }
                const cd a = Hix(j, j, r), b = Hix(j + 1, j, r);
                const double den = std::sqrt(std::norm(a) + std::norm(b));
                const cd cc = den > 0 ? std::conj(a) / den : cd(1.0);
                const cd ss = den > 0 ? std::conj(b) / den : cd(0.0);
                cs[(size_t)r * m + j] = cc;
                sn[(size_t)r * m + j] = ss;
                Hix(j, j, r) = cc * a + ss * b;
                Hix(j + 1, j, r) = 0.0;
                cd& rj = rho[(size_t)r * (m + 1) + j];
                rho[(size_t)r * (m + 1) + j + 1] = -std::conj(ss) * rj;
                rj = cc * rj;
                iters[r] += 1;
                kr[r] = j + 1;
                est[r] = std::abs(rho[(size_t)r * (m + 1) + j + 1]) / gnorm[r];
                if (est[r] <= tol || hnr == 0.0) {
                    done[r] = 1;
                    active[r] = 0;
                }
            }
            if ((rc = set_scale())) return rc;
            { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); scale_kernel<<<dim3(g1, R), 256, 0, s>>>(w, V + (size_t)(j + 1) * RN, K.scdev, N); }
            bool any = false;
            for (int r = 0; r < R; ++r) any |= (bool)active[r];
            if (!any) { ++j; break; }
        }
        // x += Z y with y from the triangular system of each RHS
        const int J = *std::max_element(kr.begin(), kr.end());
        if (J > 0) {
            std::vector<double2> yh((size_t)J * R, make_double2(0, 0));
            for (int r = 0; r < R; ++r) {
                const int k = kr[r];
                std::vector<cd> y(k);
                for (int i = k - 1; i >= 0; --i) {
                    cd acc = rho[(size_t)r * (m + 1) + i];
                    for (int l = i + 1; l < k; ++l) acc -= Hix(i, l, r) * y[l];
                    y[i] = acc / Hix(i, i, r);
                }
                for (int i = 0; i < k; ++i) yh[(size_t)i * R + r] = make_double2(y[i].real(), y[i].imag());
            }
            cudaMemcpyAsync(K.hdev, yh.data(), yh.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
            { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); update_kernel<<<dim3(g1, R), 256, 0, s>>>(Z, RN, K.hdev, J, u, N, R, +1.0); }
        }
        all_done = true;
        for (int r = 0; r < R; ++r) all_done &= (bool)done[r];
        if (all_done || total >= maxit) break;
        // restart: r = g - A u
        if ((rc = lss_matvec(c, u, w, R, mv_in, mv_out, nullptr, nullptr, s))) return rc;
        { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); sub_kernel<<<gs, 256, 0, s>>>(g, w, rv, RN); }
        dots(K, rv, 0, 1, rv, K.hdev, 0);
        if ((rc = fetch(K.hdev, R))) return rc;
        for (int r = 0; r < R; ++r) beta[r] = std::sqrt(std::max(0.0, hh[r].x));
    }
    // true residual
    if ((rc = lss_matvec(c, u, w, R, mv_in, mv_out, nullptr, nullptr, s))) return rc;
    { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); sub_kernel<<<gs, 256, 0, s>>>(g, w, rv, RN); }
    dots(K, rv, 0, 1, rv, K.hdev, 0);
    if ((rc = fetch(K.hdev, R))) return rc;
    bool conv = true;
    for (int r = 0; r < R; ++r) {
        const double rt = gnorm[r] > 0 ? std::sqrt(std::max(0.0, hh[r].x)) / gnorm[r] : 0.0;
        const bool cv = gnorm[r] == 0.0 || est[r] <= tol;
        conv &= cv;
        if (st) {
            st[r].iters = iters[r];
            st[r].converged = cv ? 1 : 0;
            st[r].relres_est = est[r];
            st[r].relres_true = rt;
        }
    }
    if ((rc = lss_check_device_err(c, s))) return rc;
    if (use_graph && !warm) {   // later solves with this R and transpose replay captured iterations
        std::vector<std::array<long long, 3>> keep;
        for (const auto& k : c->graph_warm)
            if ((unsigned long long)k[2] == c->buf_gen && !(k[0] == R && k[1] == transpose)) keep.push_back(k);
        keep.push_back({(long long)R, (long long)transpose, (long long)c->buf_gen});
        c->graph_warm.swap(keep);
    }
    return conv ? LSS_OK : lss_fail(c, LSS_ERR_NOCONVERGE, "GMRES reached max_iter before tol");
}
