// Flexible restarted GMRES (Sec. 2.5 uses standard restarted GMRES; flexible
// GMRES equals it for a fixed linear preconditioner and stays valid when the
// preconditioner is applied in reduced precision).  Right preconditioning,
// x0 = 0, classical Gram-Schmidt with one re-orthogonalisation (CGS2), R
// right-hand sides advanced together with independent Hessenberg matrices.
// Everything runs in FP64 kernels on the device: the vector work, the
// Hessenberg columns, the Givens rotations, the residual estimates and the
// per-RHS convergence masks, and the triangular solve for the update.  The
// host reads the device state once per restart cycle.  Each iteration
// (preconditioner, operator, both Gram-Schmidt passes, Givens update,
// normalisation) is replayed from a CUDA graph per basis index, guarded by a
// conditional node that skips it once every right-hand side has converged,
// so a whole cycle is enqueued without waiting for the device.
#include <algorithm>
#include <array>
#include <cmath>
#include <functional>
#include <complex>
#include <string>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

using cd = std::complex<double>;

namespace {

constexpr int kRedThreads = 256;

// Right-hand side r of a vector: entries [offs[r], offs[r+1]) when the
// right-hand sides have different lengths (the instances of a ragged batch
// side by side), else [r N, (r+1) N).
__device__ __forceinline__ void seg_of(const long long* offs, long long N, int r, long long& o, long long& len) {
    if (offs) { o = offs[r]; len = offs[r + 1] - o; }
    else { o = (long long)r * N; len = N; }
}

// part[(i*R + r)*nblk + blk] = sum over this block's x of conj(V_i[r][x]) w[r][x],
// for Q basis vectors i0 .. i0+Q-1 per CTA, reading w once for all of them;
// the block's sum in a fixed order (warp shuffles, then the warps in turn).
// Q is a compile-time count so that no predicated-off FP64 work is issued.
template <int Q>
__device__ __forceinline__ void dots_body(const double2* __restrict__ vb, long long vstride,
                                          const double2* __restrict__ wr, long long N, int R, int i0, int r,
                                          double2* __restrict__ part, double2 (*red)[kRedThreads / 32]) {
    // (vb, wr: this right-hand side's entries; N: their count)
    const int nblk = gridDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double2 acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = mk(0.0, 0.0);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)nblk * blockDim.x) {
        const double2 wv = wr[x];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] = cfma_conj(vb[(long long)q * vstride + x], wv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        for (int off = 16; off > 0; off >>= 1) {
            acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, off);
            acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, off);
        }
        if (lane == 0) red[q][wid] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < Q) {
        double2 t = mk(0.0, 0.0);
        for (int k = 0; k < kRedThreads / 32; ++k) t = t + red[threadIdx.x][k];
        part[((long long)(i0 + threadIdx.x) * R + r) * nblk + blockIdx.x] = t;
    }
}

constexpr int kDotsQ = 4;   // basis vectors per CTA of the Gram-Schmidt inner products

__global__ void __launch_bounds__(kRedThreads) dots_multi_kernel(const double2* __restrict__ V, long long vstride,
                                                                 const double2* __restrict__ w, long long N, int R,
                                                                 int J, double2* __restrict__ part,
                                                                 const long long* __restrict__ offs) {
    __shared__ double2 red[kDotsQ][kRedThreads / 32];
    const int r = blockIdx.y, i0 = blockIdx.z * kDotsQ;
    long long o, len;
    seg_of(offs, N, r, o, len);
    const double2* wr = w + o;
    const double2* vb = V + (long long)i0 * vstride + o;
    switch (min(kDotsQ, J - i0)) {
        case 1: dots_body<1>(vb, vstride, wr, len, R, i0, r, part, red); break;
        case 2: dots_body<2>(vb, vstride, wr, len, R, i0, r, part, red); break;
        case 3: dots_body<3>(vb, vstride, wr, len, R, i0, r, part, red); break;
        default: dots_body<4>(vb, vstride, wr, len, R, i0, r, part, red); break;
    }
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
                              int J, double2* __restrict__ w, long long N, int R, double sign,
                              const long long* __restrict__ offs) {
    const int r = blockIdx.y;
    long long o, len;
    seg_of(offs, N, r, o, len);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < len;
         x += (long long)gridDim.x * blockDim.x) {
        double2 acc = mk(0.0, 0.0);
        for (int i = 0; i < J; ++i) acc = cfma(h[i * R + r], V[(long long)i * vstride + o + x], acc);
        double2 wv = w[o + x];
        w[o + x] = mk(wv.x + sign * acc.x, wv.y + sign * acc.y);
    }
}

// y[r] = x[r] * scale[r]  (scale = 0 leaves zeros)
__global__ void scale_kernel(const double2* __restrict__ x, double2* __restrict__ y, const double* __restrict__ sc,
                             long long N, const long long* __restrict__ offs) {
    const int r = blockIdx.y;
    const double s = sc[r];
    long long o, len;
    seg_of(offs, N, r, o, len);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
         e += (long long)gridDim.x * blockDim.x)
        y[o + e] = s * x[o + e];
}

// y = a - b
__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ y,
                           long long tot) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
        y[e] = a[e] - b[e];
}

// ---------------------------------------------------------------- device GMRES state
// Per right-hand side r (R of them), restart length m:
//   H[(r*(m+1) + i)*m + j]   Hessenberg matrix after the rotations (upper triangular part)
//   cs, sn[r*m + j]          Givens rotations
//   rho[r*(m+1) + i]         rotated residual vector
//   gnorm, est, tol          ||g||, |rho_{k}|/||g||, tolerance (state[0])
//   kc, iters, done          steps in this cycle, steps in total, converged flag
//   any                      some right-hand side is still active
struct GState {
    double2 *H, *cs, *sn, *rho;
    double *gnorm, *est, *tol;
    int *kc, *iters, *done, *any;
};

size_t gstate_bytes(int m, int R) {
    return (size_t)R * ((size_t)(m + 1) * m + 2 * (size_t)m + (m + 1)) * sizeof(double2) +
           (size_t)(2 * R + 1) * sizeof(double) + (size_t)(3 * R + 1) * sizeof(int) + 256;
}

GState gstate_at(void* base, int m, int R) {
    GState g;
    char* p = (char*)base;
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 15) & ~(size_t)15; return (void*)q; };
    g.H = (double2*)take((size_t)R * (m + 1) * m * sizeof(double2));
    g.cs = (double2*)take((size_t)R * m * sizeof(double2));
    g.sn = (double2*)take((size_t)R * m * sizeof(double2));
    g.rho = (double2*)take((size_t)R * (m + 1) * sizeof(double2));
    g.gnorm = (double*)take(R * sizeof(double));
    g.est = (double*)take(R * sizeof(double));
    g.tol = (double*)take(sizeof(double));
    g.kc = (int*)take(R * sizeof(int));
    g.iters = (int*)take(R * sizeof(int));
    g.done = (int*)take(R * sizeof(int));
    g.any = (int*)take(sizeof(int));
    return g;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double cabsd(double2 a) { return hypot(a.x, a.y); }

// Start of a restart cycle: beta_r = ||r_r|| (from the norm reduction bn2),
// rho = beta e_1, scales 1/beta for the first basis vector.  first: also
// ||g||, the convergence flags and the step counters.  One block.
__global__ void cycle_init_kernel(GState gs, const double2* __restrict__ bn2, double* __restrict__ sc, int R, int m,
                                  int first, double tol) {
    int act = 0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double beta = sqrt(fmax(0.0, bn2[r].x));
        if (first) {
            gs.gnorm[r] = beta;
            gs.done[r] = beta == 0.0;
            gs.iters[r] = 0;
            gs.est[r] = 0.0;
        }
        gs.rho[(size_t)r * (m + 1)] = mk(beta, 0.0);
        for (int i = 1; i <= m; ++i) gs.rho[(size_t)r * (m + 1) + i] = mk(0.0, 0.0);
        gs.kc[r] = 0;
        const bool a = !gs.done[r] && beta > 0.0;
        sc[r] = a ? 1.0 / beta : 0.0;
        act |= a;
    }
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) {
        gs.any[0] = act;
        if (first) gs.tol[0] = tol;
    }
}

// Step j of the Arnoldi process for every active right-hand side: Hessenberg
// column j = h1 + h2 (the two Gram-Schmidt passes) with H(j+1, j) = ||w||,
// the previous rotations applied, a new rotation annihilating H(j+1, j), the
// rotated residual and its estimate |rho_{j+1}|/||g||; a right-hand side stops
// when the estimate reaches tol (or w vanished).  sc = 1/||w|| for the next
// basis vector (0 once stopped).  One block.
__global__ void givens_kernel(GState gs, const double2* __restrict__ h1, const double2* __restrict__ h2,
                              const double2* __restrict__ hn, double* __restrict__ sc, int R, int m, int j) {
    int act = 0;
    const double tol = gs.tol[0];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        if (gs.done[r]) { sc[r] = 0.0; continue; }
        double2* Hr = gs.H + (size_t)r * (m + 1) * m;
        double2* cs = gs.cs + (size_t)r * m;
        double2* sn = gs.sn + (size_t)r * m;
        double2* rho = gs.rho + (size_t)r * (m + 1);
        for (int i = 0; i <= j; ++i) Hr[(size_t)i * m + j] = h1[(size_t)i * R + r] + h2[(size_t)i * R + r];
        const double hnr = sqrt(fmax(0.0, hn[r].x));
        Hr[(size_t)(j + 1) * m + j] = mk(hnr, 0.0);
        for (int i = 0; i < j; ++i) {
            const double2 a = Hr[(size_t)i * m + j], b = Hr[(size_t)(i + 1) * m + j];
            const double2 cc = cs[i], ss = sn[i];
            Hr[(size_t)i * m + j] = cmul(cc, a) + cmul(ss, b);
            Hr[(size_t)(i + 1) * m + j] = cmul(conjc(cc), b) - cmul(conjc(ss), a);
        }
        const double2 a = Hr[(size_t)j * m + j], b = Hr[(size_t)(j + 1) * m + j];
        const double den = sqrt(cabs2(a) + cabs2(b));
        const double2 cc = den > 0 ? mk(a.x / den, -a.y / den) : mk(1.0, 0.0);
        const double2 ss = den > 0 ? mk(b.x / den, -b.y / den) : mk(0.0, 0.0);
        cs[j] = cc;
        sn[j] = ss;
        Hr[(size_t)j * m + j] = cmul(cc, a) + cmul(ss, b);
        Hr[(size_t)(j + 1) * m + j] = mk(0.0, 0.0);
        const double2 rj = rho[j];
        rho[j + 1] = mk(0.0, 0.0) - cmul(conjc(ss), rj);
        rho[j] = cmul(cc, rj);
        gs.iters[r] += 1;
        gs.kc[r] = j + 1;
        const double e = cabsd(rho[j + 1]) / gs.gnorm[r];
        gs.est[r] = e;
        const bool stop = e <= tol || hnr == 0.0;
        gs.done[r] = stop;
        sc[r] = (!stop && hnr > 0) ? 1.0 / hnr : 0.0;
        act |= !stop;
    }
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) gs.any[0] = act;
}

// y = R^{-1} rho for the kc[r] steps of this cycle of every right-hand side
// (back substitution with the rotated upper-triangular H), written as
// y[i*R + r] for i < J (zero beyond kc[r]).  One block.
__global__ void backsolve_kernel(GState gs, double2* __restrict__ y, int R, int m, int J) {
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const int k = gs.kc[r];
        const double2* Hr = gs.H + (size_t)r * (m + 1) * m;
        const double2* rho = gs.rho + (size_t)r * (m + 1);
        for (int i = J - 1; i >= 0; --i) {
            if (i >= k) { y[(size_t)i * R + r] = mk(0.0, 0.0); continue; }
            double2 acc = rho[i];
            for (int l = i + 1; l < k; ++l) acc = acc - cmul(Hr[(size_t)i * m + l], y[(size_t)l * R + r]);
            y[(size_t)i * R + r] = cmul(acc, crecip(Hr[(size_t)i * m + i]));
        }
    }
}

// Runs the iteration that follows only while some right-hand side is active.
__global__ void gate_kernel(const int* __restrict__ any, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, any[0] != 0 ? 1u : 0u);
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
    const long long* offs;   // per right-hand side segments (null: uniform length N)
};

// h[0..J) for every r = V_i^H w  (accumulate: h += ...)
void dots(Krylov& K, const double2* V, long long vstride, int J, const double2* w, double2* h, int accumulate) {
    ProfScope ps(K.c, K.s, LSS_PROF_KRYLOV, 2);
    dots_multi_kernel<<<dim3(K.nblk, K.R, (J + kDotsQ - 1) / kDotsQ), kRedThreads, 0, K.s>>>(V, vstride, w, K.N,
                                                                                            K.R, J, K.part, K.offs);
    const int JR = J * K.R;
    reduce_kernel<<<JR, kRedThreads, 0, K.s>>>(K.part, K.nblk, h, accumulate);
}

// The FGMRES driver over R right-hand sides of one operator: the vectors
// (RN entries each) hold the right-hand sides side by side, in segments of
// N entries or given by offs; apply_A and precond act on a whole vector.
struct FgOps {
    long long N;              // entries per right-hand side (the longest with offs)
    long long RN;             // entries of a whole vector
    const long long* offs;    // device, R + 1 segment offsets, or null
    std::function<int(const double2*, double2*, cudaStream_t)> apply_A, precond;
    bool graphs;              // iterations may be captured into CUDA graphs
    int key;                  // graph key beside R and the restart length
};

// Workspace generation that captured graphs depend on: a batch's own buffers
// and every instance's (each counter only grows, so the sum changes whenever
// any of them does).
unsigned long long gen_of(const lss_ctx* c) {
    unsigned long long g = c->buf_gen;
    for (const lss_ctx* ci : c->inst) g += ci->buf_gen;
    return g;
}

int fgmres_core(lss_ctx* c, const FgOps& F, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
                cudaStream_t s) {
    const long long N = F.N;
    const int transpose = F.key;
    auto apply_A = F.apply_A;
    const int m = o->restart;
    const int maxit = o->max_iter;
    const long long RN = F.RN;
    // storage: V (m+1), Z (m), w, r
    const size_t nvec = (size_t)(m + 1) + m + 2;
    int rc = lss_grow(c, (void**)&c->kr_buf, &c->kr_cap, nvec * RN * sizeof(double2));
    if (rc) return rc;
    double2* V = c->kr_buf;
    double2* Z = V + (size_t)(m + 1) * RN;
    double2* w = Z + (size_t)m * RN;
    double2* rv = w + RN;
    Krylov K{c, s, N, R, 0, nullptr, nullptr, nullptr, nullptr, nullptr, 0, F.offs};
    // grids sized for the whole batch: about four CTAs per SM over all right-hand sides
    K.nblk = std::max(1, std::min(4 * c->num_sms / R, (int)((N + kRedThreads - 1) / kRedThreads)));
    const size_t red_bytes = (size_t)(m + 1) * R * K.nblk * sizeof(double2) +
                             (size_t)(2 * (m + 1) + 1) * R * sizeof(double2) + (size_t)R * sizeof(double) + 64;
    rc = lss_grow(c, (void**)&c->red_buf, &c->red_cap, red_bytes);
    if (!rc) rc = lss_grow(c, &c->gm_buf, &c->gm_cap, gstate_bytes(m, R));
    if (rc) return rc;
    K.part = c->red_buf;
    K.hdev = K.part + (size_t)(m + 1) * R * K.nblk;
    K.h2dev = K.hdev + (size_t)(m + 1) * R;
    K.hnorm = K.h2dev + (size_t)(m + 1) * R;
    K.scdev = reinterpret_cast<double*>(K.hnorm + R);
    const GState gs = gstate_at(c->gm_buf, m, R);
    const int g1 = std::max(1, std::min(4 * c->num_sms / R, (int)((N + 255) / 256)));
    const int gs_grid = std::max(1, std::min(4 * c->num_sms, (int)((RN + 255) / 256)));
    const int small = std::min(1024, std::max(32, (R + 31) / 32 * 32));

    double2* hnorm = K.hnorm;

    // Iteration j on stream bs: Z_j = P V_j, w = A Z_j, two Gram-Schmidt passes
    // against V_0..V_j, ||w||^2, the Givens update of every right-hand side,
    // V_{j+1} = w / ||w||.
    auto body = [&](int j, cudaStream_t bs) -> int {
        Krylov Kb = K;
        Kb.s = bs;
        const double2* Vj = V + (size_t)j * RN;
        double2* Zj = Z + (size_t)j * RN;
        int r = F.precond(Vj, Zj, bs);
        if (!r) r = apply_A(Zj, w, bs);
        if (r) return r;
        dots(Kb, V, RN, j + 1, w, K.hdev, 0);
        { ProfScope ps_(c, bs, LSS_PROF_KRYLOV, 1); update_kernel<<<dim3(g1, R), 256, 0, bs>>>(V, RN, K.hdev, j + 1, w, N, R, -1.0, F.offs); }
        dots(Kb, V, RN, j + 1, w, K.h2dev, 0);
        { ProfScope ps_(c, bs, LSS_PROF_KRYLOV, 1); update_kernel<<<dim3(g1, R), 256, 0, bs>>>(V, RN, K.h2dev, j + 1, w, N, R, -1.0, F.offs); }
        dots(Kb, w, 0, 1, w, hnorm, 0);
        {
            ProfScope ps_(c, bs, LSS_PROF_KRYLOV, 2);
            givens_kernel<<<1, small, 0, bs>>>(gs, K.hdev, K.h2dev, hnorm, K.scdev, R, m, j);
            scale_kernel<<<dim3(g1, R), 256, 0, bs>>>(w, V + (size_t)(j + 1) * RN, K.scdev, N, F.offs);
        }
        return lss_check_cuda(c, cudaGetLastError(), "arnoldi");
    };
    // Graphs: only once a solve with this R, transpose and restart length ran
    // uncaptured at the current workspace generation (every buffer the body
    // touches exists), not while profiling (events around kernel groups), and
    // not for the 3D sweep (a cooperative grid-synchronised launch).
    const bool use_graph = F.graphs && c->graphs_on && !c->prof_on;
    bool warm = false;
    for (const auto& k : c->graph_warm)
        warm |= k[0] == R && k[1] == transpose && (unsigned long long)k[2] == gen_of(c) && k[3] == m;
    warm &= use_graph;
    // graph of iteration j: a gate kernel (sets the condition from gs.any)
    // followed by an IF node whose body is the captured iteration
    auto graph_for = [&](int j) -> cudaGraphExec_t {
        for (const auto& gr : c->graphs)
            if (gr.j == j && gr.R == R && gr.transpose == transpose && gr.gen == gen_of(c) && gr.m == m)
                return gr.exec;
        std::vector<lss_ctx::GraphRec> keep;   // drop graphs of older workspaces
        for (const auto& gr : c->graphs) {
            if (gr.gen == gen_of(c)) keep.push_back(gr);
            else if (gr.exec) cudaGraphExecDestroy(gr.exec);
        }
        c->graphs.swap(keep);
        const unsigned long long gen0 = gen_of(c);
        const std::string err0 = c->err;
        cudaGraphExec_t ex = nullptr;
        cudaGraph_t graph = nullptr;
        bool ok = (c->cap_stream || !cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) &&
                  !cudaGraphCreate(&graph, 0);
        cudaGraphConditionalHandle hcond = 0;
        cudaGraphNode_t gate = nullptr, cond = nullptr;
        if (ok) ok = !cudaGraphConditionalHandleCreate(&hcond, graph, 0, 0);
        if (ok) {
            void* args[] = {(void*)&gs.any, (void*)&hcond};
            cudaKernelNodeParams kp{};
            kp.func = (void*)gate_kernel;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1);
            kp.kernelParams = args;
            ok = !cudaGraphAddKernelNode(&gate, graph, nullptr, 0, &kp);
        }
        cudaGraph_t bodyg = nullptr;
        if (ok) {
            cudaGraphNodeParams cp{};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hcond;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            ok = !cudaGraphAddNode(&cond, graph, &gate, nullptr, 1, &cp);
            if (ok) bodyg = cp.conditional.phGraph_out[0];
        }
        if (ok) ok = !cudaStreamBeginCaptureToGraph(c->cap_stream, bodyg, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal);
        if (ok) {
            const int brc = body(j, c->cap_stream);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &out);
            ok = !brc && !e && gen_of(c) == gen0;
            if (ok && cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) ex = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();   // a refused capture leaves no error behind
        c->err = err0;
        // a body that cannot be captured (e.g. the grid-synchronised recurrence)
        // is remembered as such and runs uncaptured
        c->graphs.push_back({j, R, transpose, m, gen0, ok ? ex : nullptr});
        return ok ? ex : nullptr;
    };
    auto launch_iteration = [&](int j, bool& graphed) -> int {
        graphed = false;
        if (warm) {
            cudaGraphExec_t ex = graph_for(j);
            if (ex) {
                graphed = true;
                return lss_check_cuda(c, cudaGraphLaunch(ex, s), "iteration graph");
            }
        }
        return body(j, s);
    };

    // ||g||, cycle 0
    dots(K, g, 0, 1, g, K.hdev, 0);
    { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); cycle_init_kernel<<<1, small, 0, s>>>(gs, K.hdev, K.scdev, R, m, 1, o->tol); }
    cudaMemsetAsync(u, 0, RN * sizeof(double2), s);
    cudaMemcpyAsync(rv, g, RN * sizeof(double2), cudaMemcpyDeviceToDevice, s);

    std::vector<int> kc(R), done(R), iters(R);
    std::vector<double> est(R), gnorm(R);
    int total = 0, any = 1;
    // pipeline of graphed iterations: after iteration j the device copies its
    // "some RHS active" flag to pinned host memory and records an event; the
    // host launches iteration j + 1 while j - 1 may still run, and looks at
    // the flag of iteration j - kAhead before launching more (an iteration
    // launched after convergence is skipped by its conditional node)
    constexpr int kAhead = 2;
    if (!c->host_flags && cudaHostAlloc((void**)&c->host_flags, 8 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->host_flags = nullptr;
    }
    for (int q = 0; q < 8 && c->host_flags; ++q)
        if (!c->iter_ev[q] && cudaEventCreateWithFlags(&c->iter_ev[q], cudaEventDisableTiming) != cudaSuccess)
            return lss_check_cuda(c, cudaGetLastError(), "iteration events");
    while (true) {
        { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); scale_kernel<<<dim3(g1, R), 256, 0, s>>>(rv, V, K.scdev, N, F.offs); }
        const int nj = std::min(m, maxit - total);
        for (int j = 0; j < nj; ++j) {
            bool graphed = false;
            if ((rc = launch_iteration(j, graphed))) return rc;
            if (!graphed || !c->host_flags) {   // kernel by kernel: stop as soon as every RHS converged
                cudaError_t e = cudaMemcpyAsync(&any, gs.any, sizeof(int), cudaMemcpyDeviceToHost, s);
                if (!e) e = cudaStreamSynchronize(s);
                if ((rc = lss_check_cuda(c, e, "arnoldi status"))) return rc;
                if (!any) break;
                continue;
            }
            cudaError_t e = cudaMemcpyAsync(c->host_flags + (j & 7), gs.any, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaEventRecord(c->iter_ev[j & 7], s);
            if (!e && j >= kAhead) e = cudaEventSynchronize(c->iter_ev[(j - kAhead) & 7]);
            if ((rc = lss_check_cuda(c, e, "arnoldi status"))) return rc;
            if (j >= kAhead && !*(volatile int*)(c->host_flags + ((j - kAhead) & 7))) break;
        }
        // once per cycle: steps taken, convergence
        cudaError_t e = cudaMemcpyAsync(kc.data(), gs.kc, R * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(done.data(), gs.done, R * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if ((rc = lss_check_cuda(c, e, "krylov cycle state"))) return rc;
        const int J = *std::max_element(kc.begin(), kc.end());
        total += J;
        if (J > 0) {   // x += Z y with y from each RHS's triangular system
            ProfScope ps_(c, s, LSS_PROF_KRYLOV, 2);
            backsolve_kernel<<<1, small, 0, s>>>(gs, K.hdev, R, m, J);
            update_kernel<<<dim3(g1, R), 256, 0, s>>>(Z, RN, K.hdev, J, u, N, R, +1.0, F.offs);
        }
        bool all_done = true;
        for (int r = 0; r < R; ++r) all_done &= (bool)done[r];
        if (all_done || total >= maxit || J == 0) break;
        // restart: r = g - A u
        if ((rc = apply_A(u, w, s))) return rc;
        { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); sub_kernel<<<gs_grid, 256, 0, s>>>(g, w, rv, RN); }
        dots(K, rv, 0, 1, rv, K.hdev, 0);
        { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); cycle_init_kernel<<<1, small, 0, s>>>(gs, K.hdev, K.scdev, R, m, 0, o->tol); }
    }
    // true residual
    if ((rc = apply_A(u, w, s))) return rc;
    { ProfScope ps_(c, s, LSS_PROF_KRYLOV, 1); sub_kernel<<<gs_grid, 256, 0, s>>>(g, w, rv, RN); }
    dots(K, rv, 0, 1, rv, K.hdev, 0);
    std::vector<double2> hh(R);
    cudaError_t e = cudaMemcpyAsync(hh.data(), K.hdev, R * sizeof(double2), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(iters.data(), gs.iters, R * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(est.data(), gs.est, R * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(gnorm.data(), gs.gnorm, R * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(done.data(), gs.done, R * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if ((rc = lss_check_cuda(c, e, "krylov fetch"))) return rc;
    bool conv = true;
    for (int r = 0; r < R; ++r) {
        const double rt = gnorm[r] > 0 ? std::sqrt(std::max(0.0, hh[r].x)) / gnorm[r] : 0.0;
        const bool cv = gnorm[r] == 0.0 || est[r] <= o->tol;
        conv &= cv;
        if (st) {
            st[r].iters = iters[r];
            st[r].converged = cv ? 1 : 0;
            st[r].relres_est = est[r];
            st[r].relres_true = rt;
        }
    }
    if ((rc = lss_check_device_err(c, s))) return rc;
    if (use_graph && !warm) {   // later solves with this R, transpose and m replay captured iterations
        std::vector<std::array<long long, 4>> keep;
        for (const auto& k : c->graph_warm)
            if ((unsigned long long)k[2] == gen_of(c) && !(k[0] == R && k[1] == transpose && k[3] == m))
                keep.push_back(k);
        keep.push_back({(long long)R, (long long)transpose, (long long)gen_of(c), (long long)m});
        c->graph_warm.swap(keep);
    }
    return conv ? LSS_OK : lss_fail(c, LSS_ERR_NOCONVERGE, "GMRES reached max_iter before tol");
}

}  // namespace

int lss_fgmres(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
               cudaStream_t s, int transpose) {
    // transpose = 1: solve A^T x = g (A^T = I + omega^2 M K) preconditioned by P^T;
    // transpose = 2: the sparsified system H x = g on the n_tot^2 grid (Sec. 4)
    // preconditioned by the sweep on grid vectors
    const int mv_in = transpose ? MV_IN_U : MV_IN_MU, mv_out = transpose ? MV_OUT_AT : MV_OUT_A;
    const bool grid = transpose == 2;
    const long long N = grid ? (long long)c->n_tot * c->n_tot : c->npts();
    if (transpose == 1) {
        const int rc = lss_prepare_sweep_t(c, s);
        if (rc) return rc;
    } else {   // block LU factors before any iteration is captured
        const int rc = lss_thomas_prepare(c, R, s);
        if (rc) return rc;
    }
    FgOps F;
    F.N = N;
    F.RN = (long long)R * N;
    F.offs = nullptr;
    F.apply_A = [c, R, grid, mv_in, mv_out](const double2* x, double2* y, cudaStream_t st_) -> int {
        return grid ? lss_apply_H(c, x, y, R, st_) : lss_matvec(c, x, y, R, mv_in, mv_out, nullptr, nullptr, st_);
    };
    F.precond = [c, R, grid, transpose](const double2* x, double2* y, cudaStream_t st_) -> int {
        return grid ? lss_sweep_grid(c, x, y, R, st_)
                    : (transpose ? lss_sweep_t(c, x, y, R, st_) : lss_sweep(c, x, y, R, st_));
    };
    // not for the 3D sweep (a cooperative grid-synchronised launch)
    F.graphs = c->dim == 2;
    F.key = transpose;
    return fgmres_core(c, F, g, u, R, o, st, s);
}

// The ragged batch in lockstep: every instance's right-hand sides advance
// together as the segments of one set of Krylov vectors (instance q's R x n_q^2
// entries side by side, as in the batch layout), one driver for all of them;
// the operator and the preconditioner act on every instance (lss_batch_op).
int lss_fgmres_batch(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
                     cudaStream_t s, int transpose) {
    const int nq = (int)c->inst.size();
    const int RB = nq * R;
    std::vector<long long> offs(RB + 1);
    long long nmax = 0;
    for (int q = 0; q < nq; ++q) {
        const long long nn = c->inst_off[q + 1] - c->inst_off[q];
        nmax = std::max(nmax, nn);
        for (int r = 0; r < R; ++r) offs[q * R + r] = (long long)R * c->inst_off[q] + (long long)r * nn;
    }
    offs[RB] = (long long)R * c->inst_off[nq];
    int rc = lss_grow(c, &c->seg_buf, &c->seg_cap, offs.size() * sizeof(long long));
    if (!rc) rc = lss_check_cuda(c, cudaMemcpyAsync(c->seg_buf, offs.data(), offs.size() * sizeof(long long),
                                                    cudaMemcpyHostToDevice, s), "batch segments");
    if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "batch segments");
    if (rc) return rc;
    FgOps F;
    F.N = nmax;
    F.RN = offs[RB];
    F.offs = (const long long*)c->seg_buf;
    F.apply_A = [c, R, transpose](const double2* x, double2* y, cudaStream_t st_) -> int {
        return lss_batch_op(c, 0, x, y, R, transpose, st_);
    };
    F.precond = [c, R, transpose](const double2* x, double2* y, cudaStream_t st_) -> int {
        return lss_batch_op(c, 1, x, y, R, transpose, st_);
    };
    F.graphs = true;   // the instances' launches join the capture through the fork/join events
    F.key = transpose;
    return fgmres_core(c, F, g, u, RB, o, st, s);
}
