// LS operator (Sec. 2.1, Eq. LS_d_c): y = u + omega^2 sum_{j in I} k_{i-j} m_j u_j,
// evaluated as a zero-padded FFT convolution on an L^2 grid (L >= 2n-1, power
// of two).  Three launches per operator application, FP64 throughout:
//   1. row pass: for each of the n nonzero rows, form m.*u (or u, or m.*u_I),
//      zero-pad to L and FFT along x2;
//   2. column pass: FFT along x1 of every column (only n of L inputs are
//      nonzero), multiply by the transposed kernel transform, inverse FFT,
//      keep the n rows that land on I;
//   3. row pass: inverse FFT along x2, keep the n columns on I, fused epilogue
//      (u + ., u + m.*., or -.).
// The FFT is a shared-memory Stockham autosort transform with radix-4 stages
// (one radix-2 stage when log2 L is odd).
#include "fft_line.cuh"
#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"

namespace {

struct Dir2 { double d0, d1; };

// Pass 1.  grid (rows, R), block >= 32 threads.  Output buf[r][row][0..L).
template <int IN>
__global__ void mv_rows_fwd(const double2* __restrict__ x, const double* __restrict__ m,
                            const double* __restrict__ dirs, double2* __restrict__ uI,
                            double2* __restrict__ buf, const double2* __restrict__ tw, int n, int rows,
                            int L, int lg, double omega, double h) {
    extern __shared__ double2 sm[];
    double2* a = sm;
    double2* b = sm + L;
    const int row = blockIdx.x, r = blockIdx.y, t = threadIdx.x, nt = blockDim.x;
    const long long N = (long long)n * n;
    for (int j = t; j < L; j += nt) {
        double2 v = mk(0.0, 0.0);
        if (IN == MV_IN_RAW) {
            v = x[(long long)row * L + j];
        } else if (j < n) {
            const long long e = (long long)row * n + j;
            if (IN == MV_IN_MU) {
                v = m[e] * x[r * N + e];
            } else if (IN == MV_IN_U) {
                v = x[r * N + e];
            } else {  // plane wave u_I = exp(i omega d.p), p = ((row+1) h, (j+1) h)
                const double ph = omega * (dirs[2 * r] * (row + 1) * h + dirs[2 * r + 1] * (j + 1) * h);
                double sn, cs;
                sincos(ph, &sn, &cs);
                if (uI) uI[r * N + e] = mk(cs, sn);
                v = m[e] * mk(cs, sn);
            }
        }
        a[j] = v;
    }
    __syncthreads();
    double2* res = fft_line<false>(a, b, L, lg, tw, t, nt);
    double2* out = buf + ((long long)r * rows + row) * L;
    for (int j = t; j < L; j += nt) out[j] = res[j];
}

// Pass 2.  grid (L/C, R), block C * nt threads; group g handles column c0+g.
// CONV: forward FFT along x1, multiply by khatT, inverse FFT, store rows < n.
// !CONV: forward FFT only, store scale * result transposed into khat_out.
template <bool CONV>
__global__ void mv_cols(double2* __restrict__ buf, const double2* __restrict__ khatT,
                        double2* __restrict__ khat_out, const double2* __restrict__ tw, int rows, int L,
                        int lg, int C, double scale) {
    extern __shared__ double2 sm[];
    double2* A = sm;
    double2* B = sm + (size_t)C * L;
    const int c0 = blockIdx.x * C, r = blockIdx.y;
    const int nt = blockDim.x / C, g = threadIdx.x / nt, t = threadIdx.x % nt;
    double2* bb = buf + (long long)r * rows * L;
    for (int idx = threadIdx.x; idx < rows * C; idx += blockDim.x) {
        const int row = idx / C, c = idx % C;
        A[(size_t)c * L + row] = bb[(long long)row * L + c0 + c];
    }
    for (int idx = threadIdx.x; idx < (L - rows) * C; idx += blockDim.x) {
        const int row = rows + idx / C, c = idx % C;
        A[(size_t)c * L + row] = mk(0.0, 0.0);
    }
    __syncthreads();
    double2* res = fft_line<false>(A + (size_t)g * L, B + (size_t)g * L, L, lg, tw, t, nt);
    const int col = c0 + g;
    if (!CONV) {
        for (int k = t; k < L; k += nt) khat_out[(long long)col * L + k] = scale * res[k];
        return;
    }
    const double2* kh = khatT + (long long)col * L;
    for (int k = t; k < L; k += nt) res[k] = res[k] * __ldg(&kh[k]);
    __syncthreads();
    double2* other = (res == A + (size_t)g * L) ? B + (size_t)g * L : A + (size_t)g * L;
    double2* inv = fft_line<true>(res, other, L, lg, tw, t, nt);
    // every group's result sits in the same half (A or B): write rows < n back
    const double2* base = (inv == A + (size_t)g * L) ? A : B;
    for (int idx = threadIdx.x; idx < rows * C; idx += blockDim.x) {
        const int row = idx / C, c = idx % C;
        bb[(long long)row * L + c0 + c] = base[(size_t)c * L + row];
    }
}

// Pass 3.  grid (n, R).
template <int OUT>
__global__ void mv_rows_inv(const double2* __restrict__ buf, const double2* __restrict__ x,
                            const double* __restrict__ m, double2* __restrict__ y,
                            const double2* __restrict__ tw, int n, int L, int lg) {
    extern __shared__ double2 sm[];
    double2* a = sm;
    double2* b = sm + L;
    const int row = blockIdx.x, r = blockIdx.y, t = threadIdx.x, nt = blockDim.x;
    const long long N = (long long)n * n;
    const double2* in = buf + ((long long)r * n + row) * L;
    for (int j = t; j < L; j += nt) a[j] = in[j];
    __syncthreads();
    double2* res = fft_line<true>(a, b, L, lg, tw, t, nt);
    for (int j = t; j < n; j += nt) {
        const long long e = (long long)row * n + j;
        const double2 v = res[j];
        if (OUT == MV_OUT_A) y[r * N + e] = x[r * N + e] + v;
        else if (OUT == MV_OUT_AT) y[r * N + e] = x[r * N + e] + m[e] * v;
        else y[r * N + e] = mk(-v.x, -v.y);
    }
}

int col_group(int L) { return L >= 2048 ? 1 : 2; }
int line_threads(int L) { return L / 4 < 32 ? 32 : L / 4; }
constexpr int kFftSmax = 200 * 1024;   // dynamic shared memory the FFT kernels are opted into

int col_group(const lss_ctx* c) { return c->tune.fft_C ? c->tune.fft_C : col_group(c->L); }

}  // namespace

std::vector<int> lss_fft_col_candidates(const lss_ctx* c) {
    std::vector<int> out;
    const int L = c->L;
    for (int C : {1, 2, 4, 8})
        if (L % C == 0 && C * line_threads(L) <= 1024 && 2 * (size_t)C * L * sizeof(double2) <= (size_t)kFftSmax)
            out.push_back(C);
    return out;
}

int lss_matvec(lss_ctx* c, const double2* x, double2* y, int R, int in_mode, int out_mode,
               const double* dirs_dev, double2* uI, cudaStream_t s) {
    if (c->dim == 3) return lss3_matvec(c, x, y, R, in_mode, out_mode, dirs_dev, uI, s);
    const int n = c->n, L = c->L, lg = c->lgL;
    const size_t need = (size_t)n * L * R * sizeof(double2);
    int rc = lss_grow(c, (void**)&c->mv_buf, &c->mv_cap, need);
    if (rc) return rc;
    const int nt = line_threads(L);
    const size_t sh = 2 * (size_t)L * sizeof(double2);
    dim3 g1(n, R);
    ProfScope ps(c, s, LSS_PROF_MATVEC, 3);
    switch (in_mode) {
        case MV_IN_MU:
            mv_rows_fwd<MV_IN_MU><<<g1, nt, sh, s>>>(x, c->m, nullptr, nullptr, c->mv_buf, c->tw, n, n, L, lg,
                                                   c->omega, c->h);
            break;
        case MV_IN_U:
            mv_rows_fwd<MV_IN_U><<<g1, nt, sh, s>>>(x, c->m, nullptr, nullptr, c->mv_buf, c->tw, n, n, L, lg,
                                                  c->omega, c->h);
            break;
        case MV_IN_PLANEWAVE:
            mv_rows_fwd<MV_IN_PLANEWAVE><<<g1, nt, sh, s>>>(x, c->m, dirs_dev, uI, c->mv_buf, c->tw, n, n, L,
                                                          lg, c->omega, c->h);
            break;
        default:
            return lss_fail(c, LSS_ERR_ARG, "matvec: bad input mode");
    }
    const int C = col_group(c);
    const size_t sh2 = 2 * (size_t)C * L * sizeof(double2);
    mv_cols<true><<<dim3(L / C, R), C * nt, sh2, s>>>(c->mv_buf, c->khatT, nullptr, c->tw, n, L, lg, C, 1.0);
    switch (out_mode) {
        case MV_OUT_A:
            mv_rows_inv<MV_OUT_A><<<g1, nt, sh, s>>>(c->mv_buf, x, c->m, y, c->tw, n, L, lg);
            break;
        case MV_OUT_AT:
            mv_rows_inv<MV_OUT_AT><<<g1, nt, sh, s>>>(c->mv_buf, x, c->m, y, c->tw, n, L, lg);
            break;
        default:
            mv_rows_inv<MV_OUT_NEG><<<g1, nt, sh, s>>>(c->mv_buf, x, c->m, y, c->tw, n, L, lg);
            break;
    }
    return lss_check_cuda(c, cudaGetLastError(), "matvec launch");
}

// kc: L x L circular kernel table (device).  khatT = omega^2/L^2 * FFT2(kc), transposed.
int lss_fft_kernel_table(lss_ctx* c, const double2* kc, cudaStream_t s) {
    const int L = c->L, lg = c->lgL;
    int rc = lss_grow(c, (void**)&c->mv_buf, &c->mv_cap, (size_t)L * L * sizeof(double2));
    if (rc) return rc;
    const int nt = line_threads(L);
    const size_t sh = 2 * (size_t)L * sizeof(double2);
    ProfScope ps(c, s, LSS_PROF_SETUP, 2);
    mv_rows_fwd<MV_IN_RAW><<<dim3(L, 1), nt, sh, s>>>(kc, nullptr, nullptr, nullptr, c->mv_buf, c->tw, c->n, L,
                                                     L, lg, c->omega, c->h);
    const int C = col_group(L);
    const double scale = c->omega * c->omega / ((double)L * (double)L);
    mv_cols<false><<<dim3(L / C, 1), C * nt, 2 * (size_t)C * L * sizeof(double2), s>>>(
        c->mv_buf, nullptr, c->khatT, c->tw, L, L, lg, C, scale);
    return lss_check_cuda(c, cudaGetLastError(), "kernel table fft");
}

// Opt the FFT kernels into large dynamic shared memory once per device.
int lss_fft_configure(lss_ctx* c) {
    std::lock_guard<std::mutex> lock(lss_config_mutex());
    long long& done = lss_dev_cache((const void*)&lss_fft_configure, 0);
    if (done) return LSS_OK;
    const int smax = kFftSmax;
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(mv_rows_fwd<MV_IN_MU>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_rows_fwd<MV_IN_U>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_rows_fwd<MV_IN_PLANEWAVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_rows_fwd<MV_IN_RAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_cols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_cols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_rows_inv<MV_OUT_A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_rows_inv<MV_OUT_AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (!e) e = cudaFuncSetAttribute(mv_rows_inv<MV_OUT_NEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (e) return lss_check_cuda(c, e, "fft smem attribute");
    done = 1;
    return LSS_OK;
}
