// Sweeping factorization (Sec. 2.3-2.4, Algorithms 1 and 2).
//
// Each slab subproblem S_i (Eq. Hwv_approx) is block tridiagonal along x2 with
// w x w blocks (w layers of the slab): A_k (coupling dk = 0), C_k (dk = -1),
// B_k (dk = +1), each tridiagonal in the layer index.  It is factored by block
// Gaussian elimination, D_0 = A_0, D_k = A_k - C_k D_{k-1}^{-1} B_{k-1}, with
// partial pivoting inside each D_k (Gauss-Jordan), storing G_k = D_k^{-1}.
//
// Algorithm 2's sweep is evaluated slab-parallel.  With a_i = T~_i f_i and the
// interface maps (rows of T~_i applied to unit couplings)
//   Lambda_i = last-layer rows of T~_i H_{[i,i-1]},  Gamma_i = first-layer rows
//   of T~_i H_{[i,i-1]},  Phi_i = first-layer rows of T~_i H_{[i,i+1]},
// the forward sweep's coupling values lambda_i = last layer of u~_i (forward
// pass) and the final first layers phi_i obey
//   lambda_i = last(a_i) - Lambda_i lambda_{i-1},
//   mu_i = first(a_i) - Gamma_i lambda_{i-1},   phi_l = mu_l,
//   phi_i = mu_i - Phi_i phi_{i+1},
// and then u~_i = T~_i (f_i - H_{[i,i-1]} lambda_{i-1} - H_{[i,i+1]} phi_{i+1}),
// which is exactly Algorithm 2's result (linearity of T~_i).  The slab solves
// run for all slabs at once; only the short recurrences on n_tot-vectors are
// sequential.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

constexpr int kStages = 3;     // TMA ring depth of the slab solve
constexpr int kSolveThreads = 128;

enum ThomasMode { TH_A = 0, TH_E = 1, TH_IFACE = 2, TH_TEST = 3 };

// ---------------------------------------------------------------- factorization
template <typename T>
__global__ void __launch_bounds__(256) factor_kernel(const SlabDev* __restrict__ slabs,
                                                     const cx<T>* __restrict__ coef, cx<T>* __restrict__ fac,
                                                     int n_tot, int* err) {
    using C = cx<T>;
    const SlabDev sd = slabs[blockIdx.x];
    const int w = sd.w, w2 = 2 * sd.w, ldw = sd.ldw;
    extern __shared__ __align__(128) unsigned char smraw_f[];
    C* M = reinterpret_cast<C*>(smraw_f);  // w x 2w augmented [D | I]
    C* Gp = M + w * w2;                   // G_{k-1}
    C* X = Gp + w * w;                    // G_{k-1} B_{k-1}
    C* colj = X + w * w;
    __shared__ int piv_row;
    __shared__ C piv_inv;
    const int tid = threadIdx.x, nth = blockDim.x;
    const C* cf = coef + sd.coef_off;
    C* G = fac + sd.fac_off;
    const C zero = czero<C>();
    for (int k = 0; k < n_tot; ++k) {
        const C* ck = cf + (long long)k * sd.cstride;
        for (int idx = tid; idx < w * w2; idx += nth) {
            const int p = idx / w2, q = idx % w2;
            C v = zero;
            if (q < w) {
                const int d = q - p;
                if (d >= -1 && d <= 1) v = ck[p * 9 + (d + 1) * 3 + 1];
            } else if (q - w == p) {
                v.x = 1;
            }
            M[idx] = v;
        }
        if (k > 0) {
            const C* cp = cf + (long long)(k - 1) * sd.cstride;
            for (int idx = tid; idx < w * w; idx += nth) {
                const int p = idx / w, q = idx % w;
                C acc = zero;
                for (int a = max(0, q - 1); a <= min(w - 1, q + 1); ++a)
                    acc = cfma(Gp[p * w + a], cp[a * 9 + (q - a + 1) * 3 + 2], acc);
                X[idx] = acc;
            }
            __syncthreads();
            for (int idx = tid; idx < w * w; idx += nth) {
                const int p = idx / w, q = idx % w;
                C acc = zero;
                for (int a = max(0, p - 1); a <= min(w - 1, p + 1); ++a)
                    acc = cfma(ck[p * 9 + (a - p + 1) * 3 + 0], X[a * w + q], acc);
                M[p * w2 + q] = M[p * w2 + q] - acc;
            }
        }
        __syncthreads();
        for (int j = 0; j < w; ++j) {
            if (tid < 32) {
                const int i = j + tid;
                T val = (i < w) ? cabs2(M[i * w2 + j]) : T(-1);
                int best = i;
                for (int off = 16; off > 0; off >>= 1) {
                    const T ov = __shfl_down_sync(0xffffffffu, val, off);
                    const int ob = __shfl_down_sync(0xffffffffu, best, off);
                    if (ov > val || (ov == val && ob < best)) { val = ov; best = ob; }
                }
                if (tid == 0) {
                    piv_row = best;
                    C pv = M[best * w2 + j];
                    const T a2 = cabs2(pv);
                    if (!(a2 > T(0)) || !isfinite(a2)) {
                        atomicOr(err, LSS_DERR_SINGULAR);
                        pv = zero;
                        pv.x = T(1);
                    }
                    piv_inv = crecip(pv);
                }
            }
            __syncthreads();
            const int pr = piv_row;
            const C pinv = piv_inv;
            for (int q = tid; q < w2; q += nth) {
                const C a = M[j * w2 + q], bb = M[pr * w2 + q];
                M[j * w2 + q] = bb * pinv;
                if (pr != j) M[pr * w2 + q] = a;
            }
            __syncthreads();
            for (int i = tid; i < w; i += nth) colj[i] = (i == j) ? zero : M[i * w2 + j];
            __syncthreads();
            for (int idx = tid; idx < w * w2; idx += nth) {
                const int i = idx / w2, q = idx % w2;
                if (i != j && q > j) M[idx] = M[idx] - colj[i] * M[j * w2 + q];
            }
            __syncthreads();
        }
        C* Gk = G + (long long)k * w * ldw;
        for (int idx = tid; idx < w * ldw; idx += nth) {
            const int p = idx / ldw, q = idx % ldw;
            const C v = (q < w) ? M[p * w2 + w + q] : zero;
            Gk[idx] = v;
            if (q < w) Gp[p * w + q] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- slab solve
template <typename C>
struct ThomasArgs {
    const SlabDev* slabs;
    int n_slabs, n_tot, n, b;
    const C* coef;
    const C* fac;
    const C* f;            // TH_A, TH_E: R x n_tot^2
    C* a_first;            // TH_A: [slab][k][R]
    C* a_last;
    const C* lam;          // TH_E: [slab][k][R]
    const C* phi;
    double2* y;            // TH_E: R x n^2
    C* iface;              // TH_IFACE: [3][slab][k][n_tot]
    const double2* v_in;   // TH_TEST
    double2* w_out;
    int test_slab;
    C* zbuf;               // forward-elimination scratch
    long long zstride;     // per CTA
    int R, RC, col0;       // total RHS, RHS per CTA, first column (TH_IFACE)
    int* err;
};

template <typename C, int MODE>
__device__ __forceinline__ C thomas_rhs(const ThomasArgs<C>& A, const SlabDev& sd, int i, int side, int k, int p,
                                        int r, const C* ck) {
    C v = czero<C>();
    if (MODE == TH_IFACE) {
        const int j = r;  // column = global coupling index
        const int dk = j - k;
        if (dk >= -1 && dk <= 1) {
            if (side == 0 && p == sd.na) v = ck[p * 9 + 0 * 3 + dk + 1];
            if (side == 1 && p == sd.w - 1) v = ck[p * 9 + 2 * 3 + dk + 1];
        }
        return v;
    }
    if (p < sd.na) return v;
    const int x1 = sd.s + (p - sd.na);
    if (MODE == TH_TEST) {
        const double2 t = A.v_in[((long long)r * sd.nl + (p - sd.na)) * A.n_tot + k];
        return to_c<C>(t);
    }
    const long long nt2 = (long long)A.n_tot * A.n_tot;
    v = A.f[(long long)r * nt2 + (long long)(x1 + A.b) * A.n_tot + k];
    if (MODE == TH_E) {
        if (p == sd.na && i > 0) {
            const C* lp = A.lam + (long long)(i - 1) * A.n_tot * A.R;
            for (int dk = -1; dk <= 1; ++dk) {
                const int kk = k + dk;
                if (kk >= 0 && kk < A.n_tot) v = v - ck[p * 9 + 0 * 3 + dk + 1] * lp[(long long)kk * A.R + r];
            }
        }
        if (p == sd.w - 1 && i < A.n_slabs - 1) {
            const C* pp = A.phi + (long long)(i + 1) * A.n_tot * A.R;
            for (int dk = -1; dk <= 1; ++dk) {
                const int kk = k + dk;
                if (kk >= 0 && kk < A.n_tot) v = v - ck[p * 9 + 2 * 3 + dk + 1] * pp[(long long)kk * A.R + r];
            }
        }
    }
    return v;
}

template <typename C, int MODE>
__device__ __forceinline__ void thomas_out(const ThomasArgs<C>& A, const SlabDev& sd, int i, int side, int k, int p,
                                           int r, C x) {
    if (MODE == TH_A) {
        const long long e = ((long long)i * A.n_tot + k) * A.R + r;
        if (p == sd.na) A.a_first[e] = x;
        if (p == sd.w - 1) A.a_last[e] = x;
    } else if (MODE == TH_E) {
        if (p < sd.na) return;
        const int x1 = sd.s + (p - sd.na), i2 = k - A.b;
        if (x1 >= 1 && x1 <= A.n && i2 >= 1 && i2 <= A.n)
            A.y[(long long)r * A.n * A.n + (long long)(x1 - 1) * A.n + (i2 - 1)] = to_d(x);
    } else if (MODE == TH_IFACE) {
        const long long nt2 = (long long)A.n_tot * A.n_tot;
        const long long e = (long long)k * A.n_tot + r;
        if (side == 0) {
            if (p == sd.w - 1) A.iface[(0LL * A.n_slabs + i) * nt2 + e] = x;  // Lambda_i
            if (p == sd.na) A.iface[(1LL * A.n_slabs + i) * nt2 + e] = x;     // Gamma_i
        } else if (p == sd.na) {
            A.iface[(2LL * A.n_slabs + i) * nt2 + e] = x;                       // Phi_i
        }
    } else {
        if (p < sd.na) return;
        A.w_out[((long long)r * sd.nl + (p - sd.na)) * A.n_tot + k] = to_d(x);
    }
}

// One CTA solves S_i x = b for RC right-hand sides: forward elimination
// z_k = G_k (b_k - C_k z_{k-1}), back substitution x_k = z_k - G_k B_k x_{k+1}.
// G_k and the coefficient rows stream through a TMA ring of kStages buffers
// (1D bulk copies completing on mbarriers); the 2 n_tot - 1 block rows are
// visited as one sequence (forward k = 0..K-1, then backward k = K-2..0).
template <typename T, int MODE>
__global__ void __launch_bounds__(kSolveThreads) thomas_kernel(ThomasArgs<cx<T>> A) {
    using C = cx<T>;
    const int i = (MODE == TH_TEST) ? A.test_slab : blockIdx.x;
    const int side = blockIdx.z;
    if (MODE == TH_IFACE) {
        if (i == 0) return;
        if (side == 1 && i == A.n_slabs - 1) return;
    }
    const SlabDev sd = A.slabs[i];
    const int w = sd.w, ldw = sd.ldw, K = A.n_tot;
    const int r0 = blockIdx.y * A.RC;
    const int rtot = (MODE == TH_IFACE) ? A.n_tot : A.R;
    const int rc = min(A.RC, rtot - r0 - (MODE == TH_IFACE ? A.col0 : 0));
    if (rc <= 0) return;
    const int cbase = r0 + (MODE == TH_IFACE ? A.col0 : 0);
    const int RC = A.RC;

    extern __shared__ __align__(128) unsigned char smraw[];
    const int gsz = w * ldw, csz = sd.cstride;
    C* Gs = reinterpret_cast<C*>(smraw);                // kStages x gsz
    C* Cs = Gs + kStages * gsz;                         // kStages x csz
    C* v = Cs + kStages * csz;                          // w x RC
    C* zp = v + w * RC;                                 // w x RC
    __shared__ __align__(8) uint64_t bar[kStages];

    const C* G = A.fac + sd.fac_off;
    const C* cf = A.coef + sd.coef_off;
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    C* Z = A.zbuf + cta * A.zstride;

    const int tid = threadIdx.x, nth = blockDim.x;
    const int outs = w * rc;
    int TP = 1;
    while (TP < 32 && outs * TP * 2 <= nth) TP <<= 1;
    const int ostep = nth / TP;   // outputs per pass; passes cover all w x rc outputs

    const int nseq = 2 * K - 1;
    const unsigned gbytes = (unsigned)(gsz * sizeof(C)), cbytes = (unsigned)(csz * sizeof(C));
    auto kk_of = [K](int pos) { return pos < K ? pos : 2 * K - 2 - pos; };
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int pos = 0; pos < kStages && pos < nseq; ++pos) {
            const int k = kk_of(pos);
            mbar_expect_tx(&bar[pos], gbytes + cbytes);
            tma_load_1d(Gs + pos * gsz, G + (long long)k * gsz, gbytes, &bar[pos]);
            tma_load_1d(Cs + pos * csz, cf + (long long)k * csz, cbytes, &bar[pos]);
        }
    }
    bool ok = true;
    for (int pos = 0; pos < nseq; ++pos) {
        const int st = pos % kStages;
        const int k = kk_of(pos);
        if (!mbar_wait(&bar[st], (pos / kStages) & 1, A.err)) ok = false;
        if (!__syncthreads_and(ok)) break;
        const C* Gk = Gs + st * gsz;
        const C* ck = Cs + st * csz;
        const bool fwd = pos < K;
        // v = b_k - C_k z_{k-1}  (forward)   or   v = B_k x_{k+1}  (backward)
        for (int idx = tid; idx < w * rc; idx += nth) {
            const int p = idx % w, rr = idx / w;
            C bv = czero<C>();
            if (fwd) {
                bv = thomas_rhs<C, MODE>(A, sd, i, side, k, p, cbase + rr, ck);
                if (k > 0)
                    for (int da = -1; da <= 1; ++da) {
                        const int a = p + da;
                        if (a >= 0 && a < w) bv = bv - ck[p * 9 + (da + 1) * 3 + 0] * zp[a * RC + rr];
                    }
            } else {
                for (int da = -1; da <= 1; ++da) {
                    const int a = p + da;
                    if (a >= 0 && a < w) bv = cfma(ck[p * 9 + (da + 1) * 3 + 2], zp[a * RC + rr], bv);
                }
            }
            v[p * RC + rr] = bv;
        }
        __syncthreads();
        for (int ob = 0; ob < outs; ob += ostep) {
            const int o = ob + tid / TP, kq = tid % TP;
            const bool active = o < outs;
            const int op = active ? o % w : 0, orr = active ? o / w : 0;
            C acc = czero<C>();
            if (active)
                for (int a = kq; a < w; a += TP) acc = cfma(Gk[op * ldw + a], v[a * RC + orr], acc);
            for (int off = TP >> 1; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (active && kq == 0) {
                C x;
                if (fwd) {
                    x = acc;
                    Z[((long long)k * w + op) * RC + orr] = x;
                } else {
                    x = Z[((long long)k * w + op) * RC + orr] - acc;
                }
                zp[op * RC + orr] = x;
                if (!fwd || k == K - 1) thomas_out<C, MODE>(A, sd, i, side, k, op, cbase + orr, x);
            }
        }
        __syncthreads();
        if (tid == 0 && pos + kStages < nseq) {
            const int kn = kk_of(pos + kStages);
            mbar_expect_tx(&bar[st], gbytes + cbytes);
            tma_load_1d(Gs + st * gsz, G + (long long)kn * gsz, gbytes, &bar[st]);
            tma_load_1d(Cs + st * csz, cf + (long long)kn * csz, cbytes, &bar[st]);
        }
    }
    if (!ok && tid == 0) {
        // a wait expired: give the copies already issued (at most kStages) a
        // bounded chance to land before the CTA exits
        const unsigned long long t0 = global_ns();
        while (global_ns() - t0 < 1000000ull) __nanosleep(1000);
    }
}

// ---------------------------------------------------------------- interface recurrence
template <typename T>
__global__ void __launch_bounds__(256) recur_kernel(int n_slabs, int n_tot, int R, const cx<T>* __restrict__ iface,
                                                    const cx<T>* __restrict__ a_first,
                                                    const cx<T>* __restrict__ a_last, cx<T>* lam, cx<T>* phi,
                                                    unsigned* bar, int* err) {
    using C = cx<T>;
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < vec;
         e += (long long)gridDim.x * blockDim.x)
        lam[e] = a_last[e];
    for (int i = 1; i < n_slabs; ++i) {
        const C* lp = (i == 1) ? a_last : lam + (long long)(i - 1) * vec;
        const int nwhich = (i <= n_slabs - 2) ? 2 : 1;
        const long long ntask = nwhich * vec;
        for (long long task = gw; task < ntask; task += nw) {
            const int which = (int)(task / vec);
            const long long rem = task % vec;
            const int row = (int)(rem / R), r = (int)(rem % R);
            const C* Mrow = iface + ((long long)(which == 0 ? 1 : 0) * n_slabs + i) * nt2 + (long long)row * n_tot;
            C acc = czero<C>();
            for (int j = lane; j < n_tot; j += 32) acc = cfma(Mrow[j], lp[(long long)j * R + r], acc);
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane == 0) {
                const long long e = (long long)i * vec + (long long)row * R + r;
                if (which == 0) phi[e] = a_first[e] - acc;  // mu_i
                else lam[e] = a_last[e] - acc;              // lambda_i
            }
        }
        grid_barrier(bar, gridDim.x, err);
    }
    for (int i = n_slabs - 2; i >= 1; --i) {
        const C* pn = phi + (long long)(i + 1) * vec;
        for (long long task = gw; task < vec; task += nw) {
            const int row = (int)(task / R), r = (int)(task % R);
            const C* Mrow = iface + (2LL * n_slabs + i) * nt2 + (long long)row * n_tot;
            C acc = czero<C>();
            for (int j = lane; j < n_tot; j += 32) acc = cfma(Mrow[j], pn[(long long)j * R + r], acc);
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane == 0) {
                const long long e = (long long)i * vec + (long long)row * R + r;
                phi[e] = phi[e] - acc;
            }
        }
        grid_barrier(bar, gridDim.x, err);
    }
}

// ---------------------------------------------------------------- host helpers
template <typename T>
size_t thomas_smem(const lss_ctx* c, int RC) {
    int gmax = 0, cmax = 0, wmax = 0;
    for (const auto& s : c->slabs) {
        gmax = std::max(gmax, s.w * s.ldw);
        cmax = std::max(cmax, s.cstride);
        wmax = std::max(wmax, s.w);
    }
    return sizeof(cx<T>) * ((size_t)kStages * (gmax + cmax) + 2 * (size_t)wmax * RC);
}

int wmax_of(const lss_ctx* c) {
    int w = 0;
    for (const auto& s : c->slabs) w = std::max(w, s.w);
    return w;
}

template <typename T, int MODE>
int launch_thomas(lss_ctx* c, ThomasArgs<cx<T>> A, dim3 grid, cudaStream_t s) {
    const size_t sh = thomas_smem<T>(c, A.RC);
    static size_t configured = 0;
    if (sh > configured) {
        cudaError_t e = cudaFuncSetAttribute(thomas_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sh, 48 * 1024));
        if (e) return lss_check_cuda(c, e, "thomas attribute");
        configured = sh;
    }
    const int cat = MODE == TH_A ? LSS_PROF_SLAB_A : MODE == TH_IFACE ? LSS_PROF_IFACE : LSS_PROF_SLAB_E;
    ProfScope ps(c, s, cat, 1);
    thomas_kernel<T, MODE><<<grid, kSolveThreads, sh, s>>>(A);
    return lss_check_cuda(c, cudaGetLastError(), "thomas launch");
}

template <typename T>
ThomasArgs<cx<T>> base_args(lss_ctx* c) {
    ThomasArgs<cx<T>> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = c->n_slabs;
    A.n_tot = c->n_tot;
    A.n = c->n;
    A.b = c->b;
    A.coef = (const cx<T>*)c->coef;
    A.fac = (const cx<T>*)c->fac;
    A.err = c->d_err;
    return A;
}

int rhs_per_cta(int R) { return R >= 8 ? 8 : R; }

template <typename T>
int factor_impl(lss_ctx* c, cudaStream_t s) {
    using C = cx<T>;
    const int w = wmax_of(c);
    const size_t sh = sizeof(C) * ((size_t)w * 2 * w + 2 * (size_t)w * w + w);
    cudaError_t e =
        cudaFuncSetAttribute(factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(sh, 48 * 1024));
    if (e) return lss_check_cuda(c, e, "factor attribute");
    {
        ProfScope ps(c, s, LSS_PROF_FACTOR, 1);
        factor_kernel<T><<<c->n_slabs, 256, sh, s>>>(c->d_slabs, (const C*)c->coef, (C*)c->fac, c->n_tot, c->d_err);
    }
    int rc = lss_check_cuda(c, cudaGetLastError(), "factor launch");
    if (rc) return rc;
    if (c->n_slabs == 1) return LSS_OK;
    // interface maps: n_tot coupling columns per slab and side, in chunks that fit the scratch
    const int RC = 8;
    const long long zstride = (long long)c->n_tot * w * RC;
    const int chunks = (c->n_tot + RC - 1) / RC;
    const size_t budget = (size_t)1 << 30;
    int per = (int)std::max<long long>(1, (long long)(budget / (zstride * sizeof(C))) / (2LL * c->n_slabs));
    per = std::min(per, chunks);
    rc = lss_grow(c, &c->z_buf, &c->z_cap, (size_t)zstride * sizeof(C) * 2 * c->n_slabs * per);
    if (rc) return rc;
    for (int c0 = 0; c0 < chunks; c0 += per) {
        ThomasArgs<C> A = base_args<T>(c);
        A.iface = (C*)c->iface;
        A.zbuf = (C*)c->z_buf;
        A.zstride = zstride;
        A.RC = RC;
        A.R = c->n_tot;
        A.col0 = c0 * RC;
        const int ny = std::min(per, chunks - c0);
        rc = launch_thomas<T, TH_IFACE>(c, A, dim3(c->n_slabs, ny, 2), s);
        if (rc) return rc;
    }
    return LSS_OK;
}

template <typename T>
int recur_grid(lss_ctx* c) {
    static int cached = 0;
    if (!cached) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, recur_kernel<T>, 256, 0);
        cached = std::max(1, per) * c->num_sms;
    }
    return cached;
}

template <typename T>
int sweep_impl(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s) {
    using C = cx<T>;
    const long long nt2 = (long long)c->n_tot * c->n_tot;
    int rc = lss_grow(c, &c->f_buf, &c->f_cap, (size_t)R * nt2 * sizeof(C));
    if (rc) return rc;
    const long long vec = (long long)c->n_tot * R;
    rc = lss_grow(c, &c->side_buf, &c->side_cap, 4 * (size_t)c->n_slabs * vec * sizeof(C));
    if (rc) return rc;
    const int RC = rhs_per_cta(R);
    const int ny = (R + RC - 1) / RC;
    const long long zstride = (long long)c->n_tot * wmax_of(c) * RC;
    rc = lss_grow(c, &c->z_buf, &c->z_cap, (size_t)zstride * sizeof(C) * c->n_slabs * ny);
    if (rc) return rc;
    rc = lss_sparsify(c, r, c->f_buf, R, s);
    if (rc) return rc;
    C* side = (C*)c->side_buf;
    C* a_first = side;
    C* a_last = side + c->n_slabs * vec;
    C* lam = side + 2 * c->n_slabs * vec;
    C* phi = side + 3 * c->n_slabs * vec;
    ThomasArgs<C> A = base_args<T>(c);
    A.f = (const C*)c->f_buf;
    A.a_first = a_first;
    A.a_last = a_last;
    A.lam = lam;
    A.phi = phi;
    A.y = y;
    A.zbuf = (C*)c->z_buf;
    A.zstride = zstride;
    A.R = R;
    A.RC = RC;
    if (c->n_slabs > 1) {
        rc = launch_thomas<T, TH_A>(c, A, dim3(c->n_slabs, ny, 1), s);
        if (rc) return rc;
        int nb = recur_grid<T>(c);
        const long long tasks = 2 * vec;
        nb = (int)std::min<long long>(nb, std::max<long long>(1, (tasks + 7) / 8));
        int ns = c->n_slabs, nt = c->n_tot;
        const C* ifc = (const C*)c->iface;
        const C* af = a_first;
        const C* al = a_last;
        unsigned* bar = c->d_bar;
        int* err = c->d_err;
        void* args[] = {&ns, &nt, &R, &ifc, &af, &al, &lam, &phi, &bar, &err};
        ProfScope ps(c, s, LSS_PROF_RECUR, 1);
        cudaError_t e = cudaLaunchCooperativeKernel((void*)recur_kernel<T>, dim3(nb), dim3(256), args, 0, s);
        if (e) return lss_check_cuda(c, e, "recurrence launch");
    }
    return launch_thomas<T, TH_E>(c, A, dim3(c->n_slabs, ny, 1), s);
}

template <typename T>
int slab_apply_impl(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s) {
    using C = cx<T>;
    const int RC = rhs_per_cta(R);
    const int ny = (R + RC - 1) / RC;
    const long long zstride = (long long)c->n_tot * wmax_of(c) * RC;
    int rc = lss_grow(c, &c->z_buf, &c->z_cap, (size_t)zstride * sizeof(C) * ny);
    if (rc) return rc;
    ThomasArgs<C> A = base_args<T>(c);
    A.v_in = v;
    A.w_out = w;
    A.test_slab = slab;
    A.zbuf = (C*)c->z_buf;
    A.zstride = zstride;
    A.R = R;
    A.RC = RC;
    return launch_thomas<T, TH_TEST>(c, A, dim3(1, ny, 1), s);
}

}  // namespace

int lss_factor_slabs(lss_ctx* c, cudaStream_t s) {
    return c->prec == LSS_FP64 ? factor_impl<double>(c, s) : factor_impl<float>(c, s);
}

int lss_sweep(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s) {
    return c->prec == LSS_FP64 ? sweep_impl<double>(c, r, y, R, s) : sweep_impl<float>(c, r, y, R, s);
}

int lss_slab_apply(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s) {
    return c->prec == LSS_FP64 ? slab_apply_impl<double>(c, slab, v, w, R, s)
                               : slab_apply_impl<float>(c, slab, v, w, R, s);
}

// ---------------------------------------------------------------- fixed-scratch slab operator
// lss_apply_slab_noalloc: the slab operator of lss_apply_slab with its
// forward-elimination scratch in a fixed device array instead of the context's
// growable workspace, so that the call never reaches the device allocator.
namespace {

constexpr size_t kFixedScratchBytes = size_t(8) << 20;   // 8 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_fixed_mu;
void* g_fixed_ptr[kMaxDevices] = {};

// Device address of g_fixed_scratch for the current device.  In host code the
// symbol names a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.
int fixed_scratch(lss_ctx* c, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return lss_check_cuda(c, e, "noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return lss_fail(c, LSS_ERR_UNSUPPORTED, "noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_fixed_mu);
    if (!g_fixed_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fixed_scratch);
        if (e || !p) return lss_check_cuda(c, e ? e : cudaErrorInvalidSymbol, "noalloc: cudaGetSymbolAddress");
        g_fixed_ptr[dev] = p;
    }
    *out = g_fixed_ptr[dev];
    return LSS_OK;
}

template <typename T>
int slab_apply_fixed_impl(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s) {
    using C = cx<T>;
    const int RC = rhs_per_cta(R);
    const int ny = (R + RC - 1) / RC;
    const long long zstride = (long long)c->n_tot * wmax_of(c) * RC;
    const size_t need = (size_t)zstride * sizeof(C) * ny;
    if (need > kFixedScratchBytes)
        return lss_fail(c, LSS_ERR_UNSUPPORTED,
                        "apply_slab_noalloc: needs " + std::to_string(need) + " bytes of scratch, the fixed scratch holds " +
                            std::to_string(kFixedScratchBytes) + " (use fewer right-hand sides per call)");
    void* scratch = nullptr;
    int rc = fixed_scratch(c, &scratch);
    if (rc) return rc;
    // The forward pass writes every scratch entry before the backward pass reads
    // it, so nothing has to start at zero and no clearing is needed.
    ThomasArgs<C> A = base_args<T>(c);
    A.v_in = v;
    A.w_out = w;
    A.test_slab = slab;
    A.zbuf = (C*)scratch;
    A.zstride = zstride;
    A.R = R;
    A.RC = RC;
    const size_t sh = thomas_smem<T>(c, RC);
    cudaError_t e = cudaFuncSetAttribute(thomas_kernel<T, TH_TEST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(sh, 48 * 1024));
    if (e) return lss_check_cuda(c, e, "noalloc attribute");
    thomas_kernel<T, TH_TEST><<<dim3(1, ny, 1), kSolveThreads, sh, s>>>(A);
    return lss_check_cuda(c, cudaGetLastError(), "noalloc launch");
}

}  // namespace

extern "C" int lss_apply_slab_noalloc(lss_ctx* c, int slab, const void* v_dev, void* w_dev, int R, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!v_dev || !w_dev || R < 1 || slab < 0 || slab >= c->n_slabs)
        return lss_fail(c, LSS_ERR_ARG, "apply_slab_noalloc: bad arguments");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "apply_slab_noalloc before lss_factor");
    cudaStream_t s = (cudaStream_t)stream;
    return c->prec == LSS_FP64 ? slab_apply_fixed_impl<double>(c, slab, (const double2*)v_dev, (double2*)w_dev, R, s)
                               : slab_apply_fixed_impl<float>(c, slab, (const double2*)v_dev, (double2*)w_dev, R, s);
}
