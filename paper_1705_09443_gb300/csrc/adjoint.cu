// Transposed preconditioner P^T = Q^T Sweep^T E^T for the adjoint solve
// A^T mu = rhs (A^T = I + omega^2 M K, the bilinear transpose of Eq. LS_d_c).
//
// Sweep^T.  Algorithm 2 applies S = (I + T N_U)^{-1} (I + T N_L)^{-1} T with
// T = blockdiag(T~_i), N_L[i,i-1] = H_{[i,i-1]}, N_U[i,i+1] = H_{[i,i+1]}, so
// S^T = T^T (I + N_L^T T^T)^{-1} (I + N_U^T T^T)^{-1}: a forward pass
// w_i = v_i - H_{[i-1,i]}^T last(T~_{i-1}^T w_{i-1}) and a backward pass
// x_i = T~_i^T (w_i - H_{[i+1,i]}^T first(x_{i+1})).  It is evaluated
// slab-parallel like the forward sweep: with a'_i = T~_i^T v_i and the maps
//   Lambda'_i = last-layer rows of T~_i^T H_{[i-1,i]}^T,  Gamma'_i = first-layer
//   rows of the same,  Phi'_i = first-layer rows of T~_i^T H_{[i+1,i]}^T,
// the coupling values obey the same three recurrences (lambda', mu', phi') and
// x_i = T~_i^T (v_i - H_{[i-1,i]}^T lambda'_{i-1} - H_{[i+1,i]}^T phi'_{i+1}).
//
// T~_i^T.  Cyclic reduction of S_i^T with the stored factors of S_i: the
// reduced blocks of S_i^T are the transposes of S_i's (lower coupling of row k:
// B_{k-1}^T, upper: C_{k+1}^T, diagonal D_k^T), so
//   level 0 forward:  y_o = D_o^{-T} b_o,  b_e -= B_{e-1}^T y_{e-1} + C_{e+1}^T y_{e+1}
//                     (level 0's stencil bands of the odd rows);
//   level l >= 1:     b_e -= (D^{-1}B)_{e-1}^T b_{e-1} + (D^{-1}C)_{e+1}^T b_{e+1},
//                     then y_o = D_o^{-T} b_o;
//   top:              x_0 = D_top^{-T} b_0;
//   backward:         x_o = y_o - D_o^{-T} (B_{o-1}^T x_{o-1} + C_{o+1}^T x_{o+1})
//                     (B, C of the even rows: level-l blocks, or level 0's bands).
// Blocks are read straight from global memory (the adjoint path is not the
// timed one); one CTA per slab and right-hand side, the vectors in shared
// memory when they fit.
#include <algorithm>
#include <string>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

constexpr int kTThreads = 256;
enum TMode { T_A = 0, T_E = 1, T_IF = 2 };

__device__ __forceinline__ double2 cfnma_t(double2 a, double2 b, double2 acc) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfnma_t(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(-a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}

template <typename C>
struct TArgs {
    const SlabDev* slabs;
    int n_slabs, n_tot, n, b, R;
    const C* fac;
    const C* coef;
    const double2* y;        // T_A, T_E: R x n^2 vectors on I (E^T puts them on the grid)
    C* a_first;              // T_A outputs, [slab][k][R]
    C* a_last;
    const C* lam;            // T_E couplings lambda', phi', [slab][k][R]
    const C* phi;
    C* X;                    // T_E output: R x n_tot^2 grid, x2 index slowest
    C* maps;                 // T_IF output: Lambda', Gamma', Phi', each n_slabs x n_tot^2
    int nch;                 // T_IF: columns per slab side (n_tot)
    C* bg;                   // right-hand sides in global memory when bsm == 0
    long long bstride;
    int bsm;
};

// acc (+/-)= (M^T x)[p] = sum_a M(a, p) x[a]; M column-major G x G, zero-padded.
template <typename C, int G, bool SUB>
__device__ __forceinline__ C mvt(const C* __restrict__ M, int p, const C* x, C acc) {
    const C* col = M + p * G;
    C acc2 = czero<C>();
#pragma unroll
    for (int a = 0; a < G; a += 2) {
        if (SUB) {
            acc = cfnma_t(col[a], x[a], acc);
            acc2 = cfnma_t(col[a + 1], x[a + 1], acc2);
        } else {
            acc = cfma(col[a], x[a], acc);
            acc2 = cfma(col[a + 1], x[a + 1], acc2);
        }
    }
    return acc + acc2;
}

// acc (+/-)= (Band^T x)[p] = sum_da band[(da + 1) G + (p - da)] x[p - da]
// (band[(da + 1) G + a] couples layer a to layer a + da).
template <typename C, int G, bool SUB>
__device__ __forceinline__ C bandt(const C* __restrict__ band, int p, const C* x, C acc) {
#pragma unroll
    for (int da = -1; da <= 1; ++da) {
        const int a = p - da;
        if (a < 0 || a >= G) continue;
        const C cv = band[(da + 1) * G + a];
        acc = SUB ? cfnma_t(cv, x[a], acc) : cfma(cv, x[a], acc);
    }
    return acc;
}

template <typename T, int MODE, int G>
__device__ void t_body(const TArgs<cx<T>>& A, const SlabDev& sd, int i, int r, int side, int j, cx<T>* b) {
    using C = cx<T>;
    const int K = A.n_tot, w = sd.w, na = sd.na, bs = sd.bs;
    const int L = cr_levels(K);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
    constexpr int GPW = 32 / G;
    const int grp = lane / G, p = lane % G;
    const int ngrp = nw * GPW;
    const C* F = A.fac + sd.fac_off;
    const C* cf = A.coef + sd.coef_off;
    const C* t0 = F + cr_t0_off(K, bs);
    const int Kh = (K + 1) / 2;   // even rows come first among the bands
    __shared__ C tgs[kTThreads];
    C* tg = tgs + (warp * GPW + grp) * G;
    auto row = [&](int k) { return b + (long long)k * G; };
    const long long nt2 = (long long)K * K;

    // ---- right-hand side
    for (int e = tid; e < K * G; e += nth) {
        const int k = e / G, pp = e % G;
        C v = czero<C>();
        if (pp < w) {
            if (MODE == T_A || MODE == T_E) {
                const int x1 = sd.s + (pp - na), i2 = k - A.b;
                if (pp >= na && x1 >= 1 && x1 <= A.n && i2 >= 1 && i2 <= A.n)
                    v = to_c<C>(A.y[(long long)r * A.n * A.n + (long long)(x1 - 1) * A.n + (i2 - 1)]);
                if (MODE == T_E) {
                    const long long vec = (long long)K * A.R;
                    if (pp == na && i > 0) {   // - H_{[i-1,i]}^T lambda'_{i-1}
                        const SlabDev sl = A.slabs[i - 1];
                        const C* cl = A.coef + sl.coef_off;
                        for (int d = -1; d <= 1; ++d) {
                            const int kk = k - d;
                            if (kk >= 0 && kk < K)
                                v = cfnma_t(cl[(long long)kk * sl.cstride + (sl.w - 1) * 9 + 6 + d + 1],
                                            A.lam[(long long)(i - 1) * vec + (long long)kk * A.R + r], v);
                        }
                    }
                    if (pp == w - 1 && i < A.n_slabs - 1) {   // - H_{[i+1,i]}^T phi'_{i+1}
                        const SlabDev sr = A.slabs[i + 1];
                        const C* crt = A.coef + sr.coef_off;
                        for (int d = -1; d <= 1; ++d) {
                            const int kk = k - d;
                            if (kk >= 0 && kk < K)
                                v = cfnma_t(crt[(long long)kk * sr.cstride + sr.na * 9 + d + 1],
                                            A.phi[(long long)(i + 1) * vec + (long long)kk * A.R + r], v);
                        }
                    }
                }
            } else {
                const int d = k - j;
                if (d >= -1 && d <= 1) {
                    if (side == 0 && pp == na) {   // column j of H_{[i-1,i]}^T
                        const SlabDev sl = A.slabs[i - 1];
                        v = A.coef[sl.coef_off + (long long)j * sl.cstride + (sl.w - 1) * 9 + 6 + d + 1];
                    } else if (side == 1 && pp == w - 1) {   // column j of H_{[i+1,i]}^T
                        const SlabDev sr = A.slabs[i + 1];
                        v = A.coef[sr.coef_off + (long long)j * sr.cstride + sr.na * 9 + d + 1];
                    }
                }
            }
        }
        b[e] = v;
    }
    __syncthreads();

    // ---- forward reduction
    for (int l = 0; l < L; ++l) {
        const CrLevelOffs lv = cr_level(K, l);
        const int Kl = lv.K;
        if (l == 0) {
            for (int t0i = warp * GPW; t0i < Kl / 2; t0i += ngrp) {   // y_o = D_o^{-T} b_o
                const int t = t0i + grp;
                const bool on = t < Kl / 2;
                C* x = row(on ? 2 * t + 1 : 0);
                C acc = czero<C>();
                if (on) acc = mvt<C, G, false>(F + (lv.dinv + t) * bs, p, x, acc);
                __syncwarp();
                if (on) x[p] = acc;
                __syncwarp();
            }
            __syncthreads();
            for (int t = warp * GPW + grp; t < (Kl + 1) / 2; t += ngrp) {
                const int e = 2 * t;
                C acc = row(e)[p];
                if (e >= 1) acc = bandt<C, G, true>(t0 + ((long long)Kh + ((e - 1) >> 1)) * 6 * G + 3 * G, p, row(e - 1), acc);
                if (e + 1 < Kl) acc = bandt<C, G, true>(t0 + ((long long)Kh + ((e + 1) >> 1)) * 6 * G, p, row(e + 1), acc);
                row(e)[p] = acc;
            }
            __syncthreads();
        } else {
            for (int t = warp * GPW + grp; t < (Kl + 1) / 2; t += ngrp) {
                const int e = 2 * t, k = e << l;
                C acc = row(k)[p];
                if (e >= 1) acc = mvt<C, G, true>(F + (lv.dcdb + 2LL * (t - 1) + 1) * bs, p, row((e - 1) << l), acc);
                if (e + 1 < Kl) acc = mvt<C, G, true>(F + (lv.dcdb + 2LL * t) * bs, p, row((e + 1) << l), acc);
                row(k)[p] = acc;
            }
            __syncthreads();
            for (int t0i = warp * GPW; t0i < Kl / 2; t0i += ngrp) {
                const int t = t0i + grp;
                const bool on = t < Kl / 2;
                C* x = row(on ? (2 * t + 1) << l : 0);
                C acc = czero<C>();
                if (on) acc = mvt<C, G, false>(F + (lv.dinv + t) * bs, p, x, acc);
                __syncwarp();
                if (on) x[p] = acc;
                __syncwarp();
            }
            __syncthreads();
        }
    }
    if (warp == 0) {
        C acc = czero<C>();
        if (grp == 0) acc = mvt<C, G, false>(F + cr_level(K, L).dinv * bs, p, row(0), acc);
        __syncwarp();
        if (grp == 0) row(0)[p] = acc;
    }
    __syncthreads();
    // ---- back substitution
    for (int l = L - 1; l >= 0; --l) {
        const CrLevelOffs lv = cr_level(K, l);
        const int Kl = lv.K;
        for (int t0i = warp * GPW; t0i < Kl / 2; t0i += ngrp) {
            const int t = t0i + grp;
            const bool on = t < Kl / 2;
            const int jr = 2 * t + 1, k = jr << l;
            C tv = czero<C>();
            if (on) {
                if (l == 0) {
                    tv = bandt<C, G, false>(t0 + (long long)t * 6 * G + 3 * G, p, row(k - 1), tv);
                    if (jr + 1 < Kl) tv = bandt<C, G, false>(t0 + (long long)(t + 1) * 6 * G, p, row(k + 1), tv);
                } else {
                    tv = mvt<C, G, false>(F + (lv.cbe + 2LL * t + 1) * bs, p, row((jr - 1) << l), tv);
                    if (jr + 1 < Kl) tv = mvt<C, G, false>(F + (lv.cbe + 2LL * (t + 1)) * bs, p, row((jr + 1) << l), tv);
                }
            }
            tg[p] = tv;
            __syncwarp();
            if (on) row(k)[p] = mvt<C, G, true>(F + (lv.dinv + t) * bs, p, tg, row(k)[p]);
            __syncwarp();
        }
        __syncthreads();
    }

    // ---- outputs
    if (MODE == T_A) {
        const long long base = (long long)i * K * A.R + r;
        for (int k = tid; k < K; k += nth) {
            A.a_first[base + (long long)k * A.R] = row(k)[na];
            A.a_last[base + (long long)k * A.R] = row(k)[w - 1];
        }
    } else if (MODE == T_E) {
        for (int e = tid; e < sd.nl * K; e += nth) {
            const int k = e % K, pp = na + e / K;
            A.X[(long long)r * nt2 + (long long)k * K + sd.s + A.b + (pp - na)] = row(k)[pp];
        }
    } else {
        const int ns = A.n_slabs;
        for (int k = tid; k < K; k += nth) {
            const long long o = (long long)k * K + j;
            if (side == 0) {
                A.maps[(0LL * ns + i) * nt2 + o] = row(k)[w - 1];
                A.maps[(1LL * ns + i) * nt2 + o] = row(k)[na];
            } else {
                A.maps[(2LL * ns + i) * nt2 + o] = row(k)[na];
            }
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kTThreads) cr_solve_t_kernel(TArgs<cx<T>> A) {
    using C = cx<T>;
    extern __shared__ __align__(16) unsigned char smt[];
    int i, r = 0, side = 0, j = 0;
    if (MODE == T_IF) {
        // blocks: side 0 for slabs 1..l-1, then side 1 for slabs 1..l-2; one column each
        int t = blockIdx.x;
        const int n0 = (A.n_slabs - 1) * A.nch;
        if (t < n0) { i = 1 + t / A.nch; j = t % A.nch; }
        else { t -= n0; side = 1; i = 1 + t / A.nch; j = t % A.nch; }
    } else {   // slab-major grid: a slab's right-hand sides share its factor stream in L2
        i = blockIdx.y;
        r = blockIdx.x;
    }
    const long long cta = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    C* b = A.bsm ? reinterpret_cast<C*>(smt) : A.bg + cta * A.bstride;
    const SlabDev sd = A.slabs[i];
    if (sd.w <= 16) t_body<T, MODE, 16>(A, sd, i, r, side, j, b);
    else t_body<T, MODE, 32>(A, sd, i, r, side, j, b);
}

int ldwmax(const lss_ctx* c) {
    int m = 0;
    for (const auto& s : c->slabs) m = std::max(m, s.ldw);
    return m;
}

template <typename T, int MODE>
int launch_t(lss_ctx* c, TArgs<cx<T>> A, dim3 grid, cudaStream_t s) {
    using C = cx<T>;
    const long long per = (long long)c->n_tot * ldwmax(c);
    const size_t bb = sizeof(C) * (size_t)per;
    A.bstride = per;
    A.bsm = bb <= (size_t)200 * 1024;
    const size_t sh = A.bsm ? bb : 0;
    if (!A.bsm) {
        int rc = lss_grow(c, &c->z_buf, &c->z_cap, bb * (size_t)grid.x * grid.y);
        if (rc) return rc;
        A.bg = (C*)c->z_buf;
    }
    std::unique_lock<std::mutex> lock(lss_config_mutex());
    long long& cfg = lss_dev_cache((const void*)cr_solve_t_kernel<T, MODE>, 0);
    if ((long long)sh > cfg) {
        cudaError_t e = cudaFuncSetAttribute(cr_solve_t_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sh, 48 * 1024));
        if (e) return lss_check_cuda(c, e, "transposed solve attribute");
        cfg = (long long)sh;
    }
    lock.unlock();
    cr_solve_t_kernel<T, MODE><<<grid, kTThreads, sh, s>>>(A);
    return lss_check_cuda(c, cudaGetLastError(), "transposed solve launch");
}

template <typename C>
TArgs<C> targs(lss_ctx* c, int R) {
    TArgs<C> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = c->n_slabs;
    A.n_tot = c->n_tot;
    A.n = c->n;
    A.b = c->b;
    A.R = R;
    A.fac = (const C*)c->fac;
    A.coef = (const C*)c->coef;
    return A;
}

// Maps of the transposed sweep, once per factorization.
template <typename T>
int build_maps_t(lss_ctx* c, cudaStream_t s) {
    using C = cx<T>;
    if (c->iface_t_valid || c->n_slabs == 1) return LSS_OK;
    // 64 bytes of slack for the recurrence's 16-byte aligned copy windows
    const size_t bytes = (size_t)3 * c->n_slabs * c->n_tot * c->n_tot * sizeof(C) + 64;
    if (!c->iface_t) {
        cudaError_t e = cudaMalloc(&c->iface_t, bytes);
        if (e) return lss_check_cuda(c, e, "transposed interface maps");
    }
    TArgs<C> A = targs<C>(c, 1);
    A.maps = (C*)c->iface_t;
    A.nch = c->n_tot;
    const int nitems = (c->n_slabs - 1) * c->n_tot + std::max(0, c->n_slabs - 2) * c->n_tot;
    ProfScope ps(c, s, LSS_PROF_IFACE, 1);
    int rc = launch_t<T, T_IF>(c, A, dim3(nitems), s);
    if (!rc) c->iface_t_valid = true;
    return rc;
}

template <typename T>
int sweep_t_impl(lss_ctx* c, const double2* y, double2* r, int R, cudaStream_t s) {
    using C = cx<T>;
    int rc = build_maps_t<T>(c, s);
    if (rc) return rc;
    const long long nt2 = (long long)c->n_tot * c->n_tot;
    const long long vec = (long long)c->n_tot * R;
    rc = lss_grow(c, &c->f_buf, &c->f_cap, (size_t)R * nt2 * sizeof(C));
    if (rc) return rc;
    rc = lss_grow(c, &c->side_buf, &c->side_cap, 4 * (size_t)c->n_slabs * vec * sizeof(C));
    if (rc) return rc;
    // Q^T reads X on the (n+2)^2 region only; slabs write every layer of their D_i
    C* side = (C*)c->side_buf;
    TArgs<C> A = targs<C>(c, R);
    A.y = y;
    A.a_first = side;
    A.a_last = side + c->n_slabs * vec;
    C* lam = side + 2 * c->n_slabs * vec;
    C* phi = side + 3 * c->n_slabs * vec;
    A.lam = lam;
    A.phi = phi;
    A.X = (C*)c->f_buf;
    const dim3 grid(R, c->n_slabs);
    if (c->n_slabs > 1) {
        {
            ProfScope ps(c, s, LSS_PROF_SLAB_A, 1);
            rc = launch_t<T, T_A>(c, A, grid, s);
        }
        if (rc) return rc;
        rc = lss_recurrences(c, c->iface_t, lam, phi, A.a_first, A.a_last, R, s);
        if (rc) return rc;
    }
    {
        ProfScope ps(c, s, LSS_PROF_SLAB_E, 1);
        rc = launch_t<T, T_E>(c, A, grid, s);
    }
    if (rc) return rc;
    return lss_sparsify_t(c, c->f_buf, r, R, s);
}

}  // namespace

int lss_sweep_t(lss_ctx* c, const double2* y, double2* r, int R, cudaStream_t s) {
    return c->prec == LSS_FP64 ? sweep_t_impl<double>(c, y, r, R, s) : sweep_t_impl<float>(c, y, r, R, s);
}

int lss_prepare_sweep_t(lss_ctx* c, cudaStream_t s) {
    return c->prec == LSS_FP64 ? build_maps_t<double>(c, s) : build_maps_t<float>(c, s);
}
