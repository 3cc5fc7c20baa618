// Sweeping factorization (Sec. 2.3-2.4, Algorithms 1 and 2).
//
// Each slab subproblem S_i (Eq. Hwv_approx) is block tridiagonal along x2 with
// w x w blocks (w layers of the slab): A_k (coupling dk = 0), C_k (dk = -1),
// B_k (dk = +1), each tridiagonal in the layer index.  It is factored by block
// Gaussian elimination, D_0 = A_0, D_k = A_k - C_k D_{k-1}^{-1} B_{k-1}, with
// partial pivoting inside each D_k (Gauss-Jordan), storing G_k = D_k^{-1}.
// Per block row k the slab keeps one contiguous record: G_k transposed
// (element (p, a) at a*ldw + p) followed by the row's stencil coefficients, so
// a solve streams one record per step with a single bulk copy.
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

#include <cooperative_groups.h>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

constexpr int kStages = 3;      // TMA ring depth of the generic multi-RHS solve
constexpr int kSolveThreads = 128;

// ---------------------------------------------------------------- factorization
// One thread per column of the augmented block [D_k | I] (2w <= 64 columns) and
// NR threads splitting the rows of each column (NR = 1 for FP32, NR = 4 for
// FP64 to use all four sub-partitions).  The Schur update
// D_k = A_k - C_k (G_{k-1} B_{k-1}) is computed column by column by the thread
// owning the column; Gauss-Jordan with partial pivoting needs two barriers per
// pivot.  Writes the block-row records (G_k^T, then the coefficient row).
template <typename T, int NR>
__global__ void __launch_bounds__(64 * NR) factor_kernel(const SlabDev* __restrict__ slabs,
                                                         const cx<T>* __restrict__ coef, cx<T>* __restrict__ rec,
                                                         int n_tot, int* err) {
    using C = cx<T>;
    const SlabDev sd = slabs[blockIdx.x];
    const int w = sd.w, ldw = sd.ldw;
    constexpr int LD = 65;                        // column stride of M (column-major, padded)
    extern __shared__ __align__(128) unsigned char smraw_f[];
    C* M = reinterpret_cast<C*>(smraw_f);         // column q at M + q*LD, rows 0..w-1
    C* Gp = M + 64 * LD;                          // G_{k-1}, column-major, stride LD
    C* X = Gp + 32 * LD;                          // G_{k-1} B_{k-1}, column-major
    __shared__ int piv_row;
    __shared__ C piv_inv;
    const int q = threadIdx.x % 64, h = threadIdx.x / 64;
    const bool colq = q < 2 * w;
    const C* cf = coef + sd.coef_off;
    C* Rr = rec + sd.fac_off;
    const C zero = czero<C>();
    C* Mq = M + q * LD;
    for (int k = 0; k < n_tot; ++k) {
        const C* ck = cf + (long long)k * sd.cstride;
        C* Rk = Rr + (long long)k * sd.rsz;
        for (int e = threadIdx.x; e < sd.cstride; e += blockDim.x) Rk[w * ldw + e] = ck[e];
        if (colq && q < w) {
            // column q of X = G_{k-1} B_{k-1}
            C b0 = zero, b1 = zero, b2 = zero;   // B_{k-1}[a][q], a = q-1, q, q+1
            if (k > 0) {
                const C* cp = cf + (long long)(k - 1) * sd.cstride;
                if (q > 0) b0 = cp[(q - 1) * 9 + 2 * 3 + 2];
                b1 = cp[q * 9 + 1 * 3 + 2];
                if (q + 1 < w) b2 = cp[(q + 1) * 9 + 0 * 3 + 2];
            }
            C* Xq = X + q * LD;
            const C* G0 = Gp + (q > 0 ? q - 1 : 0) * LD;
            const C* G1 = Gp + q * LD;
            const C* G2 = Gp + (q + 1 < w ? q + 1 : q) * LD;
#pragma unroll 4
            for (int p = h; p < w; p += NR) {
                C x = zero;
                if (k > 0) {
                    x = cfma(G1[p], b1, x);
                    if (q > 0) x = cfma(G0[p], b0, x);
                    if (q + 1 < w) x = cfma(G2[p], b2, x);
                }
                Xq[p] = x;
            }
        }
        if (NR > 1) __syncthreads();
        if (colq) {
            const C* Xq = X + q * LD;
#pragma unroll 4
            for (int p = h; p < w; p += NR) {
                C v = zero;
                if (q < w) {
                    const int d = q - p;
                    if (d >= -1 && d <= 1) v = ck[p * 9 + (d + 1) * 3 + 1];
                    if (k > 0) {
                        const C* cr = ck + p * 9;
                        if (p > 0) v = v - cr[0] * Xq[p - 1];
                        v = v - cr[3] * Xq[p];
                        if (p + 1 < w) v = v - cr[6] * Xq[p + 1];
                    }
                } else if (q - w == p) {
                    v.x = T(1);
                }
                Mq[p] = v;
            }
        }
        __syncthreads();
        for (int j = 0; j < w; ++j) {
            if (threadIdx.x < 32) {
                const int i = j + threadIdx.x;
                T val = (i < w) ? cabs2(M[j * LD + i]) : T(-1);
                int best = i;
                for (int off = 16; off > 0; off >>= 1) {
                    const T ov = __shfl_down_sync(0xffffffffu, val, off);
                    const int ob = __shfl_down_sync(0xffffffffu, best, off);
                    if (ov > val || (ov == val && ob < best)) { val = ov; best = ob; }
                }
                if (threadIdx.x == 0) {
                    piv_row = best;
                    C pv = M[j * LD + best];
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
            // rows j and pr are swapped and row j scaled in every column q > j;
            // columns <= j are never read again, so they are left as they are
            const int pr = piv_row;
            C a = zero, mj = zero;
            if (colq && q > j) {
                a = Mq[j];
                mj = Mq[pr] * piv_inv;
            }
            if (NR > 1) __syncthreads();
            if (colq && q > j) {
                const C* Mj = M + j * LD;
                const C mpj = Mj[j];                  // entry (pr, j) after the swap
#pragma unroll 4
                for (int i = h; i < w; i += NR) {
                    const C mij = Mj[i];
                    const C cur = Mq[i];
                    C nv;
                    if (i == j) nv = mj;
                    else if (i == pr) nv = a - mpj * mj;
                    else nv = cur - mij * mj;
                    Mq[i] = nv;
                }
            }
            __syncthreads();
        }
        // G_k = right half; column a of G is column w + a of M
        if (colq && q >= w) {
            const int a = q - w;
            for (int p = h; p < ldw; p += NR) {
                const C v = (p < w) ? Mq[p] : zero;
                Rk[a * ldw + p] = v;
                if (p < w) Gp[a * LD + p] = v;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- generic multi-RHS slab solve
template <typename C>
struct SolveArgs {
    const SlabDev* slabs;
    int n_slabs, n_tot, n, b;
    const C* rec;
    const double2* v_in;   // R x (layers of D_i) x n_tot
    double2* w_out;
    int slab;
    C* zbuf;               // forward-elimination scratch
    long long zstride;     // per CTA
    int R, RC;             // total RHS, RHS per CTA
    int* err;
};

// One CTA solves S_i x = [0_aux; v] for RC right-hand sides and writes the
// D_i part (T~_i v): forward elimination z_k = G_k (b_k - C_k z_{k-1}), back
// substitution x_k = z_k - G_k B_k x_{k+1}.  Block-row records stream through
// a TMA ring; the 2 n_tot - 1 block rows are visited as one sequence.
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) solve_kernel(SolveArgs<cx<T>> A) {
    using C = cx<T>;
    const int i = A.slab;
    const SlabDev sd = A.slabs[i];
    const int w = sd.w, ldw = sd.ldw, K = A.n_tot, rsz = sd.rsz, gsz = w * ldw;
    const int r0 = blockIdx.y * A.RC;
    const int rc = min(A.RC, A.R - r0);
    if (rc <= 0) return;
    const int RC = A.RC;
    extern __shared__ __align__(128) unsigned char smraw_s[];
    C* Rs = reinterpret_cast<C*>(smraw_s);   // kStages x rsz
    C* v = Rs + kStages * rsz;               // w x RC
    C* zp = v + w * RC;                      // w x RC
    __shared__ __align__(8) uint64_t bar[kStages];
    const C* Rg = A.rec + sd.fac_off;
    C* Z = A.zbuf + (long long)blockIdx.y * A.zstride;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int outs = w * rc;
    int TP = 1;
    while (TP < 32 && outs * TP * 2 <= nth) TP <<= 1;
    const int ostep = nth / TP;
    const int nseq = 2 * K - 1;
    const unsigned rbytes = (unsigned)(rsz * sizeof(C));
    auto kk_of = [K](int pos) { return pos < K ? pos : 2 * K - 2 - pos; };
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int pos = 0; pos < kStages && pos < nseq; ++pos) {
            mbar_expect_tx(&bar[pos], rbytes);
            tma_load_1d(Rs + pos * rsz, Rg + (long long)kk_of(pos) * rsz, rbytes, &bar[pos]);
        }
    bool ok = true;
    for (int pos = 0; pos < nseq; ++pos) {
        const int st = pos % kStages;
        const int k = kk_of(pos);
        if (!mbar_wait(&bar[st], (pos / kStages) & 1, A.err)) ok = false;
        if (!__syncthreads_and(ok)) break;
        const C* Gk = Rs + st * rsz;
        const C* ck = Gk + gsz;
        const bool fwd = pos < K;
        for (int idx = tid; idx < w * rc; idx += nth) {
            const int p = idx % w, rr = idx / w;
            C bv = czero<C>();
            if (fwd) {
                if (p >= sd.na)
                    bv = to_c<C>(A.v_in[((long long)(r0 + rr) * sd.nl + (p - sd.na)) * K + k]);
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
                for (int a = kq; a < w; a += TP) acc = cfma(Gk[a * ldw + op], v[a * RC + orr], acc);
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
                if ((!fwd || k == K - 1) && op >= sd.na)
                    A.w_out[((long long)(r0 + orr) * sd.nl + (op - sd.na)) * K + k] = to_d(x);
            }
        }
        __syncthreads();
        if (tid == 0 && pos + kStages < nseq) {
            mbar_expect_tx(&bar[st], rbytes);
            tma_load_1d(Rs + st * rsz, Rg + (long long)kk_of(pos + kStages) * rsz, rbytes, &bar[st]);
        }
    }
    if (!ok && tid == 0) {
        // a wait expired: give the copies already issued a bounded chance to land
        const long long t0 = clock64();
        while (clock64() - t0 < 2000000ll) __nanosleep(1000);
    }
}

// ---------------------------------------------------------------- interface maps
// Work item = (slab i, side, chunk of kIfNC columns j): solve S_i X = H e_j for
// the chunk (side 0: the coupling H_{[i,i-1]} into D_i's first layer; side 1:
// H_{[i,i+1]} into its last layer) and keep only the rows needed: side 0 ->
// Lambda_i (last layer) and Gamma_i (first layer), side 1 -> Phi_i (first
// layer).  Column j's right-hand side is zero above block row j-1, so the
// forward pass of a chunk starts there.  Per block row the update is a
// (w x w) x (w x kIfNC) product: threads own (column, rows p = rg, rg + 4, ...)
// and G_k is read as a warp broadcast.  Persistent grid over the items.
constexpr int kIfNC = 64;
constexpr int kIfThreads = 256;
constexpr int kIfRows = 8;      // rows per thread: w <= 32 over 4 row groups
constexpr int kIfStages = 4;

template <typename T>
__global__ void __launch_bounds__(kIfThreads) iface_kernel(const SlabDev* __restrict__ slabs, int n_slabs,
                                                           int n_tot, const cx<T>* __restrict__ rec,
                                                           cx<T>* __restrict__ iface, cx<T>* __restrict__ zbuf,
                                                           long long zstride, int nitems, int rmax, int* err) {
    using C = cx<T>;
    const int nch = (n_tot + kIfNC - 1) / kIfNC;
    const int K = n_tot;
    const long long nt2 = (long long)n_tot * n_tot;
    extern __shared__ __align__(128) unsigned char smi[];
    C* Rs = reinterpret_cast<C*>(smi);           // kIfStages x rmax
    C* V = Rs + kIfStages * rmax;                // 32 x kIfNC
    C* zp = V + 32 * kIfNC;                      // 32 x kIfNC
    __shared__ __align__(8) uint64_t bar[kIfStages];
    const int tid = threadIdx.x;
    const int c = tid % kIfNC, rg = tid / kIfNC;
    C* Z = zbuf + (long long)blockIdx.x * zstride;
    if (tid == 0) {
        for (int st = 0; st < kIfStages; ++st) mbar_init(&bar[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned gpos = 0;   // running TMA sequence position (continues across items)
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        int t = item, i, side;
        const int n0 = (n_slabs - 1) * nch;
        if (t < n0) { i = 1 + t / nch; side = 0; t %= nch; }
        else { t -= n0; i = 1 + t / nch; side = 1; t %= nch; }
        const SlabDev sd = slabs[i];
        const int w = sd.w, ldw = sd.ldw, gsz = w * ldw, rsz = sd.rsz, na = sd.na;
        const int j0 = t * kIfNC;
        const int ncol = min(kIfNC, n_tot - j0);
        const int k0 = max(0, j0 - 1);
        const int nf = K - k0, nseq = nf + K - 1;
        const int pin = side == 0 ? na : w - 1;
        const C* Rg = rec + sd.fac_off;
        const unsigned rbytes = (unsigned)(rsz * sizeof(C));
        // forward: k = k0 + pos (pos < nf); backward: k = K - 2 - (pos - nf)
        auto kseq = [&](int pos) { return pos < nf ? k0 + pos : K - 2 - (pos - nf); };
        if (tid == 0)
            for (int pp = 0; pp < kIfStages && pp < nseq; ++pp) {
                const unsigned gp = gpos + pp;
                const int st = gp % kIfStages;
                mbar_expect_tx(&bar[st], rbytes);
                tma_load_1d(Rs + st * rmax, Rg + (long long)kseq(pp) * rsz, rbytes, &bar[st]);
            }
        for (int pos = 0; pos < nseq; ++pos) {
            const unsigned gp = gpos + pos;
            const int st = gp % kIfStages;
            const int k = kseq(pos);
            const bool fwd = pos < nf;
            // scratch values of this block row, loaded before the wait and the product
            C zold[kIfRows];
#pragma unroll
            for (int r = 0; r < kIfRows; ++r) {
                const int p = rg + 4 * r;
                zold[r] = (!fwd && p < w && k >= k0) ? Z[((long long)(k - k0) * w + p) * kIfNC + c] : czero<C>();
            }
            if (!mbar_wait(&bar[st], (gp / kIfStages) & 1, err)) ok = false;
            if (!__syncthreads_and(ok)) break;
            const C* Gk = Rs + st * rmax;
            const C* ck = Gk + gsz;
            // V = b_k - C_k z_{k-1} (forward) or B_k x_{k+1} (backward)
            for (int idx = tid; idx < w * kIfNC; idx += kIfThreads) {
                const int p = idx / kIfNC, cc = idx % kIfNC;
                C v = czero<C>();
                if (cc < ncol) {
                    const C* cp = ck + p * 9;
                    if (fwd) {
                        const int dk = j0 + cc - k;
                        if (p == pin && dk >= -1 && dk <= 1) v = cp[(side == 0 ? 0 : 6) + dk + 1];
                        if (k > k0) {
                            if (p > 0) v = v - cp[0] * zp[(p - 1) * kIfNC + cc];
                            v = v - cp[3] * zp[p * kIfNC + cc];
                            if (p + 1 < w) v = v - cp[6] * zp[(p + 1) * kIfNC + cc];
                        }
                    } else {
                        if (p > 0) v = cfma(cp[2], zp[(p - 1) * kIfNC + cc], v);
                        v = cfma(cp[5], zp[p * kIfNC + cc], v);
                        if (p + 1 < w) v = cfma(cp[8], zp[(p + 1) * kIfNC + cc], v);
                    }
                }
                V[p * kIfNC + cc] = v;
            }
            __syncthreads();
            C acc[kIfRows];
#pragma unroll
            for (int r = 0; r < kIfRows; ++r) acc[r] = czero<C>();
            for (int a = 0; a < w; ++a) {
                const C v = V[a * kIfNC + c];
#pragma unroll
                for (int r = 0; r < kIfRows; ++r) {
                    const int p = rg + 4 * r;
                    if (p < w) acc[r] = cfma(Gk[a * ldw + p], v, acc[r]);
                }
            }
            __syncthreads();   // every thread has read zp (through V), V and the stage
            if (tid == 0 && pos + kIfStages < nseq) {
                const unsigned gn = gpos + pos + kIfStages;
                const int sn = gn % kIfStages;
                mbar_expect_tx(&bar[sn], rbytes);
                tma_load_1d(Rs + sn * rmax, Rg + (long long)kseq(pos + kIfStages) * rsz, rbytes, &bar[sn]);
            }
#pragma unroll
            for (int r = 0; r < kIfRows; ++r) {
                const int p = rg + 4 * r;
                if (p >= w) continue;
                C x;
                if (fwd) {
                    x = acc[r];
                    Z[((long long)(k - k0) * w + p) * kIfNC + c] = x;
                } else {
                    x = zold[r] - acc[r];
                }
                zp[p * kIfNC + c] = x;
                if ((!fwd || k == K - 1) && c < ncol) {
                    const long long e = (long long)k * n_tot + j0 + c;
                    if (side == 0) {
                        if (p == w - 1) iface[(0LL * n_slabs + i) * nt2 + e] = x;
                        if (p == na) iface[(1LL * n_slabs + i) * nt2 + e] = x;
                    } else if (p == na) {
                        iface[(2LL * n_slabs + i) * nt2 + e] = x;
                    }
                }
            }
            __syncthreads();
        }
        gpos += nseq;
    }
    if (!ok && tid == 0) {
        const long long t0 = clock64();
        while (clock64() - t0 < 2000000ll) __nanosleep(1000);
    }
}

// ---------------------------------------------------------------- sweep slab solves
enum SweepMode { SW_A = 0, SW_E = 1 };

template <typename C>
struct SweepArgs {
    const SlabDev* slabs;
    int n_slabs, n_tot, n, b, R;
    const C* rec;
    const C* f;            // R x n_tot^2, x2 index slowest
    C* a_first;            // [slab][k][R]
    C* a_last;
    const C* lam;          // [slab][k][R]
    const C* phi;
    double2* y;            // R x n^2
    C* zbuf;               // forward-elimination scratch when it does not fit in shared memory
    long long zstride;
    int* err;
};

template <typename C>
__device__ __forceinline__ C shfl_c(C v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
    return v;
}
template <typename C>
__device__ __forceinline__ C shfl_up_c(C v) {
    v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
    v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
    return v;
}
template <typename C>
__device__ __forceinline__ C shfl_down_c(C v) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
    v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
    return v;
}

// Warp-specialised slab solve, one right-hand side per CTA.  Warp NQ is the
// producer: it streams the block-row records into a ring of S stages, RB
// consecutive records per stage in one TMA bulk copy (the forward pass walks
// k upwards, the backward pass downwards; both read contiguous record runs).
// Warps 0..NQ-1 consume.  Lane l owns row p = l mod 16 of the block row when
// 2w <= 32 (the two half-warps then split the columns of G_k), else row p = l;
// the NQ warps split the columns further and sum their slices through shared
// memory (NQ > 1, FP64).  Neighbours along the layer index come from shuffles
// and v is broadcast through a per-warp shared-memory vector.  The slab's
// right-hand-side block and the coupling vectors lambda_{i-1}, phi_{i+1} are
// preloaded into shared memory, so the consumers issue no global loads; a
// consumer warp releases a stage by arriving on its "empty" mbarrier.  The
// forward-elimination values stay in shared memory when they fit (zsmem),
// else they go to global scratch and are fetched one step ahead.
template <typename T, int MODE, int NQ, int S, int RB>
__global__ void __launch_bounds__(32 * (NQ + 1)) sweep_kernel(SweepArgs<cx<T>> A, int zsmem, int rmax, int nlmax) {
    using C = cx<T>;
    const int i = blockIdx.x, r = blockIdx.y;
    const SlabDev sd = A.slabs[i];
    const int w = sd.w, ldw = sd.ldw, K = A.n_tot, na = sd.na, nl = sd.nl, gsz = w * ldw, rsz = sd.rsz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    extern __shared__ __align__(128) unsigned char sm2[];
    C* stage0 = reinterpret_cast<C*>(sm2);         // S x RB x rmax
    C* part = stage0 + S * RB * rmax;              // 2 x NQ x 32 partial dots
    C* vsb = part + 2 * NQ * 32;                   // NQ x 32 broadcast vectors
    C* fs = vsb + NQ * 32;                         // K x nlmax: right-hand side of D_i
    C* ls = fs + (long long)K * nlmax;             // K: lambda_{i-1}
    C* ps = ls + K;                                // K: phi_{i+1}
    C* Zs = ps + K;                                // K x w (zsmem)
    __shared__ __align__(8) uint64_t full[S], empty[S], pbar[2];
    const int nfc = (K + RB - 1) / RB, nbc = (K - 1 + RB - 1) / RB, nch = nfc + nbc;
    // chunk ci -> first record lo and record count; forward chunks ascend, backward descend
    auto chunk = [&](int ci, int& lo, int& cnt) {
        if (ci < nfc) {
            lo = ci * RB;
            cnt = min(RB, K - lo);
        } else {
            const int hi = K - 2 - (ci - nfc) * RB;
            lo = max(0, hi - RB + 1);
            cnt = hi - lo + 1;
        }
    };
    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], NQ);
        }
        mbar_init(&pbar[0], NQ);
        mbar_init(&pbar[1], NQ);
        fence_mbar_init();
    }
    // preload f on D_i (and the coupling vectors) once
    {
        const long long nt2 = (long long)K * K;
        const C* fr = A.f + (long long)r * nt2 + (sd.s + A.b);
        for (int e = threadIdx.x; e < K * nl; e += blockDim.x) {
            const int k = e / nl, j = e % nl;
            fs[k * nlmax + j] = fr[(long long)k * K + j];
        }
        if (MODE == SW_E) {
            const long long vec = (long long)K * A.R;
            for (int k = threadIdx.x; k < K; k += blockDim.x) {
                ls[k] = i > 0 ? A.lam[(long long)(i - 1) * vec + (long long)k * A.R + r] : czero<C>();
                ps[k] = i < A.n_slabs - 1 ? A.phi[(long long)(i + 1) * vec + (long long)k * A.R + r] : czero<C>();
            }
        }
    }
    __syncthreads();
    if (warp == NQ) {
        // ---------------- producer: one bulk copy of RB records per stage
        if (lane == 0) {
            const C* Rg = A.rec + sd.fac_off;
            for (int ci = 0; ci < nch; ++ci) {
                const int st = ci % S;
                if (ci >= S && !mbar_wait(&empty[st], ((ci / S) - 1) & 1, A.err)) break;
                int lo, cnt;
                chunk(ci, lo, cnt);
                const unsigned bytes = (unsigned)(cnt * rsz * sizeof(C));
                mbar_expect_tx(&full[st], bytes);
                tma_load_1d(stage0 + st * RB * rmax, Rg + (long long)lo * rsz, bytes, &full[st]);
            }
        }
        return;
    }
    // ---------------- consumers
    const int q = warp;
    const int H = (2 * w <= 32) ? 2 : 1;            // half-warps splitting the columns
    const int half = H == 2 ? lane >> 4 : 0;
    const int p = H == 2 ? lane & 15 : lane;
    const int gw = H == 2 ? 16 : 32;                // shuffle group width
    const bool act = p < w;
    const bool lead = act && q == 0 && half == 0;   // writes scratch and outputs
    C* Z = zsmem ? Zs : A.zbuf + ((long long)i * gridDim.y + r) * A.zstride;
    const int nsl = NQ * H;                         // column slices
    const int per = (w + nsl - 1) / nsl;
    const int sl = q * H + half;
    const int a0 = min(w, sl * per), a1 = min(w, a0 + per);
    C* vs = vsb + q * 32;
    C z = czero<C>();
    C znext = czero<C>();   // Z[k] for the next backward step (global scratch only)
    int pos = 0;            // global step index
    bool ok = true;
    for (int ci = 0; ci < nch && ok; ++ci) {
        const int st = ci % S;
        int lo, cnt;
        chunk(ci, lo, cnt);
        const bool fwd = ci < nfc;
        if (!mbar_wait(&full[st], (ci / S) & 1, A.err)) break;
        const C* stg = stage0 + st * RB * rmax;
        for (int jj = 0; jj < cnt; ++jj, ++pos) {
            const int k = fwd ? lo + jj : lo + cnt - 1 - jj;
            const C zold = znext;
            if (!zsmem && !fwd && act && half == 0) {
                const int kn = k - 1;   // next backward block row
                if (kn >= 0) znext = Z[(long long)kn * w + p];
            } else if (!zsmem && fwd && k == K - 1 && act && half == 0 && K >= 2) {
                znext = Z[(long long)(K - 2) * w + p];
            }
            const C* Gk = stg + (k - lo) * rsz;
            const C* ck = Gk + gsz;
            C zm, zpl;
            zm.x = __shfl_up_sync(0xffffffffu, z.x, 1, gw);
            zm.y = __shfl_up_sync(0xffffffffu, z.y, 1, gw);
            zpl.x = __shfl_down_sync(0xffffffffu, z.x, 1, gw);
            zpl.y = __shfl_down_sync(0xffffffffu, z.y, 1, gw);
            C v = czero<C>();
            if (act) {
                const C* cp = ck + p * 9;
                if (fwd) {
                    if (p >= na) v = fs[k * nlmax + (p - na)];
                    if (MODE == SW_E) {
                        if (p == na && i > 0)
                            for (int dk = -1; dk <= 1; ++dk) {
                                const int kk = k + dk;
                                if (kk >= 0 && kk < K) v = v - cp[0 * 3 + dk + 1] * ls[kk];
                            }
                        if (p == w - 1 && i < A.n_slabs - 1)
                            for (int dk = -1; dk <= 1; ++dk) {
                                const int kk = k + dk;
                                if (kk >= 0 && kk < K) v = v - cp[2 * 3 + dk + 1] * ps[kk];
                            }
                    }
                    if (k > 0) {
                        if (p > 0) v = v - cp[0] * zm;
                        v = v - cp[3] * z;
                        if (p + 1 < w) v = v - cp[6] * zpl;
                    }
                } else {
                    if (p > 0) v = cfma(cp[2], zm, v);
                    v = cfma(cp[5], z, v);
                    if (p + 1 < w) v = cfma(cp[8], zpl, v);
                }
            }
            __syncwarp();
            if (half == 0) vs[lane] = v;
            __syncwarp();
            C acc0 = czero<C>(), acc1 = czero<C>();
            if (act) {
                int a = a0;
                for (; a + 1 < a1; a += 2) {
                    acc0 = cfma(Gk[a * ldw + p], vs[a], acc0);
                    acc1 = cfma(Gk[(a + 1) * ldw + p], vs[a + 1], acc1);
                }
                if (a < a1) acc0 = cfma(Gk[a * ldw + p], vs[a], acc0);
            }
            C acc = acc0 + acc1;
            if (H == 2) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
            }
            if (NQ > 1) {
                // sum the column slices of the warps: a bounded mbarrier exchange, two buffers
                C* pb = part + (pos & 1) * NQ * 32;
                pb[q * 32 + lane] = acc;
                __syncwarp();
                if (lane == 0) mbar_arrive(&pbar[pos & 1]);
                if (!mbar_wait(&pbar[pos & 1], (pos >> 1) & 1, A.err)) { ok = false; break; }
                acc = pb[lane];
                for (int qq = 1; qq < NQ; ++qq) acc = acc + pb[qq * 32 + lane];
            }
            if (fwd) {
                z = acc;
                if (lead) Z[(long long)k * w + p] = z;
            } else {
                const C zk = zsmem ? Z[(long long)k * w + p] : zold;
                z = act ? zk - acc : czero<C>();
                if (!zsmem) {   // the half-warp / other warps take the value from the lead lane
                    z.x = __shfl_sync(0xffffffffu, z.x, p, 32);
                    z.y = __shfl_sync(0xffffffffu, z.y, p, 32);
                }
            }
            if (lead && (!fwd || k == K - 1)) {
                if (MODE == SW_A) {
                    const long long e = ((long long)i * K + k) * A.R + r;
                    if (p == na) A.a_first[e] = z;
                    if (p == w - 1) A.a_last[e] = z;
                } else if (p >= na) {
                    const int x1 = sd.s + (p - na), i2 = k - A.b;
                    if (x1 >= 1 && x1 <= A.n && i2 >= 1 && i2 <= A.n)
                        A.y[(long long)r * A.n * A.n + (long long)(x1 - 1) * A.n + (i2 - 1)] = to_d(z);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);   // stage no longer read by this warp
    }
}

// ---------------------------------------------------------------- interface recurrences
// Grid-wide version (cooperative launch, bounded grid barrier): the fallback
// when the vectors or rows do not fit the cluster kernel below.
template <typename T>
__global__ void __launch_bounds__(256) recur_grid_kernel(int n_slabs, int n_tot, int R,
                                                         const cx<T>* __restrict__ iface,
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

// Interface recurrences inside one thread-block cluster.  Each CTA owns a
// block of rows of the n_tot x n_tot maps and keeps the current vector
// (lambda_{i-1} or phi_{i+1}) replicated in its shared memory; new entries are
// stored into every CTA's copy through distributed shared memory, and the
// cluster barrier closes each step.  Each warp owns at most RW (row, rhs)
// tasks and holds their matrix rows for the next step in registers (CW
// entries per lane), loaded before the barrier so the load latency overlaps
// it.  mu_i (not on the chain) is computed for all slabs in one parallel phase
// between the two chains.
template <typename T, int RW, int CW, int NT>
__global__ void __launch_bounds__(NT) recur_cluster_kernel(int n_slabs, int n_tot, int R,
                                                           const cx<T>* __restrict__ iface,
                                                           const cx<T>* __restrict__ a_first,
                                                           const cx<T>* __restrict__ a_last, cx<T>* lam,
                                                           cx<T>* phi) {
    using C = cx<T>;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smr[];
    C* vb = reinterpret_cast<C*>(smr);   // 2 x n_tot x R
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const int rows_per = (n_tot + CL - 1) / CL;
    const int r0 = min(n_tot, cr * rows_per), r1 = min(n_tot, r0 + rows_per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int ntask = (r1 - r0) * R;
    C Mr[RW][CW];

    auto load_rows = [&](const C* M) {
#pragma unroll
        for (int t = 0; t < RW; ++t) {
            const int task = warp + t * nw;
            const int row = r0 + (task < ntask ? task / R : 0);
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) {
                const int j = lane + 32 * cc;
                Mr[t][cc] = (task < ntask && j < n_tot) ? M[(long long)row * n_tot + j] : czero<C>();
            }
        }
    };
    auto step = [&](const C* base_vec, long long out_off, C* gout, int cur) {
#pragma unroll
        for (int t = 0; t < RW; ++t) {
            const int task = warp + t * nw;
            if (task >= ntask) break;
            const int row = r0 + task / R, rr = task % R;
            const C* x = vb + cur * vec + rr;
            C acc = czero<C>();
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) {
                const int j = lane + 32 * cc;
                if (j < n_tot) acc = cfma(Mr[t][cc], x[(long long)j * R], acc);
            }
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane < CL) {
                const long long e = (long long)row * R + rr;
                const C val = base_vec[out_off + e] - acc;
                if (lane == 0) gout[out_off + e] = val;
                C* dst = cl.map_shared_rank(vb, lane);
                dst[(cur ^ 1) * vec + e] = val;
            }
        }
    };

    for (long long e = threadIdx.x; e < vec; e += blockDim.x) vb[e] = a_last[e];
    for (long long e = (long long)r0 * R + threadIdx.x; e < (long long)r1 * R; e += blockDim.x) lam[e] = a_last[e];
    if (n_slabs - 2 >= 1) load_rows(iface + (0LL * n_slabs + 1) * nt2);
    __syncthreads();
    int cur = 0;
    // lambda chain: lambda_i = last(a_i) - Lambda_i lambda_{i-1}
    for (int i = 1; i <= n_slabs - 2; ++i) {
        step(a_last, (long long)i * vec, lam, cur);
        if (i + 1 <= n_slabs - 2) load_rows(iface + (0LL * n_slabs + i + 1) * nt2);
        cl.sync();
        cur ^= 1;
    }
    // mu_i = first(a_i) - Gamma_i lambda_{i-1} for every slab, in parallel
    {
        const long long total = (long long)(n_slabs - 1) * vec;
        for (long long t = (long long)cr * nw + warp; t < total; t += (long long)CL * nw) {
            const int i = 1 + (int)(t / vec);
            const long long rem = t % vec;
            const int row = (int)(rem / R), rr = (int)(rem % R);
            const C* lp = (i == 1 ? a_last : lam + (long long)(i - 1) * vec) + rr;
            const C* Mrow = iface + (1LL * n_slabs + i) * nt2 + (long long)row * n_tot;
            C acc = czero<C>();
#pragma unroll 4
            for (int j = lane; j < n_tot; j += 32) acc = cfma(Mrow[j], lp[(long long)j * R], acc);
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane == 0) phi[(long long)i * vec + rem] = a_first[(long long)i * vec + rem] - acc;
        }
    }
    if (n_slabs - 2 >= 1) load_rows(iface + (2LL * n_slabs + n_slabs - 2) * nt2);
    cl.sync();
    // phi chain: phi_{l-1} = mu_{l-1}, phi_i = mu_i - Phi_i phi_{i+1}
    for (long long e = threadIdx.x; e < vec; e += blockDim.x) vb[cur * vec + e] = phi[(long long)(n_slabs - 1) * vec + e];
    __syncthreads();
    for (int i = n_slabs - 2; i >= 1; --i) {
        step(phi, (long long)i * vec, phi, cur);
        if (i - 1 >= 1) load_rows(iface + (2LL * n_slabs + i - 1) * nt2);
        cl.sync();
        cur ^= 1;
    }
}

// ---------------------------------------------------------------- host helpers
int wmax_of(const lss_ctx* c) {
    int w = 0;
    for (const auto& s : c->slabs) w = std::max(w, s.w);
    return w;
}
int rmax_of(const lss_ctx* c) {
    int r = 0;
    for (const auto& s : c->slabs) r = std::max(r, s.rsz);
    return r;
}
int nlmax_of(const lss_ctx* c) {
    int r = 0;
    for (const auto& s : c->slabs) r = std::max(r, s.nl);
    return r;
}

template <typename F>
int set_smem(lss_ctx* c, F kern, size_t sh, size_t* configured) {
    if (sh <= *configured) return LSS_OK;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(sh, 48 * 1024));
    if (e) return lss_check_cuda(c, e, "shared memory attribute");
    *configured = sh;
    return LSS_OK;
}

int rhs_per_cta(int R) { return R >= 8 ? 8 : R; }

template <typename T>
int factor_impl(lss_ctx* c, cudaStream_t s) {
    using C = cx<T>;
    constexpr int NR = sizeof(T) == 8 ? 4 : 8;
    const int w = wmax_of(c);
    const size_t sh = sizeof(C) * (size_t)(64 + 32 + 32) * 65;
    static size_t cfg_f = 0;
    int rc = set_smem(c, factor_kernel<T, NR>, sh, &cfg_f);
    if (rc) return rc;
    {
        ProfScope ps(c, s, LSS_PROF_FACTOR, 1);
        factor_kernel<T, NR><<<c->n_slabs, 64 * NR, sh, s>>>(c->d_slabs, (const C*)c->coef, (C*)c->fac, c->n_tot,
                                                            c->d_err);
    }
    rc = lss_check_cuda(c, cudaGetLastError(), "factor launch");
    if (rc) return rc;
    if (c->n_slabs == 1) return LSS_OK;
    // interface maps: persistent grid over (slab, side, column chunk) items
    const int nch = (c->n_tot + kIfNC - 1) / kIfNC;
    const int nitems = (c->n_slabs - 1) * nch + std::max(0, c->n_slabs - 2) * nch;
    const int grid = std::min(nitems, 2 * c->num_sms);
    const long long zstride = (long long)c->n_tot * w * kIfNC;
    rc = lss_grow(c, &c->z_buf, &c->z_cap, (size_t)zstride * sizeof(C) * grid);
    if (rc) return rc;
    const int rmax = (rmax_of(c) + 1) & ~1;
    const size_t shi = sizeof(C) * ((size_t)kIfStages * rmax + 2 * 32 * (size_t)kIfNC);
    static size_t cfg_i = 0;
    rc = set_smem(c, iface_kernel<T>, shi, &cfg_i);
    if (rc) return rc;
    ProfScope ps(c, s, LSS_PROF_IFACE, 1);
    iface_kernel<T><<<grid, kIfThreads, shi, s>>>(c->d_slabs, c->n_slabs, c->n_tot, (const C*)c->fac, (C*)c->iface,
                                                  (C*)c->z_buf, zstride, nitems, rmax, c->d_err);
    return lss_check_cuda(c, cudaGetLastError(), "iface launch");
}

template <typename T, int MODE>
int launch_sweep(lss_ctx* c, SweepArgs<cx<T>> A, cudaStream_t s) {
    using C = cx<T>;
    constexpr int NQ = sizeof(T) == 8 ? 4 : 1;
    constexpr int S = sizeof(T) == 8 ? 2 : 3;
    constexpr int RB = 4;
    const int rmax = (rmax_of(c) + 1) & ~1, nlmax = nlmax_of(c), wmax = wmax_of(c);
    const size_t base = sizeof(C) * ((size_t)S * RB * rmax + 3 * NQ * 32 + (size_t)c->n_tot * nlmax +
                                     2 * (size_t)c->n_tot);
    const size_t zb = sizeof(C) * (size_t)c->n_tot * wmax;
    const int zsmem = (base + zb <= (size_t)220 * 1024) ? 1 : 0;
    const size_t sh = base + (zsmem ? zb : 0);
    if (sh > (size_t)225 * 1024) return lss_fail(c, LSS_ERR_UNSUPPORTED, "slab solve does not fit in shared memory");
    static size_t cfg = 0;
    int rc = set_smem(c, sweep_kernel<T, MODE, NQ, S, RB>, sh, &cfg);
    if (rc) return rc;
    if (!zsmem) {
        A.zstride = (long long)c->n_tot * wmax;
        rc = lss_grow(c, &c->z_buf, &c->z_cap, (size_t)A.zstride * sizeof(C) * c->n_slabs * A.R);
        if (rc) return rc;
        A.zbuf = (C*)c->z_buf;
    }
    ProfScope ps(c, s, MODE == SW_A ? LSS_PROF_SLAB_A : LSS_PROF_SLAB_E, 1);
    sweep_kernel<T, MODE, NQ, S, RB><<<dim3(c->n_slabs, A.R), 32 * (NQ + 1), sh, s>>>(A, zsmem, rmax, nlmax);
    return lss_check_cuda(c, cudaGetLastError(), "sweep launch");
}

// Cluster size for the recurrence kernel: 16 CTAs when the GPU can co-schedule
// them (non-portable size), else 8.  Returns LSS_ERR_UNSUPPORTED when a warp
// would own more rows than its prefetch registers hold, so the caller uses the
// grid kernel.
template <typename T, int RW, int CW, int NT>
int launch_recur_cluster_cfg(lss_ctx* c, cx<T>* lam, cx<T>* phi, const cx<T>* a_first, const cx<T>* a_last, int R,
                             cudaStream_t s) {
    const size_t sh = 2 * (size_t)c->n_tot * R * sizeof(cx<T>);
    static int cl_size = 0;
    static size_t configured = 0;
    auto kern = recur_cluster_kernel<T, RW, CW, NT>;
    if (sh > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sh, 48 * 1024));
        if (!e) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e) return lss_check_cuda(c, e, "recurrence attribute");
        configured = sh;
        cl_size = 0;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = std::max<size_t>(sh, 16);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!cl_size) {
        for (int cand : {16, 8}) {
            attr[0].val.clusterDim.x = cand;
            cfg.gridDim = dim3(cand);
            int nclusters = 0;
            cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, (void*)kern, &cfg);
            if (!e && nclusters > 0) { cl_size = cand; break; }
            cudaGetLastError();
        }
        if (!cl_size) return LSS_ERR_UNSUPPORTED;
    }
    const int rows_per = (c->n_tot + cl_size - 1) / cl_size;
    if ((rows_per * R + NT / 32 - 1) / (NT / 32) > RW || c->n_tot > 32 * CW) return LSS_ERR_UNSUPPORTED;
    attr[0].val.clusterDim.x = cl_size;
    cfg.gridDim = dim3(cl_size);
    int ns = c->n_slabs, nt = c->n_tot;
    const cx<T>* ifc = (const cx<T>*)c->iface;
    ProfScope ps(c, s, LSS_PROF_RECUR, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ns, nt, R, ifc, a_first, a_last, lam, phi);
    return lss_check_cuda(c, e, "recurrence cluster launch");
}

template <typename T>
int launch_recur(lss_ctx* c, cx<T>* lam, cx<T>* phi, const cx<T>* a_first, const cx<T>* a_last, int R,
                 cudaStream_t s) {
    using C = cx<T>;
    const size_t sh = 2 * (size_t)c->n_tot * R * sizeof(C);
    int rc = LSS_ERR_UNSUPPORTED;
    if (sh <= (size_t)160 * 1024) {
        if constexpr (sizeof(T) == 4) {
            if (c->n_tot <= 384) rc = launch_recur_cluster_cfg<T, 3, 12, 256>(c, lam, phi, a_first, a_last, R, s);
            else rc = launch_recur_cluster_cfg<T, 3, 20, 384>(c, lam, phi, a_first, a_last, R, s);
        } else {
            rc = launch_recur_cluster_cfg<T, 3, 9, 256>(c, lam, phi, a_first, a_last, R, s);
        }
    }
    if (rc != LSS_ERR_UNSUPPORTED) return rc;
    static int grid = 0;
    if (!grid) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, recur_grid_kernel<T>, 256, 0);
        grid = std::max(1, per) * c->num_sms;
    }
    const long long vec = (long long)c->n_tot * R;
    int nb = (int)std::min<long long>(grid, std::max<long long>(1, (2 * vec + 7) / 8));
    int ns = c->n_slabs, nt = c->n_tot;
    const C* ifc = (const C*)c->iface;
    unsigned* bar = c->d_bar;
    int* err = c->d_err;
    void* args[] = {&ns, &nt, &R, &ifc, (void*)&a_first, (void*)&a_last, &lam, &phi, &bar, &err};
    ProfScope ps(c, s, LSS_PROF_RECUR, 1);
    cudaError_t e = cudaLaunchCooperativeKernel((void*)recur_grid_kernel<T>, dim3(nb), dim3(256), args, 0, s);
    return lss_check_cuda(c, e, "recurrence launch");
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
    rc = lss_sparsify(c, r, c->f_buf, R, s);
    if (rc) return rc;
    C* side = (C*)c->side_buf;
    SweepArgs<C> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = c->n_slabs;
    A.n_tot = c->n_tot;
    A.n = c->n;
    A.b = c->b;
    A.R = R;
    A.rec = (const C*)c->fac;
    A.f = (const C*)c->f_buf;
    A.a_first = side;
    A.a_last = side + c->n_slabs * vec;
    C* lam = side + 2 * c->n_slabs * vec;
    C* phi = side + 3 * c->n_slabs * vec;
    A.lam = lam;
    A.phi = phi;
    A.y = y;
    A.err = c->d_err;
    if (c->n_slabs > 1) {
        rc = launch_sweep<T, SW_A>(c, A, s);
        if (rc) return rc;
        rc = launch_recur<T>(c, lam, phi, A.a_first, A.a_last, R, s);
        if (rc) return rc;
    }
    return launch_sweep<T, SW_E>(c, A, s);
}

template <typename T>
int slab_apply_impl(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s) {
    using C = cx<T>;
    const int RC = rhs_per_cta(R);
    const int ny = (R + RC - 1) / RC;
    const long long zstride = (long long)c->n_tot * wmax_of(c) * RC;
    int rc = lss_grow(c, &c->z_buf, &c->z_cap, (size_t)zstride * sizeof(C) * ny);
    if (rc) return rc;
    SolveArgs<C> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = c->n_slabs;
    A.n_tot = c->n_tot;
    A.n = c->n;
    A.b = c->b;
    A.rec = (const C*)c->fac;
    A.v_in = v;
    A.w_out = w;
    A.slab = slab;
    A.zbuf = (C*)c->z_buf;
    A.zstride = zstride;
    A.R = R;
    A.RC = RC;
    A.err = c->d_err;
    const size_t sh = sizeof(C) * ((size_t)kStages * ((rmax_of(c) + 1) & ~1) + 2 * (size_t)wmax_of(c) * RC);
    static size_t cfg = 0;
    rc = set_smem(c, solve_kernel<T>, sh, &cfg);
    if (rc) return rc;
    ProfScope ps(c, s, LSS_PROF_SLAB_E, 1);
    solve_kernel<T><<<dim3(1, ny), kSolveThreads, sh, s>>>(A);
    return lss_check_cuda(c, cudaGetLastError(), "slab solve launch");
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
    SolveArgs<C> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = c->n_slabs;
    A.n_tot = c->n_tot;
    A.n = c->n;
    A.b = c->b;
    A.rec = (const C*)c->fac;
    A.v_in = v;
    A.w_out = w;
    A.slab = slab;
    A.zbuf = (C*)scratch;
    A.zstride = zstride;
    A.R = R;
    A.RC = RC;
    A.err = c->d_err;
    const size_t sh = sizeof(C) * ((size_t)kStages * ((rmax_of(c) + 1) & ~1) + 2 * (size_t)wmax_of(c) * RC);
    cudaError_t e = cudaFuncSetAttribute(solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(sh, 48 * 1024));
    if (e) return lss_check_cuda(c, e, "noalloc attribute");
    solve_kernel<T><<<dim3(1, ny), kSolveThreads, sh, s>>>(A);
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
