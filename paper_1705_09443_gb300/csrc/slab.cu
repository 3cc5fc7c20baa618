// Sweeping factorization (Sec. 2.3-2.4, Algorithms 1 and 2).
//
// Each slab subproblem S_i (Eq. Hwv_approx) is block tridiagonal along x2 with
// w x w blocks (w layers of the slab): A_k (coupling dk = 0), C_k (dk = -1),
// B_k (dk = +1), each tridiagonal in the layer index.  It is factored by block
// cyclic reduction along x2: at level l the odd rows are eliminated, which
// leaves the even rows coupled by
//   A'_e = A_e - C_e D_{e-1}^{-1} B_{e-1} - B_e D_{e+1}^{-1} C_{e+1},
//   C'_e = -C_e D_{e-1}^{-1} C_{e-1},  B'_e = -B_e D_{e+1}^{-1} B_{e+1},
// with D_o = A_o inverted by Gauss-Jordan with partial pivoting.  A solve is
//   forward:  y_o = D_o^{-1} b_o,  b_e <- b_e - C_e y_{e-1} - B_e y_{e+1},
//   top:      x_0 = D_top^{-1} b_0,
//   backward: x_o = y_o - D_o^{-1}C_o x_{o-1} - D_o^{-1}B_o x_{o+1}
//             (level 0: x_o = y_o - D_o^{-1} (C_o x_{o-1} + B_o x_{o+1}) with the
//             tridiagonal stencil bands),
// log2(n_tot) levels deep instead of n_tot sequential block steps; every row
// of a level is independent.  This is block Gaussian elimination in the
// odd-even order, so it gives the same T~_i as the sequential sweep of the
// block rows up to rounding.  The factors are stored in the order a solve
// reads them, and a solve streams them through shared memory with TMA bulk
// copies.
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
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"

namespace {

constexpr int kSolveThreads = 384;
constexpr size_t kSmemBudget = size_t(220) * 1024;

// acc - a*b
__device__ __forceinline__ double2 cfnma(double2 a, double2 b, double2 acc) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfnma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(-a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}


// ---------------------------------------------------------------- factorization
// Level 0's blocks from the stencil rows of the coefficient table (row p of
// block row k: entry (da + 1) * 3 + (dk + 1) couples layer p + da of row k + dk),
// dense in the work area (C_0 = B_{K-1} = 0), and the banded copy the solves read.
template <typename T>
__global__ void cr_build0_kernel(const SlabDev* __restrict__ slabs, const cx<T>* __restrict__ coef,
                                 cx<T>* __restrict__ work, cx<T>* __restrict__ fac, int K0) {
    using C = cx<T>;
    const SlabDev sd = slabs[blockIdx.y];
    const int k = blockIdx.x;
    const int w = sd.w, ldw = sd.ldw, bs = sd.bs;
    const C* ck = coef + sd.coef_off + (long long)k * sd.cstride;
    C* W = work + sd.work_off;
    C* Ab = W + (long long)k * bs;
    C* Cb = W + ((long long)K0 + 2LL * k) * bs;
    C* Bb = Cb + bs;
    for (int e = threadIdx.x; e < bs; e += blockDim.x) {
        const int q = e / ldw, p = e % ldw;   // element (p, q) at q * ldw + p
        C a = czero<C>(), cm = czero<C>(), cp = czero<C>();
        const int d = q - p;
        if (p < w && q < w && d >= -1 && d <= 1) {
            const C* r = ck + p * 9 + (d + 1) * 3;
            a = r[1];
            if (k > 0) cm = r[0];
            if (k + 1 < K0) cp = r[2];
        }
        Ab[e] = a;
        Cb[e] = cm;
        Bb[e] = cp;
    }
    const long long row = (k & 1) ? (K0 + 1) / 2 + k / 2 : k / 2;
    C* band = fac + sd.fac_off + cr_t0_off(K0, bs) + row * 6 * ldw;
    for (int e = threadIdx.x; e < 6 * ldw; e += blockDim.x) {
        const int bnd = e / ldw, p = e % ldw;
        const int da = bnd % 3 - 1, slot = bnd < 3 ? 0 : 2;
        C v = czero<C>();
        const bool has = bnd < 3 ? k > 0 : k + 1 < K0;
        if (p < w && p + da >= 0 && p + da < w && has) v = ck[p * 9 + (da + 1) * 3 + slot];
        band[e] = v;
    }
}

// Level 0's odd rows: A, C and B are tridiagonal in the layer index (the
// stencil couplings), so D^{-1} = A^{-1}, D^{-1}C and D^{-1}B come from one LU
// factorization of the tridiagonal A with partial pivoting (a row is exchanged
// with the next one when the subdiagonal entry is the larger; U then has a
// second superdiagonal) and 3w column solves: O(w^2) work instead of the O(w^3)
// of Gauss-Jordan.  One warp per odd row: lane 0 factors A into shared memory,
// every lane solves right-hand-side columns of [I | C | B] in registers.
constexpr int kGj0Warps = 4;

template <typename T>
struct Gt0Sm {
    cx<T> d[32], dl[32], du[32], du2[32];
    int piv[32];
};

template <typename T, int G>
__device__ void gj0_body(const SlabDev& sd, const cx<T>* __restrict__ coef, cx<T>* __restrict__ fac,
                         cx<T>* __restrict__ work, int K0, int o, Gt0Sm<T>& sm, int* err) {
    using C = cx<T>;
    const int lane = threadIdx.x & 31;
    const int w = sd.w, bs = G * G, na = sd.na;
    const int j = 2 * o + 1;
    const C* ck = coef + sd.coef_off + (long long)j * sd.cstride;   // row p at ck + 9p, entry (da+1)*3 + (dk+1)
    const bool hasB = j + 1 < K0;
    if (lane == 0) {
        for (int p = 0; p < w; ++p) {
            sm.d[p] = ck[p * 9 + 4];
            sm.du[p] = p + 1 < w ? ck[p * 9 + 7] : czero<C>();        // A(p, p+1)
            sm.dl[p] = p + 1 < w ? ck[(p + 1) * 9 + 1] : czero<C>();  // A(p+1, p)
            sm.du2[p] = czero<C>();
            sm.piv[p] = 0;
        }
        bool sing = false;
        for (int i = 0; i + 1 < w; ++i) {
            if (cabs2(sm.d[i]) >= cabs2(sm.dl[i])) {
                if (!(cabs2(sm.d[i]) > T(0))) { sing = true; sm.d[i] = czero<C>(); sm.d[i].x = T(1); }
                const C f = sm.dl[i] * crecip(sm.d[i]);
                sm.dl[i] = f;
                sm.d[i + 1] = cfnma(f, sm.du[i], sm.d[i + 1]);
            } else {
                const C f = sm.d[i] * crecip(sm.dl[i]);
                sm.d[i] = sm.dl[i];
                sm.dl[i] = f;
                const C t = sm.du[i];
                sm.du[i] = sm.d[i + 1];
                sm.d[i + 1] = cfnma(f, sm.d[i + 1], t);
                sm.piv[i] = 1;
                if (i + 2 < w) {
                    sm.du2[i] = sm.du[i + 1];
                    sm.du[i + 1] = mk(-f.x, -f.y) * sm.du[i + 1];
                }
            }
        }
        for (int i = 0; i < w; ++i) {
            if (!(cabs2(sm.d[i]) > T(0)) || !isfinite(cabs2(sm.d[i]))) { sing = true; sm.d[i] = czero<C>(); sm.d[i].x = T(1); }
            sm.d[i] = crecip(sm.d[i]);   // reciprocals of U's diagonal
        }
        if (sing) atomicOr(err, LSS_DERR_SINGULAR);
    }
    __syncwarp();
    C* Dout = fac + sd.fac_off + (cr_level(K0, 0).dinv + o) * bs;
    C* DCw = work + sd.work_off + (3LL * K0 + 2LL * o) * bs;
    C* P0 = fac + sd.fac_off + cr_p0_off(K0, bs, G) + 2LL * o * G;
    for (int q = lane; q < 3 * G; q += 32) {
        const int blk = q / G, a = q % G;   // block 0: D^{-1}, 1: D^{-1}C, 2: D^{-1}B; column a
        C* out = blk == 0 ? Dout + a * G : DCw + (blk - 1) * bs + a * G;
        C b[G];
#pragma unroll
        for (int p = 0; p < G; ++p) {
            C v = czero<C>();
            if (a < w && p < w) {
                if (blk == 0) {
                    if (p == a) v.x = T(1);
                } else if (p >= a - 1 && p <= a + 1 && (blk == 1 || hasB)) {
                    v = ck[p * 9 + (a - p + 1) * 3 + (blk == 1 ? 0 : 2)];   // C(p, a) or B(p, a)
                }
            }
            b[p] = v;
        }
        if (a < w) {
#pragma unroll
            for (int i = 0; i + 1 < G; ++i) {   // L, with the row exchanges
                if (i + 1 < w) {
                    if (sm.piv[i]) {
                        const C t = b[i];
                        b[i] = b[i + 1];
                        b[i + 1] = cfnma(sm.dl[i], b[i], t);
                    } else {
                        b[i + 1] = cfnma(sm.dl[i], b[i], b[i + 1]);
                    }
                }
            }
#pragma unroll
            for (int i = G - 1; i >= 0; --i) {   // U: diagonal, superdiagonal, second superdiagonal
                if (i < w) {
                    C v = b[i];
                    if (i + 1 < G && i + 1 < w) v = cfnma(sm.du[i], b[i + 1], v);
                    if (i + 2 < G && i + 2 < w) v = cfnma(sm.du2[i], b[i + 2], v);
                    b[i] = v * sm.d[i];
                }
            }
        }
        C v_first = czero<C>(), v_last = czero<C>();   // rows na and ll (selected, not indexed)
#pragma unroll
        for (int p = 0; p < G; ++p) {
            const C v = (a < w && p < w) ? b[p] : czero<C>();
            out[p] = v;
            if (p == na) v_first = v;
            if (p == sd.ll) v_last = v;
        }
        if (blk == 0) {   // rows na and ll (D_i's first and last layers) of D^{-1}, column a
            P0[a] = v_first;
            P0[G + a] = v_last;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kGj0Warps) cr_gj0_kernel(const SlabDev* __restrict__ slabs,
                                                                const cx<T>* __restrict__ coef,
                                                                cx<T>* __restrict__ fac, cx<T>* __restrict__ work,
                                                                int K0, int per_slab, int slab0, int n_slabs,
                                                                int* err) {
    __shared__ Gt0Sm<T> sm[kGj0Warps];
    const int warp = threadIdx.x >> 5;
    const int task = blockIdx.x * kGj0Warps + warp;
    if (task >= per_slab * n_slabs) return;   // the whole warp leaves
    const SlabDev sd = slabs[slab0 + task / per_slab];
    const int o = task % per_slab;
    if (sd.w <= 16) gj0_body<T, 16>(sd, coef, fac, work, K0, o, sm[warp], err);
    else gj0_body<T, 32>(sd, coef, fac, work, K0, o, sm[warp], err);
}

// Levels >= 1 of the factorization: a CTA per block row (a warp per row left
// each row's dependent elimination chain exposed; the levels with few rows
// and the wide slabs set the factorization time).
constexpr int kWideThreads = 256;

// Gauss-Jordan with partial pivoting (largest modulus in the column, lowest
// row on ties) on [A | I | C | B] for the odd rows of level l, giving D^{-1},
// D^{-1}C and D^{-1}B, or on [A | I] for the top row.  The augmented matrix
// sits row-major in shared memory (row stride rs); warp 0 picks the pivot,
// the threads swap and scale row jj column-wise, then thread (column q, row
// parity) eliminates every other row i = parity, parity+2, ...
template <typename T>
__global__ void __launch_bounds__(kWideThreads) cr_gjw_kernel(const SlabDev* __restrict__ slabs,
                                                             cx<T>* __restrict__ fac, cx<T>* __restrict__ work,
                                                             long long work_len, int K0, int l, int per_slab,
                                                             int slab0, int top, int rs, int* err) {
    using C = cx<T>;
    extern __shared__ __align__(16) unsigned char smw[];
    __shared__ int s_piv;
    const int tid = threadIdx.x, lane = tid & 31;
    const int task = blockIdx.x;
    const int si = slab0 + task / per_slab, o = task % per_slab;
    const SlabDev sd = slabs[si];
    const int w = sd.w, ldw = sd.ldw, bs = sd.bs;
    C* M = reinterpret_cast<C*>(smw);
    const CrLevelOffs lo = cr_level(K0, l);
    const int K = lo.K;
    C* W = work + sd.work_off + (l & 1) * work_len;
    C* F = fac + sd.fac_off;
    const int j = top ? 0 : 2 * o + 1;
    const int ncol = top ? 2 * w : 4 * w;
    const C* Ab = W + (long long)j * bs;
    const C* Cb = W + ((long long)K0 + 2LL * j) * bs;
    const C* Bb = Cb + bs;
    const bool hasB = !top && j + 1 < K;
    for (int e = tid; e < w * ncol; e += kWideThreads) {
        const int i = e / ncol, q = e % ncol;
        C v = czero<C>();
        if (q < w) v = Ab[(long long)q * ldw + i];
        else if (q < 2 * w) { if (q - w == i) v.x = T(1); }
        else if (q < 3 * w) v = Cb[(long long)(q - 2 * w) * ldw + i];
        else if (hasB) v = Bb[(long long)(q - 3 * w) * ldw + i];
        M[i * rs + q] = v;
    }
    __syncthreads();
    const int tq = tid % 128, par = tid / 128;
    for (int jj = 0; jj < w; ++jj) {
        if (tid < 32) {
            T val = (lane >= jj && lane < w) ? cabs2(M[lane * rs + jj]) : T(-1);
            if (!(val >= T(0)) || !isfinite(val)) val = (lane >= jj && lane < w) ? T(0) : T(-1);
            int best = lane;
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, val, off);
                const int ob = __shfl_xor_sync(0xffffffffu, best, off);
                if (ov > val || (ov == val && ob < best)) { val = ov; best = ob; }
            }
            if (lane == 0) s_piv = best;
        }
        __syncthreads();
        const int r = s_piv;
        if (r != jj)
            for (int q = jj + tid; q < ncol; q += kWideThreads) {
                const C t = M[jj * rs + q];
                M[jj * rs + q] = M[r * rs + q];
                M[r * rs + q] = t;
            }
        __syncthreads();
        C pv = M[jj * rs + jj];
        const T a2 = cabs2(pv);
        if (!(a2 > T(0)) || !isfinite(a2)) {
            if (tid == 0) atomicOr(err, LSS_DERR_SINGULAR);
            pv = czero<C>();
            pv.x = T(1);
        }
        const C pinv = crecip(pv);
        __syncthreads();   // every thread has read the pivot before row jj is scaled
        for (int q = jj + 1 + tid; q < ncol; q += kWideThreads) M[jj * rs + q] = M[jj * rs + q] * pinv;
        __syncthreads();
        // column jj is not written below and not read after this pivot
        for (int q = jj + 1 + tq; q < ncol; q += 128) {
            const C mj = M[jj * rs + q];
            for (int i = par; i < w; i += 2)
                if (i != jj) M[i * rs + q] = cfnma(M[i * rs + jj], mj, M[i * rs + q]);
        }
        __syncthreads();
    }
    C* Dout = F + (lo.dinv + (top ? 0 : o)) * bs;
    C* DCw = W + (3LL * K0 + 2LL * o) * bs;
    C* DCf = (!top && l >= 1) ? F + (lo.dcdb + 2LL * o) * bs : nullptr;
    for (int e = tid; e < bs; e += kWideThreads) {
        const int q = e / ldw, p = e % ldw;
        const bool in = p < w && q < w;
        Dout[e] = in ? M[p * rs + w + q] : czero<C>();
        if (!top) {
            const C dc = in ? M[p * rs + 2 * w + q] : czero<C>();
            const C db = in ? M[p * rs + 3 * w + q] : czero<C>();
            DCw[e] = dc;
            DCw[bs + e] = db;
            if (DCf) {
                DCf[e] = dc;
                DCf[bs + e] = db;
            }
        }
    }
}

// Even rows of level l: A'_e, C'_e, B'_e of level l+1 from D^{-1}C and D^{-1}B
// of the neighbouring odd rows, into the other work parity (and, for the even
// rows of level l+1, C' and B' into the factors).  C_e, B_e row-major and the
// four right factors transposed (row a of a factor holds its entries (a, q)
// for all columns q) in shared memory; thread (column q, row group g) computes
// rows g, g+8, g+16, g+24 of column q of A', C', B', summing over a in
// ascending order (at level 0, where C and B are tridiagonal, over the band).
template <typename T>
__global__ void __launch_bounds__(kWideThreads) cr_evenw_kernel(const SlabDev* __restrict__ slabs,
                                                               cx<T>* __restrict__ fac, cx<T>* __restrict__ work,
                                                               long long work_len, int K0, int l, int per_slab,
                                                               int slab0, int nlev) {
    using C = cx<T>;
    constexpr int LS = 33;
    extern __shared__ __align__(16) unsigned char smv[];
    const int tid = threadIdx.x;
    const int si = slab0 + blockIdx.x / per_slab, t = blockIdx.x % per_slab;
    const SlabDev sd = slabs[si];
    const int w = sd.w, ldw = sd.ldw, bs = sd.bs;
    const int K = cr_level(K0, l).K;
    const C* W = work + sd.work_off + (l & 1) * work_len;
    C* Wn = work + sd.work_off + ((l + 1) & 1) * work_len;
    C* F = fac + sd.fac_off;
    const int e = 2 * t;
    const bool hasL = e >= 1, hasR = e + 1 < K;
    const C* Ae = W + (long long)e * bs;
    const C* Ce = W + ((long long)K0 + 2LL * e) * bs;
    const C* Be = Ce + bs;
    const C* DCm = W + (3LL * K0 + 2LL * (t - 1)) * bs;   // odd row e-1
    const C* DCp = W + (3LL * K0 + 2LL * t) * bs;         // odd row e+1
    C* An = Wn + (long long)t * bs;
    const bool next_cb = l + 1 < nlev;
    C* Cn = Wn + ((long long)K0 + 2LL * t) * bs;
    C* Bn = Cn + bs;
    C* Cf = nullptr;
    if (next_cb && (t & 1) == 0) Cf = F + (cr_level(K0, l + 1).cbe + 2LL * (t >> 1)) * bs;
    C* L0 = reinterpret_cast<C*>(smv);   // C_e, row-major, stride LS
    C* L1 = L0 + 32 * LS;                // B_e
    C* Rt = L1 + 32 * LS;                // 4 right factors, transposed, stride LS
    const C* rsrc[4] = {DCm + bs, DCp, DCm, DCp + bs};   // (D^{-1}B)_{e-1}, (D^{-1}C)_{e+1}, (D^{-1}C)_{e-1}, (D^{-1}B)_{e+1}
    const bool rhas[4] = {hasL, hasR, hasL && next_cb, hasR && next_cb};
    for (int x = tid; x < w * w; x += kWideThreads) {
        const int p = x % w, a = x / w;
        L0[p * LS + a] = Ce[(long long)a * ldw + p];
        L1[p * LS + a] = Be[(long long)a * ldw + p];
#pragma unroll
        for (int f = 0; f < 4; ++f)   // entry (p, a) of column a of factor f -> row p of its transpose
            if (rhas[f]) Rt[f * 32 * LS + p * LS + a] = rsrc[f][(long long)a * ldw + p];
    }
    __syncthreads();
    const int q = tid & 31, g = tid >> 5;
    // out (rows g + 8 u) = init - L R_f for the staged left factor L
    auto product = [&](const C* L, int f, C (&out)[4]) {
        const C* R = Rt + f * 32 * LS;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int pp = g + 8 * u;
            if (pp >= w) break;
            C acc = czero<C>();
            if (l == 0) {
#pragma unroll
                for (int da = -1; da <= 1; ++da)
                    if (pp + da >= 0 && pp + da < w) acc = cfma(L[pp * LS + pp + da], R[(pp + da) * LS + q], acc);
            } else {
                for (int a = 0; a < w; ++a) acc = cfma(L[pp * LS + a], R[a * LS + q], acc);
            }
            out[u] = out[u] - acc;
        }
    };
    if (q < ldw) {
        C oa[4], oc[4], ob[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int pp = g + 8 * u;
            oa[u] = (q < w && pp < w) ? Ae[(long long)q * ldw + pp] : czero<C>();
            oc[u] = czero<C>();
            ob[u] = czero<C>();
        }
        if (q < w) {
            if (hasL) product(L0, 0, oa);
            if (hasR) product(L1, 1, oa);
            if (next_cb) {
                if (hasL) product(L0, 2, oc);
                if (hasR) product(L1, 3, ob);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int pp = g + 8 * u;
            if (pp >= ldw) break;
            const bool in = q < w && pp < w;
            const long long o = (long long)q * ldw + pp;
            An[o] = in ? oa[u] : czero<C>();
            if (next_cb) {
                Cn[o] = in ? oc[u] : czero<C>();
                Bn[o] = in ? ob[u] : czero<C>();
                if (Cf) {
                    Cf[o] = in ? oc[u] : czero<C>();
                    Cf[bs + o] = in ? ob[u] : czero<C>();
                }
            }
        }
    }
}

// ---------------------------------------------------------------- slab solves
// One kernel for the three uses of T~_i:
//   CR_A    sweep, first pass: a_i = T~_i f_i, first and last layers kept;
//   CR_E    sweep, second pass: T~_i (f_i - H lambda_{i-1} - H phi_{i+1}) on D_i;
//   CR_TEST T~_i applied to given vectors (lss_apply_slab).
// A CTA solves one right-hand side of one slab, held in shared memory (or
// per-CTA global scratch when it does not fit), block row k at b + k * G.  The
// factors stream through a ring of shared-memory stages in the order the solve
// reads them, one TMA bulk copy (two for the finest backward level) per chunk
// of block rows.  The chunk sequence depends only on n_tot, the block size, the
// output (first/last layers or all) and the stage size, so the host builds it
// once as a table of copies; thread 0 reads the next entry and issues it,
// every thread waits on the stage's mbarrier (bounded) and the block-wide
// barrier after each chunk frees its stage.  Lanes are grouped by G (16 when
// the slab is at most 16 layers wide, else 32): lane p of a group owns layer p
// of one block row.
enum CrMode { CR_A = 0, CR_E = 1, CR_TEST = 2 };
enum CrPhase { PH_FODD = 0, PH_FEVEN = 1, PH_TOP = 2, PH_BODD = 3, PH_B0 = 4 };

// One chunk of a solve: phase, level, block rows [r0, r1) of the phase, and the
// one or two copies (entry offsets from the slab's factor base, entries).
struct CrChunk {
    int kind, l, r0, r1;
    int ent, ent2;
    long long src, src2;
};

template <typename C>
struct CrArgs {
    const SlabDev* slabs;
    int n_slabs, n_tot, n, b, R;
    const C* fac;
    const C* coef;
    const C* f;              // sweep: R x n_tot^2 sparsified right-hand side, x2 index slowest
    C* a_first;              // CR_A outputs, [slab][k][R]
    C* a_last;
    const C* lam;            // CR_E inputs, [slab][k][R]
    const C* phi;
    double2* y;              // CR_E output, R x n^2 (or R x n_tot^2 when y_grid)
    int y_grid;              // CR_E: write every point of D_i on the grid (x2 slowest) instead of I
    int slab;                // CR_TEST
    const double2* v_in;     // R x (layers of D_i) x n_tot
    double2* w_out;
    const CrChunk* tab16;    // chunk tables for 16- and 32-wide blocks
    const CrChunk* tab32;
    int n16, n32;
    C* bg;                   // right-hand sides in global memory when bsm == 0
    long long bstride;       // entries of b per CTA
    int bsm;
    int nst, stage_ent;      // ring stages and complex entries per stage
    int slab0;               // CR_A / CR_E: first slab of the launch (grid y = slab - slab0)
    int* err;
};

struct CrLv {
    int K;
    long long dinv, cbe, dcdb;
};

// acc[c] (+/-)= sum_a M(p, a) x_c[a] for ncol <= CPT columns (x_c at x + c * xs):
// the block's row is read into registers once (16 entries at a time, 8 in
// double precision) and applied to every column.
template <typename C, int G, int CPT, bool SUB>
__device__ __forceinline__ void mv_cols(const C* M, int p, const C* x, int xs, int ncol, C (&acc)[CPT]) {
    constexpr int HB = sizeof(C) == 16 ? 8 : 16;
#pragma unroll
    for (int h = 0; h < G; h += HB) {
        C m[HB];
#pragma unroll
        for (int u = 0; u < HB; ++u) m[u] = M[(h + u) * G + p];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (c < ncol) {
                const C* xc = x + c * xs + h;
                C s0 = czero<C>(), s1 = czero<C>();
#pragma unroll
                for (int u = 0; u < HB; u += 2) {
                    s0 = cfma(m[u], xc[u], s0);
                    s1 = cfma(m[u + 1], xc[u + 1], s1);
                }
                acc[c] = SUB ? acc[c] - (s0 + s1) : acc[c] + (s0 + s1);
            }
        }
    }
}

// Level-0 off-diagonal block from its bands (band[(da + 1) * G + p] couples
// layer p to layer p + da, zero outside the slab): acc (+/-)= sum_da band x[p + da].
template <typename C, int G, bool SUB>
__device__ __forceinline__ C band_row(const C* band, int p, const C* x, C acc) {
#pragma unroll
    for (int da = -1; da <= 1; ++da) {
        const int a = p + da;
        if (a < 0 || a >= G) continue;
        const C cv = band[(da + 1) * G + p];
        acc = SUB ? cfnma(cv, x[a], acc) : cfma(cv, x[a], acc);
    }
    return acc;
}

// Partial product sum_{a0 <= a < a0 + N} M(p, a) x[a] of one block row (M
// column-major G x G in shared memory).
template <typename C, int G, int N>
__device__ __forceinline__ C mv_part(const C* M, int p, const C* x, int a0) {
    C s0 = czero<C>(), s1 = czero<C>();
#pragma unroll
    for (int u = 0; u < N; u += 2) {
        s0 = cfma(M[(a0 + u) * G + p], x[a0 + u], s0);
        s1 = cfma(M[(a0 + u + 1) * G + p], x[a0 + u + 1], s1);
    }
    return s0 + s1;
}

// Phases whose 32-wide block rows are split over four warps, and the most
// block rows such a chunk holds (4 x 6 warp tasks: two per warp)
constexpr int kSplitRows = 6;
__host__ __device__ __forceinline__ bool cr_split_phase(int G, int kind, int l, bool part) {
    return G == 32 && !(kind == PH_FEVEN && l == 0) && !(kind == PH_B0 && part);
}

// The chunk sequence of one solve (host side): phases FODD(l), FEVEN(l) for
// l = 0..L-1, TOP, BODD(l) for l = L-1..1, B0; each phase's block rows in chunks
// of at most min(2 x lane groups, stage / row size) rows.
std::vector<CrChunk> cr_chunk_table(int K, int G, bool part, int stage_ent, int groups) {
    std::vector<CrChunk> out;
    const int L = cr_levels(K), bs = G * G;
    const long long t0 = cr_t0_off(K, bs), p0 = cr_p0_off(K, bs, G);
    const CrLevelOffs top = cr_level(K, L);
    for (int ph = 0; ph < 3 * L + 1; ++ph) {
        int kind, l, rb;
        if (ph < 2 * L) {
            l = ph >> 1;
            kind = (ph & 1) ? PH_FEVEN : PH_FODD;
            const int Kl = cr_level(K, l).K;
            rb = kind == PH_FODD ? Kl / 2 : (Kl + 1) / 2;
        } else if (ph == 2 * L) {
            kind = PH_TOP; l = L; rb = 1;
        } else if (ph < 3 * L) {
            kind = PH_BODD; l = 3 * L - ph; rb = cr_level(K, l).K / 2;
        } else {
            kind = PH_B0; l = 0; rb = K / 2;
        }
        int row;
        switch (kind) {
            case PH_FODD: case PH_TOP: row = bs; break;
            case PH_FEVEN: row = l == 0 ? 6 * G : 2 * bs; break;
            case PH_BODD: row = 2 * bs; break;
            default: row = 6 * G + (part ? 2 * G : bs);
        }
        int rpc = std::max(1, std::min(2 * groups, stage_ent / row));
        if (cr_split_phase(G, kind, l, part)) rpc = std::min(rpc, kSplitRows);
        const CrLevelOffs lv = cr_level(K, l);
        for (int r0 = 0; r0 < rb; r0 += rpc) {
            const int r1 = std::min(rb, r0 + rpc), nr = r1 - r0;
            CrChunk ch{kind, l, r0, r1, 0, 0, 0, 0};
            switch (kind) {
                case PH_FODD: ch.src = (lv.dinv + r0) * bs; ch.ent = nr * bs; break;
                case PH_FEVEN:
                    if (l == 0) { ch.src = t0 + (long long)r0 * 6 * G; ch.ent = nr * 6 * G; }
                    else { ch.src = (lv.cbe + 2LL * r0) * bs; ch.ent = 2 * nr * bs; }
                    break;
                case PH_TOP: ch.src = top.dinv * bs; ch.ent = bs; break;
                case PH_BODD: ch.src = (lv.dcdb + 2LL * r0) * bs; ch.ent = 2 * nr * bs; break;
                default:
                    ch.src = t0 + ((long long)(K + 1) / 2 + r0) * 6 * G;
                    ch.ent = nr * 6 * G;
                    if (part) { ch.src2 = p0 + 2LL * r0 * G; ch.ent2 = 2 * nr * G; }
                    else { ch.src2 = (cr_level(K, 0).dinv + r0) * bs; ch.ent2 = nr * bs; }
            }
            out.push_back(ch);
        }
    }
    return out;
}

// One CTA solves slab i's subproblem for NR right-hand sides r, r+1, ..,
// each factor chunk serving all of them (NR = 2 only with 16-wide blocks);
// b holds the NR right-hand sides one after another.
template <typename C, int MODE, int G, int NR>
__device__ __forceinline__ void cr_body(const CrArgs<C>& A, const SlabDev& sd, int i, int r, C* b, C* tb, C* ring,
                                        uint64_t* full, int4* desc, const CrLv* lv, bool& ok) {
    static_assert(NR == 1 || G == 16, "several right-hand sides per CTA with 16-wide blocks only");
    const int K = A.n_tot, w = sd.w, bs = sd.bs, na = sd.na;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
    constexpr int GPW = 32 / G;
    constexpr int CPT = 1;
    constexpr int lw = G;
    const int nc = 1;
    const int grp = lane / G, p = lane % G;
    const C* F = A.fac + sd.fac_off;
    const C* cf = A.coef + sd.coef_off;
    C* tg = tb + (size_t)(warp * GPW + grp) * G;
    auto row = [&](int k) { return b + (long long)k * lw; };
    const long long nt2 = (long long)K * K;
    constexpr bool kPart = MODE == CR_A;
    const CrChunk* tab = G == 16 ? A.tab16 : A.tab32;
    const int ntab = G == 16 ? A.n16 : A.n32;

    // ---- first chunks in flight while the right-hand side is written; thread
    // 0 publishes each chunk's descriptor beside its stage (kind -1: the end)
    // thread 0 keeps the descriptor of the next chunk to issue in registers,
    // loaded one chunk ahead, so that no table load sits between two barriers
    CrChunk pre{};
    auto issue_next = [&](int g) {
        const int st = g % A.nst;
        if (g < ntab) {
            const CrChunk ch = g >= A.nst ? pre : tab[g];
            if (g >= A.nst - 1 && g + 1 < ntab) pre = tab[g + 1];
            desc[st] = make_int4(ch.kind, ch.l, ch.r0, ch.r1);
            C* dst = ring + (size_t)st * A.stage_ent;
            mbar_expect_tx(&full[st], (unsigned)((ch.ent + ch.ent2) * (int)sizeof(C)));
            tma_load_1d(dst, F + ch.src, (unsigned)(ch.ent * sizeof(C)), &full[st]);
            if (ch.ent2) tma_load_1d(dst + ch.ent, F + ch.src2, (unsigned)(ch.ent2 * sizeof(C)), &full[st]);
        } else {
            desc[st] = make_int4(-1, 0, 0, 0);
        }
    };
    if (tid == 0)
        for (int st = 0; st < A.nst; ++st) issue_next(st);

    // ---- right-hand side
    for (int e = tid; e < NR * K * lw; e += nth) {   // right-hand side r + e / (K lw), block row k
        const int pp = e % lw;
        const int k = (e / lw) % K;
        const int rq = r + e / (K * lw);
        C v = czero<C>();
        if (pp < w && rq < A.R) {
            const int r = rq;
            if (MODE == CR_A || MODE == CR_E) {
                if (pp >= na && pp <= sd.ll) v = A.f[(long long)r * nt2 + (long long)k * K + sd.s + A.b + (pp - na)];
                if (MODE == CR_E) {
                    const C* ck = cf + (long long)k * sd.cstride + pp * 9;
                    const long long vec = (long long)K * A.R;
                    if (pp == na && i > 0)
                        for (int dk = -1; dk <= 1; ++dk) {
                            const int kk = k + dk;
                            if (kk >= 0 && kk < K)
                                v = cfnma(ck[dk + 1], A.lam[(long long)(i - 1) * vec + (long long)kk * A.R + r], v);
                        }
                    if (pp == sd.ll && i < A.n_slabs - 1)
                        for (int dk = -1; dk <= 1; ++dk) {
                            const int kk = k + dk;
                            if (kk >= 0 && kk < K)
                                v = cfnma(ck[6 + dk + 1], A.phi[(long long)(i + 1) * vec + (long long)kk * A.R + r], v);
                        }
                }
            } else {
                if (pp >= na && pp <= sd.ll) v = to_c<C>(A.v_in[((long long)r * sd.nl + (pp - na)) * K + k]);
            }
        }
        b[e] = v;
    }
    __syncthreads();   // b written, first descriptors published

    // ---- the chunk walk
    for (int g = 0;; ++g) {
        const int st = g % A.nst;
        const int4 dsc = desc[st];
        if (dsc.x < 0) break;
        const int kind = dsc.x, l = dsc.y, r0 = dsc.z, r1 = dsc.w;
        // every thread waits for the stage itself (no block-wide consensus
        // barrier here); after an expired wait a thread stops waiting and the
        // walk runs to its end on stale data, whose results the host discards
        // (the status word carries the timeout)
        if (ok && !mbar_wait(&full[st], (g / A.nst) & 1, A.err)) ok = false;
        const C* S = ring + (size_t)st * A.stage_ent;
        const int cnt = r1 - r0;
        const int Kl = lv[l].K;
        // 32-wide blocks: only a few block rows fit a stage, so each row's
        // products are split over four warps (column quarters, or block x half
        // of the columns in the two-block phases) and the partial sums meet in
        // shared memory after one more barrier
        const bool split = cr_split_phase(G, kind, l, kPart);
        if (split) {
            C* part = tb + kSolveThreads;   // kSplitRows x 4 x 32 partial sums
            for (int t0 = warp; t0 < cnt * 4; t0 += nw) {   // one warp per (row, part); G == 32
                const int t = t0 >> 2, qs = t0 & 3;
                const int rr = r0 + t;
                C acc = czero<C>();
                if (kind == PH_FODD || kind == PH_TOP) {
                    const int k = kind == PH_TOP ? 0 : (2 * rr + 1) << l;
                    acc = mv_part<C, G, 8>(S + (size_t)t * bs, p, row(k), qs * 8);
                } else if (kind == PH_FEVEN || kind == PH_BODD) {
                    const int blk = qs >> 1, half = qs & 1;
                    const int j = kind == PH_FEVEN ? 2 * rr : 2 * rr + 1;
                    const int nb = blk == 0 ? j - 1 : j + 1;
                    if (nb >= 0 && nb < Kl)
                        acc = mv_part<C, G, 16>(S + (size_t)(2 * t + blk) * bs, p, row(nb << l), half * 16);
                } else {   // level 0, all layers: t = C x_{k-1} + B x_{k+1}, then a quarter of D^{-1} t
                    const int k = 2 * rr + 1;
                    const C* band = S + (size_t)t * 6 * G;
                    C tv = band_row<C, G, false>(band, p, row(k - 1), czero<C>());
                    if (k + 1 < Kl) tv = band_row<C, G, false>(band + 3 * G, p, row(k + 1), tv);
                    const C* D = S + (size_t)cnt * 6 * G + (size_t)t * bs;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int a = qs * 8 + u;
                        C ta;
                        ta.x = __shfl_sync(0xffffffffu, tv.x, a);
                        ta.y = __shfl_sync(0xffffffffu, tv.y, a);
                        acc = cfma(D[a * G + p], ta, acc);
                    }
                }
                part[(t * 4 + qs) * 32 + p] = acc;
            }
            __syncthreads();
            for (int t = warp; t < cnt; t += nw) {
                const int rr = r0 + t;
                int k;
                if (kind == PH_TOP) k = 0;
                else if (kind == PH_FEVEN) k = (2 * rr) << l;
                else if (kind == PH_B0) k = 2 * rr + 1;
                else k = (2 * rr + 1) << l;
                const C* pt = part + t * 4 * 32 + p;
                const C sum = (pt[0] + pt[32]) + (pt[64] + pt[96]);
                C* x = row(k);
                x[p] = (kind == PH_FODD || kind == PH_TOP) ? sum : x[p] - sum;
            }
        } else
        for (int t0 = warp * GPW; t0 < cnt * NR; t0 += nw * GPW) {
            // task = (right-hand side q, row t of the chunk)
            const int tq = t0 + grp;
            const bool on = tq < cnt * NR;
            const int q = on ? tq / cnt : 0;
            const int t = on ? tq - q * cnt : 0;
            C* const bq = b + (long long)q * K * lw;
            auto row = [&](int k) { return bq + (long long)k * lw; };
            const int rr = r0 + t;
            C acc[CPT];
            if (kind == PH_FODD || kind == PH_TOP) {
                // y_o = D_o^{-1} b_o (top: x_0 = D^{-1} b_0); the group reads its row first
                const int k = kind == PH_TOP ? 0 : (2 * rr + 1) << l;
                C* x = row(k);
                acc[0] = czero<C>();
                if (on) mv_cols<C, G, CPT, false>(S + (size_t)t * bs, p, x, lw, nc, acc);
                __syncwarp();
                if (on) x[p] = acc[0];
                __syncwarp();
            } else if (kind == PH_FEVEN) {
                // b_e -= C_e y_{e-1} + B_e y_{e+1}
                if (!on) continue;
                const int e = 2 * rr, k = e << l;
                C* x = row(k);
                acc[0] = x[p];
                if (l == 0) {
                    const C* band = S + (size_t)t * 6 * G;
                    if (e >= 1) acc[0] = band_row<C, G, true>(band, p, row(k - 1), acc[0]);
                    if (e + 1 < Kl) acc[0] = band_row<C, G, true>(band + 3 * G, p, row(k + 1), acc[0]);
                } else {
                    const C* Cm = S + (size_t)2 * t * bs;
                    if (e >= 1) mv_cols<C, G, CPT, true>(Cm, p, row((e - 1) << l), lw, nc, acc);
                    if (e + 1 < Kl) mv_cols<C, G, CPT, true>(Cm + bs, p, row((e + 1) << l), lw, nc, acc);
                }
                x[p] = acc[0];
            } else if (kind == PH_BODD) {
                // x_o = y_o - D^{-1}C x_{o-1} - D^{-1}B x_{o+1}
                if (!on) continue;
                const int j = 2 * rr + 1, k = j << l;
                C* x = row(k);
                acc[0] = x[p];
                const C* DC = S + (size_t)2 * t * bs;
                mv_cols<C, G, CPT, true>(DC, p, row((j - 1) << l), lw, nc, acc);
                if (j + 1 < Kl) mv_cols<C, G, CPT, true>(DC + bs, p, row((j + 1) << l), lw, nc, acc);
                x[p] = acc[0];
            } else {
                // level 0: x_o = y_o - D_o^{-1} (C_o x_{o-1} + B_o x_{o+1})
                const int k = 2 * rr + 1;
                const C* band = S + (size_t)t * 6 * G;
                C tv = czero<C>();
                if (on) {
                    tv = band_row<C, G, false>(band, p, row(k - 1), tv);
                    if (k + 1 < Kl) tv = band_row<C, G, false>(band + 3 * G, p, row(k + 1), tv);
                }
                const C* Dp = S + (size_t)cnt * 6 * G;
                C* x = row(k);
                if (!kPart) {
                    tg[p] = tv;
                    __syncwarp();
                    acc[0] = on ? x[p] : czero<C>();
                    if (on) mv_cols<C, G, CPT, true>(Dp + (size_t)t * bs, p, tg, G, nc, acc);
                    if (on) x[p] = acc[0];
                    __syncwarp();
                } else {
                    // only layers na and ll: the two rows of D^{-1} against t, reduced over the group
                    const C* pr = Dp + (size_t)t * 2 * G;
                    const C q0 = on ? pr[p] : czero<C>(), q1 = on ? pr[G + p] : czero<C>();
                    C d0 = q0 * tv, d1 = q1 * tv;
#pragma unroll
                    for (int off = G / 2; off > 0; off >>= 1) {
                        d0.x += __shfl_xor_sync(0xffffffffu, d0.x, off, G);
                        d0.y += __shfl_xor_sync(0xffffffffu, d0.y, off, G);
                        d1.x += __shfl_xor_sync(0xffffffffu, d1.x, off, G);
                        d1.y += __shfl_xor_sync(0xffffffffu, d1.y, off, G);
                    }
                    if (on && p == na) x[na] = x[na] - d0;
                    if (on && p == sd.ll && sd.ll != na) x[sd.ll] = x[sd.ll] - d1;
                }
            }
        }
        __syncthreads();   // the stage is free, the phase's rows are written
        if (tid == 0) issue_next(g + A.nst);
    }

    // ---- outputs, per right-hand side
    for (int q = 0; q < NR; ++q) {
        const int rq = r + q;
        if (rq >= A.R) break;
        C* const bq = b + (long long)q * K * lw;
        auto rowo = [&](int k) { return bq + (long long)k * lw; };
        if (MODE == CR_A) {
            const long long base = (long long)i * K * A.R + rq;
            for (int k = tid; k < K; k += nth) {
                A.a_first[base + (long long)k * A.R] = rowo(k)[na];
                A.a_last[base + (long long)k * A.R] = rowo(k)[sd.ll];
            }
        } else if (MODE == CR_E) {
            const int nl = sd.nl;
            for (int e = tid; e < nl * K; e += nth) {
                const int k = e % K, pp = na + e / K;
                const int x1 = sd.s + (pp - na), i2 = k - A.b;
                if (A.y_grid)
                    A.y[(long long)rq * A.n_tot * A.n_tot + (long long)k * A.n_tot + (x1 + A.b)] = to_d(rowo(k)[pp]);
                else if (x1 >= 1 && x1 <= A.n && i2 >= 1 && i2 <= A.n)
                    A.y[(long long)rq * A.n * A.n + (long long)(x1 - 1) * A.n + (i2 - 1)] = to_d(rowo(k)[pp]);
            }
        } else {
            const int nl = sd.nl;
            for (int e = tid; e < nl * K; e += nth) {
                const int k = e % K, pp = na + e / K;
                A.w_out[((long long)rq * nl + (pp - na)) * K + k] = to_d(rowo(k)[pp]);
            }
        }
    }
}

template <typename T, int MODE, int NR = 1>
__global__ void __launch_bounds__(kSolveThreads) cr_solve_kernel(CrArgs<cx<T>> A) {
    using C = cx<T>;
    __shared__ CrLv lv[33];
    __shared__ __align__(8) uint64_t full[4];
    __shared__ int4 desc[4];
    extern __shared__ __align__(128) unsigned char sms[];
    const int K = A.n_tot;
    C* tb = reinterpret_cast<C*>(sms) + (A.bsm ? A.bstride : 0);
    C* ring = tb + (size_t)kSolveThreads + kSplitRows * 4 * 32;
    if (threadIdx.x == 0) {
        const int L = cr_levels(K);
        for (int l = 0; l <= L; ++l) {
            const CrLevelOffs o = cr_level(K, l);
            lv[l] = CrLv{o.K, o.dinv, o.cbe, o.dcdb};
        }
        for (int st = 0; st < A.nst; ++st) mbar_init(&full[st], 1);
        fence_mbar_init();
    }
    bool ok = true;
    __syncthreads();
    int i, r;
    long long cta;
    if (MODE == CR_TEST) { i = A.slab; r = blockIdx.x; cta = blockIdx.x; }
    // slab-major grid: a slab's right-hand sides run together and share its factor stream in L2
    else { i = A.slab0 + blockIdx.y; r = blockIdx.x * NR; cta = (long long)blockIdx.y * gridDim.x + blockIdx.x; }
    const SlabDev sd = A.slabs[i];
    C* b = A.bsm ? reinterpret_cast<C*>(sms) : A.bg + cta * A.bstride;
    if (sd.w <= 16) cr_body<C, MODE, 16, NR>(A, sd, i, r, b, tb, ring, full, desc, lv, ok);
    else if constexpr (NR == 1) cr_body<C, MODE, 32, 1>(A, sd, i, r, b, tb, ring, full, desc, lv, ok);
    else if (threadIdx.x == 0) atomicOr(A.err, LSS_DERR_CONFIG);   // the host launches NR > 1 for 16-wide slabs only
    if (__syncthreads_or(!ok) && threadIdx.x == 0) {
        // a wait expired: give the copies already issued a bounded chance to land
        const long long t0 = clock64();
        while (clock64() - t0 < 2000000ll) __nanosleep(1000);
    }
}

// ---------------------------------------------------------------- interface recurrences
// Grid-wide version (cooperative launch, bounded grid barrier): the fallback
// when the vectors or rows do not fit the cluster kernel below.
// Tiles of the grid-synchronised recurrence: each step is a product of an
// n_tot x n_tot map with the n_tot x R block of current vectors; a CTA forms a
// kGtR x kGtC tile of it over K chunks of kGtK staged in shared memory
// (coalesced loads of map rows and vector rows, the next chunk loaded into
// registers while the current one is multiplied).  Each thread owns four rows
// of one column, so a vector entry read from shared memory serves four
// products and the map entries are read as broadcasts.
// Tiles of TR = 64 rows (4 per thread) when a step has enough of them,
// else TR = 32 (2 per thread).  The K chunks stream into a ring of kGtS
// shared-memory stages by cp.async copies issued kGtS - 1 chunks ahead (many
// bytes in flight per SM: the maps come from DRAM at every step).
constexpr int kGtC = 16, kGtK = 32, kGtS = 4;


// entries of one ring stage: the map tile (TR rows, kGtK + 2 per row) and
// the vector tile (kGtK rows, kGtC + 1 per row)
template <int TR>
constexpr int gt_stage_ent() { return TR * (kGtK + 2) + kGtK * (kGtC + 1); }

template <typename T, int TR>
__device__ __forceinline__ void recur_tile(const cx<T>* __restrict__ M, const cx<T>* x, const cx<T>* base,
                                           cx<T>* out, int n_tot, int R, int rt, int ct, cx<T>* ring) {
    using C = cx<T>;
    constexpr int RPT = TR / 16;                  // rows per thread
    constexpr int LA = TR * kGtK / 256;           // map entries a thread copies per chunk
    constexpr int LB = kGtK * kGtC / 256;         // vector entries a thread copies per chunk
    constexpr int SE = gt_stage_ent<TR>();
    static_assert(TR * kGtK % 256 == 0 && kGtK * kGtC % 256 == 0, "a chunk must split evenly over the threads");
    const int tid = threadIdx.x;
    const int ty = tid / kGtC, tx = tid % kGtC;   // rows RPT ty .. RPT ty + RPT - 1, column tx
    const int nch = (n_tot + kGtK - 1) / kGtK;
    auto issue = [&](int ch) {
        if (ch < nch) {
            C* As = ring + (ch % kGtS) * SE;
            C* Bs = As + TR * (kGtK + 2);
            const int k0 = ch * kGtK;
#pragma unroll
            for (int u = 0; u < LA; ++u) {
                const int e = tid + 256 * u;
                const int a = e / kGtK, kk = e % kGtK;
                const int gr = rt * TR + a, gk = k0 + kk;
                const bool ok = gr < n_tot && gk < n_tot;
                cp_async_entry(As + a * (kGtK + 2) + kk, ok ? M + (long long)gr * n_tot + gk : M, ok);
            }
#pragma unroll
            for (int u = 0; u < LB; ++u) {
                const int e = tid + 256 * u;
                const int kk = e / kGtC, c = e % kGtC;
                const int gk = k0 + kk, gc = ct * kGtC + c;
                const bool ok = gk < n_tot && gc < R;
                cp_async_entry(Bs + kk * (kGtC + 1) + c, ok ? x + (long long)gk * R + gc : x, ok);
            }
        }
        cp_async_commit();   // (an empty group past the last chunk keeps the count uniform)
    };
    C acc[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i] = czero<C>();
#pragma unroll
    for (int q = 0; q < kGtS - 1; ++q) issue(q);
    for (int ch = 0; ch < nch; ++ch) {
        cp_async_wait<kGtS - 2>();   // chunk ch has landed (this thread's copies)
        __syncthreads();             // ... and every thread's
        const C* As = ring + (ch % kGtS) * SE;
        const C* Bs = As + TR * (kGtK + 2);
#pragma unroll 8
        for (int kk = 0; kk < kGtK; ++kk) {
            const C bv = Bs[kk * (kGtC + 1) + tx];
#pragma unroll
            for (int i = 0; i < RPT; ++i) acc[i] = cfma(As[(RPT * ty + i) * (kGtK + 2) + kk], bv, acc[i]);
        }
        __syncthreads();             // the stage of chunk ch may be refilled
        issue(ch + kGtS - 1);
    }
    cp_async_wait<0>();
    const int col = ct * kGtC + tx;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = rt * TR + RPT * ty + i;
        if (row < n_tot && col < R) {
            const long long e = (long long)row * R + col;
            out[e] = base[e] - acc[i];
        }
    }
}

// Few right-hand sides (R <= RM, RM in 1, 2, 4, 8): a 16-column tile would
// spend most of its multiply-adds on absent columns (on FP64, where the pipe
// is the bound, up to 16 times the work), so a tile is TR rows instead, two
// per warp: lanes stride over k (coalesced map rows, the vector entries shared
// by the warp's two rows), then a shuffle reduction per row and column.
template <typename T, int RM>
__device__ __forceinline__ void recur_rows(const cx<T>* __restrict__ M, const cx<T>* x, const cx<T>* base,
                                           cx<T>* out, int n_tot, int R, int row0, int nrows) {
    using C = cx<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = 2 * warp; p < nrows; p += 2 * nw) {
        const int r0 = row0 + p;
        const bool two = p + 1 < nrows;
        const C* m0 = M + (long long)r0 * n_tot;
        const C* m1 = two ? m0 + n_tot : m0;
        C a0[RM], a1[RM];
#pragma unroll
        for (int c = 0; c < RM; ++c) a0[c] = a1[c] = czero<C>();
#pragma unroll 2
        for (int k = lane; k < n_tot; k += 32) {
            const C u0 = m0[k], u1 = m1[k];
#pragma unroll
            for (int c = 0; c < RM; ++c) {
                if (RM > 1 && c >= R) break;
                const C xv = x[(long long)k * R + c];
                a0[c] = cfma(u0, xv, a0[c]);
                a1[c] = cfma(u1, xv, a1[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < RM; ++c) {
            if (RM > 1 && c >= R) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a0[c].x += __shfl_xor_sync(0xffffffffu, a0[c].x, o);
                a0[c].y += __shfl_xor_sync(0xffffffffu, a0[c].y, o);
                a1[c].x += __shfl_xor_sync(0xffffffffu, a1[c].x, o);
                a1[c].y += __shfl_xor_sync(0xffffffffu, a1[c].y, o);
            }
            if (lane == 0) {
                const long long e0 = (long long)r0 * R + c;
                C v = base[e0];
                v.x -= a0[c].x;
                v.y -= a0[c].y;
                out[e0] = v;
                if (two) {
                    C w = base[e0 + R];
                    w.x -= a1[c].x;
                    w.y -= a1[c].y;
                    out[e0 + R] = w;
                }
            }
        }
    }
}

// One task of a recurrence step: tile (rt, ct) of out = base - M x.  RM = 0:
// TR x kGtC tiles staged through the ring; RM > 0: TR-row tiles, every column.
template <typename T, int TR, int RM>
__device__ __forceinline__ void recur_task(const cx<T>* __restrict__ M, const cx<T>* x, const cx<T>* base,
                                           cx<T>* out, int n_tot, int R, int rt, int ct, cx<T>* ring) {
    if constexpr (RM == 0)
        recur_tile<T, TR>(M, x, base, out, n_tot, R, rt, ct, ring);
    else
        recur_rows<T, RM>(M, x, base, out, n_tot, R, rt * TR, min(TR, n_tot - rt * TR));
}

template <int RM>
__host__ __device__ constexpr int recur_col_tiles(int R) { return RM ? 1 : (R + kGtC - 1) / kGtC; }

// Recurrences of all slabs with one cooperative grid when the vectors do not
// fit the cluster kernels (many right-hand sides): lambda and mu, then phi,
// one step per slab, a grid barrier between steps; the tiles of a step are
// spread over the CTAs.
template <typename T, int TR, int RM>
__global__ void __launch_bounds__(256) recur_grid_kernel(int n_slabs, int n_tot, int R,
                                                         const cx<T>* __restrict__ iface,
                                                         const cx<T>* __restrict__ a_first,
                                                         const cx<T>* __restrict__ a_last, cx<T>* lam, cx<T>* phi,
                                                         unsigned* bar, int* err) {
    using C = cx<T>;
    extern __shared__ __align__(16) unsigned char gts[];
    C* ring = reinterpret_cast<C*>(gts);   // kGtS stages of gt_stage_ent<TR>() entries
    unsigned nbar = 0;                     // grid barriers passed (the arrival counter starts at zero)
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const int nrt = (n_tot + TR - 1) / TR, nct = recur_col_tiles<RM>(R);
    const int ntile = nrt * nct;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < vec;
         e += (long long)gridDim.x * blockDim.x)
        lam[e] = a_last[e];
    for (int i = 1; i < n_slabs; ++i) {
        const C* lp = (i == 1) ? a_last : lam + (long long)(i - 1) * vec;
        const int nwhich = (i <= n_slabs - 2) ? 2 : 1;
        for (int task = blockIdx.x; task < nwhich * ntile; task += gridDim.x) {   // uniform per CTA
            const int which = task / ntile, t = task % ntile;
            if (which == 0)   // mu_i = first(a_i) - Gamma_i lambda_{i-1}
                recur_task<T, TR, RM>(iface + (1LL * n_slabs + i) * nt2, lp, a_first + (long long)i * vec,
                              phi + (long long)i * vec, n_tot, R, t / nct, t % nct, ring);
            else              // lambda_i = last(a_i) - Lambda_i lambda_{i-1}
                recur_task<T, TR, RM>(iface + (long long)i * nt2, lp, a_last + (long long)i * vec,
                              lam + (long long)i * vec, n_tot, R, t / nct, t % nct, ring);
        }
        grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    }
    for (int i = n_slabs - 2; i >= 1; --i) {   // phi_i = mu_i - Phi_i phi_{i+1}
        for (int task = blockIdx.x; task < ntile; task += gridDim.x)
            recur_task<T, TR, RM>(iface + (2LL * n_slabs + i) * nt2, phi + (long long)(i + 1) * vec,
                          phi + (long long)i * vec, phi + (long long)i * vec, n_tot, R, task / nct, task % nct, ring);
        grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    }
}

// The recurrences of the two-front sweep (Sec. 2.4 remark 1) with one
// cooperative grid.  Slabs left of the middle slab c carry lambda_i (their
// forward solution's last layer) and then phi_i (the final first layer);
// slabs right of c carry phi_i = rho_i (their forward solution's first layer,
// from the right front) and then lambda_i (the final last layer).  Maps:
// Lambda (first-layer pin -> last layer), Gamma (-> first layer), Phi
// (last-layer pin -> first layer), Psi (-> last layer).
//   fronts:  lambda_i = last(a_i) - Lambda_i lambda_{i-1},  mu_i = first(a_i) - Gamma_i lambda_{i-1}  (i < c)
//            phi_i = first(a_i) - Phi_i phi_{i+1},          nu_i = last(a_i) - Psi_i phi_{i+1}       (i > c)
//   middle:  phi_c = first(a_c) - Gamma_c lambda_{c-1} - Phi_c phi_{c+1}
//            lambda_c = last(a_c) - Lambda_c lambda_{c-1} - Psi_c phi_{c+1}
//   back:    phi_i = mu_i - Phi_i phi_{i+1} (i < c),  lambda_i = nu_i - Lambda_i lambda_{i-1} (i > c)
// Both fronts advance in the same grid step, so the dependent steps are about
// half of the one-front recurrences'.
template <typename T, int TR, int RM>
__global__ void __launch_bounds__(256) recur_grid2_kernel(int n_slabs, int mid, int n_tot, int R,
                                                          const cx<T>* __restrict__ iface,
                                                          const cx<T>* __restrict__ a_first,
                                                          const cx<T>* __restrict__ a_last, cx<T>* lam, cx<T>* phi,
                                                          unsigned* bar, int* err) {
    using C = cx<T>;
    extern __shared__ __align__(16) unsigned char gts[];
    C* ring = reinterpret_cast<C*>(gts);   // kGtS stages of gt_stage_ent<TR>() entries
    unsigned nbar = 0;                     // grid barriers passed (the arrival counter starts at zero)
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const int nrt = (n_tot + TR - 1) / TR, nct = recur_col_tiles<RM>(R);
    const int ntile = nrt * nct;
    const int ns = n_slabs, c = mid;
    const C* LAM = iface;
    const C* GAM = iface + (long long)ns * nt2;
    const C* PHI = iface + 2LL * ns * nt2;
    const C* PSI = iface + 3LL * ns * nt2;
    auto V = [&](C* a, int i) { return a + (long long)i * vec; };
    auto Vc = [&](const C* a, int i) { return a + (long long)i * vec; };
    // lambda_0 and rho_{l-1}; phi_c = first(a_c) when nothing is left of c
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < vec;
         e += (long long)gridDim.x * blockDim.x) {
        lam[e] = a_last[e];
        V(phi, ns - 1)[e] = Vc(a_first, ns - 1)[e];
        if (c == 0) phi[e] = a_first[e];
    }
    grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    const int S = max(c - 1, ns - 2 - c);
    for (int st = 0; st < S; ++st) {   // both fronts toward c
        const int iL = 1 + st, iR = ns - 2 - st;
        const bool onL = iL <= c - 1, onR = iR >= c + 1;
        const int nw = 2 * (onL + onR);
        for (int task = blockIdx.x; task < nw * ntile; task += gridDim.x) {   // uniform per CTA
            int which = task / ntile;
            const int t = task % ntile;
            if (!onL) which += 2;
            if (which == 0)
                recur_task<T, TR, RM>(LAM + iL * nt2, V(lam, iL - 1), Vc(a_last, iL), V(lam, iL), n_tot, R, t / nct, t % nct, ring);
            else if (which == 1)
                recur_task<T, TR, RM>(GAM + iL * nt2, V(lam, iL - 1), Vc(a_first, iL), V(phi, iL), n_tot, R, t / nct,
                              t % nct, ring);
            else if (which == 2)
                recur_task<T, TR, RM>(PHI + iR * nt2, V(phi, iR + 1), Vc(a_first, iR), V(phi, iR), n_tot, R, t / nct,
                              t % nct, ring);
            else
                recur_task<T, TR, RM>(PSI + iR * nt2, V(phi, iR + 1), Vc(a_last, iR), V(lam, iR), n_tot, R, t / nct, t % nct, ring);
        }
        grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    }
    // the middle slab: the left coupling (when c > 0), then the right one
    if (c > 0) {
        for (int task = blockIdx.x; task < 2 * ntile; task += gridDim.x) {
            const int t = task % ntile;
            if (task < ntile)
                recur_task<T, TR, RM>(GAM + c * nt2, V(lam, c - 1), Vc(a_first, c), V(phi, c), n_tot, R, t / nct, t % nct, ring);
            else
                recur_task<T, TR, RM>(LAM + c * nt2, V(lam, c - 1), Vc(a_last, c), V(lam, c), n_tot, R, t / nct, t % nct, ring);
        }
        grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    }
    for (int task = blockIdx.x; task < 2 * ntile; task += gridDim.x) {
        const int t = task % ntile;
        if (task < ntile)
            recur_task<T, TR, RM>(PHI + c * nt2, V(phi, c + 1), V(phi, c), V(phi, c), n_tot, R, t / nct, t % nct, ring);
        else
            recur_task<T, TR, RM>(PSI + c * nt2, V(phi, c + 1), V(lam, c), V(lam, c), n_tot, R, t / nct, t % nct, ring);
    }
    grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    for (int st = 0; st < S; ++st) {   // both fronts back toward the boundaries
        const int iL = c - 1 - st, iR = c + 1 + st;
        const bool onL = iL >= 1, onR = iR <= ns - 2;
        const int nw = onL + onR;
        for (int task = blockIdx.x; task < nw * ntile; task += gridDim.x) {
            const int t = task % ntile;
            const bool left = onL && task < ntile;
            if (left)
                recur_task<T, TR, RM>(PHI + iL * nt2, V(phi, iL + 1), V(phi, iL), V(phi, iL), n_tot, R, t / nct, t % nct, ring);
            else
                recur_task<T, TR, RM>(LAM + iR * nt2, V(lam, iR - 1), V(lam, iR), V(lam, iR), n_tot, R, t / nct, t % nct, ring);
        }
        grid_barrier_count(bar, (++nbar) * gridDim.x, err);
    }
}

// One interface recurrence over slabs i = i0, i0 + di, ... (nsteps of them):
//   out_i = base_i - M_i out_{i-di},  out_{i0-di} = init.
// One front: lambda forward (i = 1..l-2, M = Lambda, di = +1), phi backward
// (i = l-2..1, M = Phi, di = -1).  Two fronts run two chains at once, one per
// cluster of the launch.
template <typename C>
struct ChainSpec {
    const C* maps;      // M_i at maps + i n_tot^2
    const C* base;      // base_i at base + i n_tot R
    const C* init;
    C* out;
    int i0, nsteps, di;
};
template <typename C>
struct ChainPair {
    ChainSpec<C> c[2];
};

// One interface recurrence inside one thread-block cluster (the cluster's
// index in the launch selects the chain of the pair).
// Each CTA owns a block of rows of the n_tot x n_tot maps and keeps the current
// vector replicated in its shared memory; new entries are stored into every
// CTA's copy through distributed shared memory, and the cluster barrier closes
// each step.  Each warp owns at most RW (row, rhs) tasks and holds their next
// matrix rows (CW entries per lane) and base values in registers, loaded before
// the barrier so their latency overlaps it.
template <typename T, int RW, int CW, int NT>
__global__ void __launch_bounds__(NT) recur_chain_kernel(int n_tot, int R, ChainPair<cx<T>> P) {
    using C = cx<T>;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    const ChainSpec<C> S = P.c[blockIdx.x / CL];
    const C* __restrict__ maps = S.maps;
    const C* base = S.base;
    const C* __restrict__ init = S.init;
    C* out = S.out;
    extern __shared__ __align__(16) unsigned char smr[];
    C* vb = reinterpret_cast<C*>(smr);   // 2 x n_tot x R
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const int rows_per = (n_tot + CL - 1) / CL;
    const int r0 = min(n_tot, cr * rows_per), r1 = min(n_tot, r0 + rows_per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int ntask = (r1 - r0) * R;
    const int nsteps = S.nsteps;
    const int i0 = S.i0, di = S.di;
    C Mr[RW][CW];
    C bv[RW];

    auto prefetch = [&](int i) {
        const C* M = maps + (long long)i * nt2;
#pragma unroll
        for (int t = 0; t < RW; ++t) {
            const int task = warp + t * nw;
            const bool on = task < ntask;
            const int row = r0 + (on ? task / R : 0), rr = on ? task % R : 0;
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) {
                const int j = lane + 32 * cc;
                Mr[t][cc] = (on && j < n_tot) ? M[(long long)row * n_tot + j] : czero<C>();
            }
            bv[t] = on ? base[(long long)i * vec + (long long)row * R + rr] : czero<C>();
        }
    };

    // out_{i0 - di} = init, replicated into every CTA's vector
    const long long o0 = (long long)(i0 - di) * vec;
    for (long long e = threadIdx.x; e < vec; e += blockDim.x) vb[e] = init[e];
    if (out + o0 != init)
        for (long long e = (long long)r0 * R + threadIdx.x; e < (long long)r1 * R; e += blockDim.x) out[o0 + e] = init[e];
    if (nsteps >= 1) prefetch(i0);
    cl.sync();   // every CTA of the cluster is running before remote stores
    int cur = 0;
    for (int s = 0; s < nsteps; ++s) {
        const int i = i0 + s * di;
        C acc[RW];
#pragma unroll
        for (int t = 0; t < RW; ++t) {
            const int task = warp + t * nw;
            const int rr = task < ntask ? task % R : 0;
            const C* x = vb + cur * vec + rr;
            C a = czero<C>();
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) {
                const int j = lane + 32 * cc;
                if (j < n_tot) a = cfma(Mr[t][cc], x[(long long)j * R], a);
            }
            acc[t] = a;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int t = 0; t < RW; ++t) {
                acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, off);
                acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, off);
            }
#pragma unroll
        for (int t = 0; t < RW; ++t) {
            const int task = warp + t * nw;
            if (task < ntask && lane < CL) {
                const long long e = (long long)(r0 + task / R) * R + task % R;
                const C val = bv[t] - acc[t];
                if (lane == 0) out[(long long)i * vec + e] = val;
                C* dst = cl.map_shared_rank(vb, lane);
                dst[(cur ^ 1) * vec + e] = val;
            }
        }
        if (s + 1 < nsteps) prefetch(i + di);
        cl.sync();
        cur ^= 1;
    }
}

// The same recurrence with each CTA's rows of the next maps moved into a ring
// of shared-memory stages by TMA bulk copies, NB steps ahead (one thread issues,
// every thread waits on the stage's mbarrier, bounded); the dot products read
// the rows from shared memory, so the number of (row, rhs) tasks per warp is
// free.  The base values of a warp's first tasks are loaded one step ahead.
// Ring stage of the TMA recurrence kernel, in entries: a CTA's rows of one
// map plus one entry of alignment lead, rounded up to an even count so every
// stage starts on a 16-byte boundary.
LSS_HD inline long long recur_stage_ent(int rows_per, int n_tot) { return ((long long)rows_per * n_tot + 2) & ~1LL; }

template <typename T, int NT>
__global__ void __launch_bounds__(NT) recur_tma_kernel(int n_tot, int R, ChainPair<cx<T>> P, int nb, int* err) {
    using C = cx<T>;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    const ChainSpec<C> S = P.c[blockIdx.x / CL];
    const C* __restrict__ maps = S.maps;
    const C* base = S.base;
    const C* __restrict__ init = S.init;
    C* out = S.out;
    extern __shared__ __align__(128) unsigned char smr2[];
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const int rows_per = (n_tot + CL - 1) / CL;
    const int r0 = min(n_tot, cr * rows_per), r1 = min(n_tot, r0 + rows_per);
    const int nrow = r1 - r0;
    // a stage holds the CTA's rows of one map, copied from the 16-byte aligned
    // address at or before their first entry (rows of odd length in single
    // precision start on 8-byte boundaries) and rounded up to 16 bytes
    const long long stage_ent = recur_stage_ent(rows_per, n_tot);
    C* ring = reinterpret_cast<C*>(smr2);                 // nb x stage_ent
    C* vb = ring + nb * stage_ent;                        // 2 x n_tot x R
    __shared__ __align__(8) uint64_t full[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = NT >> 5;
    const int ntask = nrow * R;
    const int nsteps = S.nsteps;
    const int i0 = S.i0, di = S.di;
    auto lead_of = [&](int step) {   // entries between the aligned copy start and the CTA's first row
        const C* src = maps + (long long)(i0 + step * di) * nt2 + (long long)r0 * n_tot;
        return (int)((reinterpret_cast<uintptr_t>(src) & 15) / sizeof(C));
    };
    auto issue = [&](int step) {
        const int st = step % nb;
        const int lead = lead_of(step);
        const C* src = maps + (long long)(i0 + step * di) * nt2 + (long long)r0 * n_tot - lead;
        const unsigned bytes = (unsigned)((((long long)nrow * n_tot + lead) * sizeof(C) + 15) & ~15LL);
        mbar_expect_tx(&full[st], bytes);
        tma_load_1d(ring + st * stage_ent, src, bytes, &full[st]);
    };
    if (threadIdx.x == 0) {
        for (int st = 0; st < nb; ++st) mbar_init(&full[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && nrow > 0)
        for (int step = 0; step < nb && step < nsteps; ++step) issue(step);
    // out_{i0 - di} = init, replicated into every CTA's vector
    const long long o0 = (long long)(i0 - di) * vec;
    for (long long e = threadIdx.x; e < vec; e += NT) vb[e] = init[e];
    if (out + o0 != init)
        for (long long e = (long long)r0 * R + threadIdx.x; e < (long long)r1 * R; e += NT) out[o0 + e] = init[e];
    cl.sync();   // every CTA of the cluster is running before remote stores
    // base values of the warp's first BV tasks, one step ahead
    constexpr int BV = 4;
    C bvn[BV];
    auto load_bv = [&](int step) {
#pragma unroll
        for (int q = 0; q < BV; ++q) {
            const int t0 = warp + q * nw;
            bvn[q] = (t0 < ntask && step < nsteps)
                         ? base[(long long)(i0 + step * di) * vec + (long long)(r0 + t0 / R) * R + t0 % R]
                         : czero<C>();
        }
    };
    load_bv(0);
    bool ok = true;
    int cur = 0;
    for (int s = 0; s < nsteps; ++s) {
        const int i = i0 + s * di;
        const int st = s % nb;
        C bvc[BV];
#pragma unroll
        for (int q = 0; q < BV; ++q) bvc[q] = bvn[q];
        load_bv(s + 1);
        if (nrow > 0 && !mbar_wait(&full[st], (s / nb) & 1, err)) ok = false;
        const C* M = ring + st * stage_ent + lead_of(s);
        for (int t0 = warp, q = 0; t0 < ntask; t0 += nw, ++q) {
            const int rl = t0 / R, rr = t0 % R;
            const long long e = (long long)(r0 + rl) * R + rr;
            C bv;
            if (q < BV) {
#pragma unroll
                for (int u = 0; u < BV; ++u)
                    if (u == q) bv = bvc[u];
            } else {
                bv = base[(long long)i * vec + e];
            }
            const C* mrow = M + (long long)rl * n_tot;
            const C* x = vb + cur * vec + rr;
            C a0 = czero<C>(), a1 = czero<C>();
            int j = lane;
            for (; j + 32 < n_tot; j += 64) {
                a0 = cfma(mrow[j], x[(long long)j * R], a0);
                a1 = cfma(mrow[j + 32], x[(long long)(j + 32) * R], a1);
            }
            if (j < n_tot) a0 = cfma(mrow[j], x[(long long)j * R], a0);
            C acc = a0 + a1;
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane < CL) {
                const C val = bv - acc;
                if (lane == 0) out[(long long)i * vec + e] = val;
                C* dst = cl.map_shared_rank(vb, lane);
                dst[(cur ^ 1) * vec + e] = val;
            }
        }
        // once every thread of the cluster has arrived, this CTA's reads of the
        // stage and all remote stores of the new vector are done: refill the
        // stage with the rows of step s + nb
        cl.barrier_wait(cl.barrier_arrive());
        if (threadIdx.x == 0 && nrow > 0 && s + nb < nsteps) issue(s + nb);
        cur ^= 1;
    }
    if (!ok && threadIdx.x == 0) {
        // a wait expired: give the copies already issued a bounded chance to land
        const long long t0 = clock64();
        while (clock64() - t0 < 2000000ll) __nanosleep(1000);
    }
}

// out_i = base_i - M_i x_{i+dx} for slabs i = i_lo..i_hi, all independent
// (mu_i = first(a_i) - Gamma_i lambda_{i-1}; with two fronts also
// nu_i = last(a_i) - Psi_i phi_{i+1} and the middle slab's two couplings):
// one warp per (slab, row, rhs) dot product over the whole GPU.  out may be
// base (each entry is read, then written, by one warp); x is never out.
template <typename T>
__global__ void __launch_bounds__(256) recur_mu_kernel(int i_lo, int i_hi, int n_tot, int R, const cx<T>* __restrict__ maps,
                                                       const cx<T>* base, const cx<T>* __restrict__ xv, int dx,
                                                       cx<T>* out) {
    using C = cx<T>;
    const long long nt2 = (long long)n_tot * n_tot;
    const long long vec = (long long)n_tot * R;
    const long long task = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (task >= (long long)(i_hi - i_lo + 1) * vec) return;
    const int i = i_lo + (int)(task / vec);
    const long long rem = task % vec;
    const int row = (int)(rem / R), rr = (int)(rem % R);
    const C* lp = xv + (long long)(i + dx) * vec + rr;
    const C* Mrow = maps + (long long)i * nt2 + (long long)row * n_tot;
    C acc = czero<C>(), acc2 = czero<C>();
    int j = lane;
    for (; j + 32 < n_tot; j += 64) {
        acc = cfma(Mrow[j], lp[(long long)j * R], acc);
        acc2 = cfma(Mrow[j + 32], lp[(long long)(j + 32) * R], acc2);
    }
    if (j < n_tot) acc = cfma(Mrow[j], lp[(long long)j * R], acc);
    acc = acc + acc2;
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) out[(long long)i * vec + rem] = base[(long long)i * vec + rem] - acc;
}

// ---------------------------------------------------------------- host helpers
int ldwmax_of(const lss_ctx* c) {
    int w = 0;
    for (const auto& s : c->slabs) w = std::max(w, s.ldw);
    return w;
}
// Largest chunk row of any slab's factor stream, in complex entries.
long long max_row_ent(const lss_ctx* c) {
    long long m = 0;
    for (const auto& s : c->slabs) m = std::max<long long>(m, std::max<long long>(2LL * s.bs, 6LL * s.ldw + s.bs));
    return m;
}

// Opts kern into sh bytes of dynamic shared memory on the current device
// (once per size increase).
template <typename F>
int set_smem(lss_ctx* c, F kern, size_t sh) {
    std::lock_guard<std::mutex> lock(lss_config_mutex());
    long long& configured = lss_dev_cache((const void*)kern, 0);
    if ((long long)sh <= configured) return LSS_OK;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(sh, 48 * 1024));
    if (e) return lss_check_cuda(c, e, "shared memory attribute");
    configured = (long long)sh;
    return LSS_OK;
}

template <typename C>
CrArgs<C> base_args(lss_ctx* c) {
    CrArgs<C> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = c->n_slabs;
    A.n_tot = c->n_tot;
    A.n = c->n;
    A.b = c->b;
    A.R = 1;
    A.fac = (const C*)c->fac;
    A.coef = (const C*)c->coef;
    A.err = c->d_err;
    return A;
}

struct CrArgsTables {
    void* t16;
    void* t32;
    int n16, n32;
};

// Shared-memory plan of a solve launch: right-hand sides (bb bytes, in shared
// memory when they fit), per-group scratch (tb bytes) and the factor ring.
struct SolvePlan {
    int bsm, nst, stage_ent;
    size_t sh;
};
// ldw > 0: plan for slabs of that block width only.
template <typename C>
bool plan_solve(const lss_ctx* c, size_t bb, size_t tb, bool allow_smem_b, SolvePlan* P, int ldw = 0) {
    const long long row_ent = ldw > 0 ? std::max<long long>(2LL * ldw * ldw, 6LL * ldw + (long long)ldw * ldw)
                                      : max_row_ent(c);
    const size_t min_stage = sizeof(C) * (size_t)row_ent;
    const size_t want = std::max<size_t>(48 * 1024, min_stage);
    if (c->tune.solve_bsm == 0) allow_smem_b = false;
    const int tn = (ldw == 32 && c->tune.solve_nst_w) ? c->tune.solve_nst_w : c->tune.solve_nst;
    // half the budget leaves room for a second CTA on the SM (latency hiding)
    const size_t budget = c->tune.solve_half ? kSmemBudget / 2 : kSmemBudget;
    for (int bsm = allow_smem_b ? 1 : 0; bsm >= 0; --bsm) {
        const size_t fixed = tb + (bsm ? bb : 0);
        if (fixed + 2 * min_stage > budget) continue;
        const size_t avail = budget - fixed;
        int nst = (int)std::min<size_t>(4, avail / want);
        size_t stage = want;
        if (tn >= 2 && avail / tn >= min_stage) {   // tuned: tn stages sharing the free shared memory
            nst = tn;
            stage = (avail / tn) / 16 * 16;
        } else if (nst < 2) {
            nst = 2;
            stage = (avail / 2) / 16 * 16;
        }
        P->bsm = bsm;
        P->nst = nst;
        P->stage_ent = (int)(stage / sizeof(C)) & ~1;
        P->sh = fixed + (size_t)nst * P->stage_ent * sizeof(C);
        return true;
    }
    return false;
}

// Chunk tables (16- and 32-wide blocks) of one output kind and stage size,
// built and uploaded on first use (on stream s, ahead of the solves that read
// them: a copy on the legacy default stream would not be ordered before
// kernels on a non-blocking stream).
int chunk_tables(lss_ctx* c, bool part, int stage_ent, CrArgsTables* out, cudaStream_t s) {
    for (size_t q = 0; q < c->chunk_keys.size(); ++q)
        if (c->chunk_keys[q][0] == (part ? 1 : 0) && c->chunk_keys[q][1] == stage_ent) {
            out->t16 = c->chunk_dev[2 * q];
            out->t32 = c->chunk_dev[2 * q + 1];
            out->n16 = (int)c->chunk_keys[q][2];
            out->n32 = (int)c->chunk_keys[q][3];
            return LSS_OK;
        }
    const std::vector<CrChunk> t16 = cr_chunk_table(c->n_tot, 16, part, stage_ent, kSolveThreads / 16);
    const std::vector<CrChunk> t32 = cr_chunk_table(c->n_tot, 32, part, stage_ent, kSolveThreads / 32);
    void* d16 = nullptr;
    void* d32 = nullptr;
    cudaError_t e = cudaMalloc(&d16, t16.size() * sizeof(CrChunk));
    if (!e) e = cudaMalloc(&d32, t32.size() * sizeof(CrChunk));
    if (!e) e = cudaMemcpyAsync(d16, t16.data(), t16.size() * sizeof(CrChunk), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d32, t32.data(), t32.size() * sizeof(CrChunk), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);   // the host tables go out of scope
    if (e) {
        if (d16) cudaFree(d16);
        if (d32) cudaFree(d32);
        return lss_check_cuda(c, e, "chunk tables");
    }
    c->chunk_keys.push_back({part ? 1LL : 0LL, (long long)stage_ent, (long long)t16.size(), (long long)t32.size()});
    c->chunk_dev.push_back(d16);
    c->chunk_dev.push_back(d32);
    out->t16 = d16;
    out->t32 = d32;
    out->n16 = (int)t16.size();
    out->n32 = (int)t32.size();
    return LSS_OK;
}

// Launches the slab-solve kernel with per_cta complex entries of right-hand
// sides per CTA: in shared memory when they fit (and no fixed scratch is
// given), else in global scratch (the fixed array `scratch`, or the context's
// growable buffer).
// ldw > 0: the launch covers slabs of that block width only (its right-hand
// sides and stages are sized for it); z_off: byte offset of this launch's part
// of the context's global right-hand-side scratch.
template <typename T, int MODE, int NR = 1>
int launch_solve(lss_ctx* c, CrArgs<cx<T>> A, dim3 grid, long long per_cta, void* scratch, size_t scratch_bytes,
                 cudaStream_t s, int ldw = 0, size_t z_off = 0) {
    using C = cx<T>;
    auto kern = cr_solve_kernel<T, MODE, NR>;
    const size_t tb = sizeof(C) * ((size_t)kSolveThreads + kSplitRows * 4 * 32);
    const size_t bb = sizeof(C) * (size_t)per_cta;
    SolvePlan P;
    if (!plan_solve<C>(c, bb, tb, scratch == nullptr, &P, ldw))
        return lss_fail(c, LSS_ERR_UNSUPPORTED, "slab solve: the factor stream does not fit in shared memory");
    A.bstride = per_cta;
    A.bsm = P.bsm;
    A.nst = P.nst;
    A.stage_ent = P.stage_ent;
    CrArgsTables tabs;
    int rc = chunk_tables(c, MODE == CR_A, P.stage_ent, &tabs, s);
    if (rc) return rc;
    A.tab16 = (const CrChunk*)tabs.t16;
    A.tab32 = (const CrChunk*)tabs.t32;
    A.n16 = tabs.n16;
    A.n32 = tabs.n32;
    rc = set_smem(c, kern, P.sh);
    if (rc) return rc;
    if (!A.bsm) {
        const size_t need = bb * (size_t)grid.x * grid.y;
        if (scratch) {
            if (need > scratch_bytes)
                return lss_fail(c, LSS_ERR_UNSUPPORTED,
                                "apply_slab_noalloc: needs " + std::to_string(need) +
                                    " bytes of scratch, the fixed scratch holds " + std::to_string(scratch_bytes) +
                                    " (use fewer right-hand sides per call)");
            A.bg = (C*)scratch;
        } else {   // z_off: this launch's part of a scratch shared by concurrent launches
            rc = lss_grow(c, &c->z_buf, &c->z_cap, z_off + need);
            if (rc) return rc;
            A.bg = (C*)((char*)c->z_buf + z_off);
        }
    }
    kern<<<grid, kSolveThreads, P.sh, s>>>(A);
    return lss_check_cuda(c, cudaGetLastError(), "slab solve launch");
}

// ---------------------------------------------------------------- block LU slab solves (many right-hand sides)
// With at least kThMinR right-hand sides the 16-wide slabs are solved by the
// block LU factorization along x2 (block Thomas) instead of the cyclic
// reduction: its forward and backward sweeps are one dense (16 x 16)(16 x NRB)
// product per block row, so each factor entry read serves NRB right-hand
// sides from registers.  Bottom-up Schur complements (rows k = K-1 .. 0):
//   T_{K-1} = D_{K-1},  T_k = D_k + B_k Y_{k+1},  Y_k = -T_k^{-1} C_k,
// stored per block row as T_k^{-1}, V_k = -T_k^{-1} B_k and Y_k.  Solve:
//   q_{K-1} = T_{K-1}^{-1} f_{K-1},  q_k = T_k^{-1} f_k + V_k q_{k+1}   (bottom-up)
//   x_0 = q_0,  x_k = q_k + Y_k x_{k-1}                                  (top-down)
// (For the rows C_k x_{k-1} + D_k x_k + B_k x_{k+1} = f_k: from the bottom row
// up, T_k x_k + C_k x_{k-1} = g_k with g_{K-1} = f_{K-1} and
// g_k = f_k - B_k T_{k+1}^{-1} g_{k+1}; q_k = T_k^{-1} g_k.)  The
// factorization is a chain of K dependent 16 x 16 inversions per slab, one
// warp each (Gauss-Jordan with partial pivoting by warp reductions and
// shuffles): computed when a sweep first needs it, and from then on with
// every factorization, on its own stream.
constexpr int kThMinR = 16;
constexpr int kThThreads = 128;
constexpr int kThCoefMax = 16 * 9;

// A 16 x 16 complex matrix held by one warp: lane l owns row l % 16, columns
// 8 (l / 16) .. 8 (l / 16) + 7.
template <typename T>
struct WMat16 {
    cx<T> v[8];
};

__device__ __forceinline__ float2 shfl_c(float2 a, int src) {
    return make_float2(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src));
}
__device__ __forceinline__ double2 shfl_c(double2 a, int src) {
    return make_double2(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src));
}

// 1/a scaled by the larger component (no overflow or underflow in |a|^2).
template <typename C>
__device__ __forceinline__ C piv_recip(C a) {
    using T = decltype(a.x);
    const T s = T(1) / fmax(fabs(a.x), fabs(a.y));
    const T xs = a.x * s, ys = a.y * s;
    const T d = s / (xs * xs + ys * ys);
    return mk(xs * d, -ys * d);
}

// Warp-synchronous Gauss-Jordan inversion with partial pivoting (candidate of
// largest modulus by one warp reduction of a single-precision key, ties to the
// lower row; rows exchanged only when the pivot is off the diagonal).  On
// return the warp holds (P A)^{-1}; perm names, per row position, the row of A
// placed there, so that A^{-1} = (P A)^{-1} P.  sing: every candidate zero.
template <typename T>
__device__ __forceinline__ void warp_gj16(WMat16<T>& A, int& perm, bool& sing) {
    using C = cx<T>;
    const int lane = threadIdx.x & 31, r = lane & 15, h = lane >> 4;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int ih = i >> 3, iu = i & 7;
        const C ci = A.v[iu];
        unsigned key = 0;
        if (h == ih && r >= i) key = (__float_as_uint((float)cabs2(ci)) & ~31u) | (unsigned)(31 - r);
        key = __reduce_max_sync(0xffffffffu, key);
        const int p = 31 - (int)(key & 31u);
        sing |= (key >> 5) == 0u;
        if (p != i) {
            const int src = (r == i ? p : (r == p ? i : r)) + 16 * h;
#pragma unroll
            for (int u = 0; u < 8; ++u) A.v[u] = shfl_c(A.v[u], src);
            const int perm_i = __shfl_sync(0xffffffffu, perm, i), perm_p = __shfl_sync(0xffffffffu, perm, p);
            if (r == i) perm = perm_p;
            else if (r == p) perm = perm_i;
        }
        const C cn = A.v[iu];
        const C inv = piv_recip(shfl_c(cn, i + 16 * ih));
        const C f = shfl_c(cn, r + 16 * ih) * inv;   // A[r][i] / pivot
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const C pr = shfl_c(A.v[u], i + 16 * h);
            const int c = 8 * h + u;
            C nv = r == i ? pr * inv : A.v[u] - f * pr;
            if (c == i) nv = r == i ? inv : mk(-f.x, -f.y);
            A.v[u] = nv;
        }
    }
}

// Coefficient of row (r, k) toward unknown (a, k + slot - 1) of a w-wide
// subproblem: zero outside the w x w block and off the layer tridiagonal.
template <typename C>
__device__ __forceinline__ C th_cf(const C* row, int w, int r, int a, int slot) {
    if (r >= w || a < 0 || a >= w || a - r < -1 || a - r > 1) return czero<C>();
    return row[r * 9 + (a - r + 1) * 3 + slot];
}

// The bottom-up Schur chain of one 16-wide slab (one warp): T_k^{-1}, V_k, Y_k
// at th + i * 3 K 256 (three K x 256 arrays).  Layers w..15 are identity rows.
template <typename T>
__global__ void __launch_bounds__(32) th_chain_kernel(const SlabDev* __restrict__ slabs, const cx<T>* __restrict__ coef,
                                                      cx<T>* th, int K, int* err) {
    using C = cx<T>;
    constexpr int G = 16, LD = 17, GG = 256;
    const SlabDev sd = slabs[blockIdx.x];
    if (sd.ldw != 16) return;
    __shared__ C Ts[G * LD];
    __shared__ C Ys[GG];
    __shared__ __align__(16) C cr[2][kThCoefMax];
    __shared__ int ipos[G];
    const int w = sd.w, cs = sd.cstride;
    const int lane = threadIdx.x & 31, r = lane & 15, h = lane >> 4, cb = 8 * h;
    const C* cf = coef + sd.coef_off;
    C* Ti = th + (long long)blockIdx.x * 3 * K * GG;
    C* V = Ti + (long long)K * GG;
    C* Y = V + (long long)K * GG;
    auto fetch = [&](int t) {
        if (t < K) {
            const C* src = cf + (long long)(K - 1 - t) * cs;
            for (int e = lane; e < cs; e += 32) cp_async_entry(&cr[t & 1][e], src + e, true);
        }
        cp_async_commit();
    };
    fetch(0);
    bool sing = false;
    for (int t = 0; t < K; ++t) {
        const int k = K - 1 - t;
        cp_async_wait<0>();
        __syncwarp();   // row k staged; the previous step's reads of Ts, Ys and ipos done
        fetch(t + 1);
        const C* ck = cr[t & 1];
        WMat16<T> M;
#pragma unroll
        for (int u = 0; u < 8; ++u) {   // T_k = D_k + B_k Y_{k+1}
            const int c = cb + u;
            C v = czero<C>();
            if (r < w) {
                v = th_cf(ck, w, r, c, 1);
                if (t > 0 && c < w)
                    for (int a = max(0, r - 1); a <= min(w - 1, r + 1); ++a)
                        v = cfma(th_cf(ck, w, r, a, 2), Ys[a * G + c], v);
            } else if (r == c) {
                v.x = T(1);
            }
            M.v[u] = v;
        }
        int perm = r;
        warp_gj16<T>(M, perm, sing);
        __syncwarp();   // every lane's reads of Ys done
#pragma unroll
        for (int u = 0; u < 8; ++u) Ts[r * LD + cb + u] = M.v[u];
        if (h == 0) ipos[perm] = r;
        __syncwarp();
        const long long o = (long long)k * GG + r * G;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = cb + u;
            Ti[o + c] = Ts[r * LD + ipos[c]];
            C vb = czero<C>(), yc = czero<C>();
            if (c < w)
                for (int b = max(0, c - 1); b <= min(w - 1, c + 1); ++b) {
                    const C tb = Ts[r * LD + ipos[b]];
                    if (k + 1 < K) vb = cfma(tb, th_cf(ck, w, b, c, 2), vb);
                    if (k > 0) yc = cfma(tb, th_cf(ck, w, b, c, 0), yc);
                }
            V[o + c] = mk(-vb.x, -vb.y);
            Y[o + c] = mk(-yc.x, -yc.y);
            Ys[r * G + c] = mk(-yc.x, -yc.y);
        }
    }
    cp_async_wait<0>();
    if (sing && lane == 0) atomicOr(err, LSS_DERR_SINGULAR);
}

// The sweep passes on a run of 16-wide slabs by the block LU: CTA (column
// group, slab) solves NRB right-hand sides; thread (pg, cg) owns rows
// 4 pg .. 4 pg + 3 of columns 2 cg, 2 cg + 1 (a 4 x 2 register tile: per k
// of a product, four map entries and two vector entries serve eight
// multiply-adds).  The per-row maps arrive by cp.async one step ahead, the
// right-hand-side row is loaded one step ahead, q_k goes to a global scratch
// (read back by the same thread in the top-down sweep).
// Pass E's outputs on I go through a shared-memory buffer of kThYS block
// rows, so that each right-hand side's values of one x1 line leave as
// contiguous runs along x2 (the vector layout's fast index) instead of one
// scattered entry per block row.
constexpr int kThYS = 8;

template <int NRB>
constexpr size_t th_smem_entries() { return 4 * 16 * 17 + 4 * 16 * (size_t)NRB; }

template <typename T, int MODE, int NRB>
__global__ void __launch_bounds__(kThThreads) th_solve_kernel(CrArgs<cx<T>> A, const cx<T>* __restrict__ th,
                                                             cx<T>* qscr) {
    using C = cx<T>;
    constexpr int G = 16, LD = 17, GG = 256, PT = 4, CT = 2, NPG = G / PT, NCG = (NRB + CT - 1) / CT;
    constexpr int FE = (G * NRB + kThThreads - 1) / kThThreads;   // right-hand-side entries staged per thread
    static_assert(NPG * NCG <= kThThreads, "tile grid fits the CTA");
    extern __shared__ __align__(16) unsigned char smt[];
    C* Ms = reinterpret_cast<C*>(smt);   // [2 stages][2 maps][G x LD]
    C* Fs = Ms + 4 * G * LD;             // [2][G][NRB] right-hand-side rows
    C* Xs = Fs + 2 * G * NRB;            // [2][G][NRB] q / x rows
    C* Yb = Xs + 2 * G * NRB;            // pass E on I: [G][NRB][kThYS]
    const int K = A.n_tot, tid = threadIdx.x;
    const int i = A.slab0 + blockIdx.y, r0 = blockIdx.x * NRB;
    const SlabDev sd = A.slabs[i];
    const int w = sd.w, na = sd.na, ll = sd.ll;
    const int pg = tid % NPG, cg = tid / NPG, p0 = PT * pg, c0 = CT * cg;
    const bool act = cg < NCG;
    const C* Ti = th + (long long)i * 3 * K * GG;
    const C* V = Ti + (long long)K * GG;
    const C* Y = V + (long long)K * GG;
    C* q = qscr + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * K * G * NRB;
    const long long nt2 = (long long)K * K, vec = (long long)K * A.R;
    const C* cf = A.coef + sd.coef_off;
    // right-hand side entry (block row k, layer p, column c) of Algorithm 2's pass
    // Right-hand side entry (block row k, layer p, column c) of Algorithm 2's
    // pass, in two halves so that its loads stay in flight for a whole block
    // row: rhs_load issues them (the f value and, in pass E on the first or
    // last layer, the three coupling coefficients and neighbour values of
    // lambda_{i-1} or phi_{i+1}); rhs_value combines them one row later.  (A
    // one-layer slab needs both couplings on one entry: rare, combined at once.)
    struct RhsPre {
        C f, cc[3], nb[3];
    };
    auto rhs_load = [&](int k, int p, int c, RhsPre& o) {
        o.f = czero<C>();
#pragma unroll
        for (int d = 0; d < 3; ++d) o.cc[d] = o.nb[d] = czero<C>();
        const int rq = r0 + c;
        if (k < 0 || c >= NRB || rq >= A.R || p >= w) return;
        if (p >= na && p <= ll) o.f = A.f[(long long)rq * nt2 + (long long)k * K + sd.s + A.b + (p - na)];
        if (MODE != CR_E) return;
        const C* ck = cf + (long long)k * sd.cstride + p * 9;
        const bool left = p == na && i > 0, right = p == ll && i < A.n_slabs - 1;
        if (left && right) {   // both couplings on one entry: combined here, in the usual order
            C v = o.f;
            for (int dk = -1; dk <= 1; ++dk) {
                const int kk = k + dk;
                if (kk >= 0 && kk < K) v = cfnma(ck[dk + 1], A.lam[(long long)(i - 1) * vec + (long long)kk * A.R + rq], v);
            }
            for (int dk = -1; dk <= 1; ++dk) {
                const int kk = k + dk;
                if (kk >= 0 && kk < K) v = cfnma(ck[6 + dk + 1], A.phi[(long long)(i + 1) * vec + (long long)kk * A.R + rq], v);
            }
            o.f = v;
            return;
        }
        if (!left && !right) return;
        const C* nbv = left ? A.lam + (long long)(i - 1) * vec : A.phi + (long long)(i + 1) * vec;
        const int off = left ? 0 : 6;
#pragma unroll
        for (int dk = -1; dk <= 1; ++dk) {
            const int kk = k + dk;
            if (kk >= 0 && kk < K) {
                o.cc[dk + 1] = ck[off + dk + 1];
                o.nb[dk + 1] = nbv[(long long)kk * A.R + rq];
            }
        }
    };
    auto rhs_value = [&](const RhsPre& o) -> C {
        C v = o.f;
        if (MODE == CR_E) {
#pragma unroll
            for (int d = 0; d < 3; ++d) v = cfnma(o.cc[d], o.nb[d], v);
        }
        return v;
    };
    auto fetch = [&](int stage, const C* m0, const C* m1) {
        C* d = Ms + (size_t)stage * 2 * G * LD;
        for (int e = tid; e < GG; e += kThThreads) {
            cp_async_entry(d + (e >> 4) * LD + (e & 15), m0 + e, true);
            if (m1) cp_async_entry(d + G * LD + (e >> 4) * LD + (e & 15), m1 + e, true);
        }
        cp_async_commit();
    };
    RhsPre fr[FE];   // this thread's entries of the next row in flight: e = tid + 128 u -> (c = e / G, p = e % G)
    auto load_f = [&](int k) {
#pragma unroll
        for (int u = 0; u < FE; ++u) {
            const int e = tid + kThThreads * u;
            rhs_load(e < G * NRB ? k : -1, e % G, e / G, fr[u]);
        }
    };
    auto store_f = [&](int stage) {
#pragma unroll
        for (int u = 0; u < FE; ++u) {
            const int e = tid + kThThreads * u;
            if (e < G * NRB) Fs[stage * G * NRB + (e % G) * NRB + e / G] = rhs_value(fr[u]);
        }
    };
    // ---- bottom-up: q_k = T_k^{-1} f_k + V_k q_{k+1}
    load_f(K - 1);
    store_f(0);
    fetch(0, Ti + (long long)(K - 1) * GG, nullptr);
    load_f(K - 2);
    for (int s = 0; s < K; ++s) {
        const int k = K - 1 - s;
        cp_async_wait<0>();
        __syncthreads();   // maps and right-hand side of row k staged; q_{k+1} complete
        if (s + 1 < K) {
            fetch((s + 1) & 1, Ti + (long long)(k - 1) * GG, V + (long long)(k - 1) * GG);
            store_f((s + 1) & 1);
            load_f(k - 2);
        }
        if (act) {
            C acc[PT][CT];
#pragma unroll
            for (int a = 0; a < PT; ++a)
#pragma unroll
                for (int b = 0; b < CT; ++b) acc[a][b] = czero<C>();
            const C* M0 = Ms + (size_t)(s & 1) * 2 * G * LD;
            const C* F = Fs + (s & 1) * G * NRB;
#pragma unroll 4
            for (int a = 0; a < G; ++a) {
                C m[PT], x[CT];
#pragma unroll
                for (int u = 0; u < PT; ++u) m[u] = M0[(p0 + u) * LD + a];
#pragma unroll
                for (int b = 0; b < CT; ++b) x[b] = c0 + b < NRB ? F[a * NRB + c0 + b] : czero<C>();
#pragma unroll
                for (int u = 0; u < PT; ++u)
#pragma unroll
                    for (int b = 0; b < CT; ++b) acc[u][b] = cfma(m[u], x[b], acc[u][b]);
            }
            if (s > 0) {
                const C* M1 = M0 + G * LD;
                const C* X = Xs + ((s + 1) & 1) * G * NRB;
#pragma unroll 4
                for (int a = 0; a < G; ++a) {
                    C m[PT], x[CT];
#pragma unroll
                    for (int u = 0; u < PT; ++u) m[u] = M1[(p0 + u) * LD + a];
#pragma unroll
                    for (int b = 0; b < CT; ++b) x[b] = c0 + b < NRB ? X[a * NRB + c0 + b] : czero<C>();
#pragma unroll
                    for (int u = 0; u < PT; ++u)
#pragma unroll
                        for (int b = 0; b < CT; ++b) acc[u][b] = cfma(m[u], x[b], acc[u][b]);
                }
            }
            C* Xo = Xs + (s & 1) * G * NRB;
#pragma unroll
            for (int u = 0; u < PT; ++u)
#pragma unroll
                for (int b = 0; b < CT; ++b)
                    if (c0 + b < NRB) {
                        Xo[(p0 + u) * NRB + c0 + b] = acc[u][b];
                        q[((long long)k * G + p0 + u) * NRB + c0 + b] = acc[u][b];
                    }
        }
    }
    // ---- top-down: x_0 = q_0, x_k = q_k + Y_k x_{k-1}
    cp_async_wait<0>();
    __syncthreads();   // the bottom-up sweep's last reads of both stages are done
    fetch(0, Y + GG, nullptr);   // (row 0 needs no map; stage 0 holds Y_1 for s = 1)
    C qn[PT][CT];                // q_k of this thread's tile, loaded one row ahead
    auto load_q = [&](int k) {
#pragma unroll
        for (int u = 0; u < PT; ++u)
#pragma unroll
            for (int b = 0; b < CT; ++b)
                qn[u][b] = (act && k < K && c0 + b < NRB) ? q[((long long)k * G + p0 + u) * NRB + c0 + b] : czero<C>();
    };
    load_q(0);
    for (int s = 0; s < K; ++s) {
        const int k = s;
        cp_async_wait<0>();
        __syncthreads();
        if (s >= 1 && s + 1 < K) fetch(s & 1, Y + (long long)(k + 1) * GG, nullptr);   // Y_{k+1} into the other stage
        C acc[PT][CT];
#pragma unroll
        for (int u = 0; u < PT; ++u)
#pragma unroll
            for (int b = 0; b < CT; ++b) acc[u][b] = qn[u][b];
        load_q(k + 1);
        if (act) {
            if (s > 0) {
                const C* M = Ms + (size_t)((s - 1) & 1) * 2 * G * LD;   // Y_k
                const C* X = Xs + ((s + 1) & 1) * G * NRB;
#pragma unroll 4
                for (int a = 0; a < G; ++a) {
                    C m[PT], x[CT];
#pragma unroll
                    for (int u = 0; u < PT; ++u) m[u] = M[(p0 + u) * LD + a];
#pragma unroll
                    for (int b = 0; b < CT; ++b) x[b] = c0 + b < NRB ? X[a * NRB + c0 + b] : czero<C>();
#pragma unroll
                    for (int u = 0; u < PT; ++u)
#pragma unroll
                        for (int b = 0; b < CT; ++b) acc[u][b] = cfma(m[u], x[b], acc[u][b]);
                }
            }
            C* Xo = Xs + (s & 1) * G * NRB;
#pragma unroll
            for (int u = 0; u < PT; ++u) {
                const int p = p0 + u;
#pragma unroll
                for (int b = 0; b < CT; ++b) {
                    const int c = c0 + b, rq = r0 + c;
                    if (c >= NRB) continue;
                    Xo[p * NRB + c] = acc[u][b];
                    if (rq >= A.R) continue;
                    if (MODE == CR_A) {
                        const long long o = ((long long)i * K + k) * A.R + rq;
                        if (p == na) A.a_first[o] = acc[u][b];
                        if (p == ll) A.a_last[o] = acc[u][b];
                    } else if (p >= na && p <= ll) {
                        const int x1 = sd.s + (p - na);
                        if (A.y_grid) {
                            A.y[(long long)rq * nt2 + (long long)k * K + (x1 + A.b)] = to_d(acc[u][b]);
                        } else {
                            Yb[((p - na) * NRB + c) * kThYS + k % kThYS] = acc[u][b];
                        }
                    }
                }
            }
        }
        if (MODE == CR_E && !A.y_grid && (k % kThYS == kThYS - 1 || k == K - 1)) {
            // rows k0 .. k of every line x1 of D_i and right-hand side, x2 fastest
            __syncthreads();
            const int k0 = k - k % kThYS, nk = k - k0 + 1, nl = ll - na + 1;
            for (int e = tid; e < nl * NRB * kThYS; e += kThThreads) {
                const int kk = e % kThYS, c = (e / kThYS) % NRB, pl = e / (kThYS * NRB);
                const int rq = r0 + c, x1 = sd.s + pl, i2 = k0 + kk - A.b;
                if (kk < nk && rq < A.R && x1 >= 1 && x1 <= A.n && i2 >= 1 && i2 <= A.n) {
                    A.y[(long long)rq * A.n * A.n + (long long)(x1 - 1) * A.n + (i2 - 1)] =
                        to_d(Yb[(pl * NRB + c) * kThYS + kk]);
                }
            }
        }
    }
    cp_async_wait<0>();
}

// The sweep's slab solves run per run of consecutive slabs with the same
// block width, concurrently (run 0 on the caller's stream, the others on
// auxiliary streams): each launch sizes its right-hand sides and ring stages
// for its width (16-wide slabs need half the shared memory of 32-wide ones).
struct SweepRun { int s0, n, ldw; };
std::vector<SweepRun> sweep_runs(const lss_ctx* c) {
    std::vector<SweepRun> runs;
    for (int i = 0; i < c->n_slabs; ++i) {
        const int ldw = c->slabs[i].ldw;
        if (runs.empty() || runs.back().ldw != ldw) runs.push_back({i, 0, ldw});
        runs.back().n += 1;
    }
    return runs;
}

// Chunk tables of every solve plan the entry points can use (right-hand sides
// in shared or in global memory, all layers or first/last only, and the plans
// of the sweep's runs), built at factorization so that no later call allocates.
template <typename T>
int prepare_chunk_tables(lss_ctx* c, cudaStream_t s) {
    using C = cx<T>;
    const size_t tb = sizeof(C) * ((size_t)kSolveThreads + kSplitRows * 4 * 32);
    const size_t bb = sizeof(C) * (size_t)c->n_tot * ldwmax_of(c);
    std::vector<SolvePlan> plans;
    for (int smem_b = 0; smem_b < 2; ++smem_b) {
        SolvePlan P;
        if (plan_solve<C>(c, bb, tb, smem_b == 1, &P)) plans.push_back(P);
    }
    for (const SweepRun& u : sweep_runs(c)) {
        SolvePlan P;
        for (int nr = 1; nr <= (u.ldw == 16 ? 2 : 1); ++nr)   // one or two right-hand sides per CTA
            for (int smem_b = 0; smem_b < 2; ++smem_b)
                if (plan_solve<C>(c, sizeof(C) * (size_t)nr * c->n_tot * u.ldw, tb, smem_b == 1, &P, u.ldw))
                    plans.push_back(P);
    }
    for (const SolvePlan& P : plans)
        for (int part = 0; part < 2; ++part) {
            CrArgsTables t;
            const int rc = chunk_tables(c, part == 1, P.stage_ent, &t, s);
            if (rc) return rc;
        }
    return LSS_OK;
}

// One sweep pass (MODE CR_A or CR_E) over every slab, run by run.
// Block LU solves switched off by LSS_SLAB_SOLVE=cr (cyclic reduction for every run).
bool thomas_enabled() {
    const char* v = std::getenv("LSS_SLAB_SOLVE");
    return !(v && v[0] == 'c');
}

// Columns per CTA of the block LU solves: 16 (at n = 512 with 64 right-hand
// sides, 32 per CTA took 15.6 + 29.8 ms for the step's passes A and E, 16
// took 15.1 + 18.9 ms: twice the CTAs, and pass E's output staging keeps
// more of them resident).
int th_nrb(int) { return 16; }

// The block LU factors of every 16-wide slab (one warp per slab).  Called
// when a sweep with many right-hand sides finds them missing; once a context
// has used them, each later factorization computes them beside the cyclic
// reduction and the interface maps (th_wanted), on an auxiliary stream.
template <typename T>
int thomas_prepare_t(lss_ctx* c, cudaStream_t s) {
    using C = cx<T>;
    c->th_wanted = true;
    if (c->th_valid) return LSS_OK;
    const size_t bytes = sizeof(C) * (size_t)c->n_slabs * 3 * c->n_tot * 256;
    int rc = lss_grow(c, &c->th_buf, &c->th_cap, bytes);
    if (rc) return rc;
    ProfScope ps(c, s, LSS_PROF_FACTOR, 1);
    th_chain_kernel<T><<<c->n_slabs, 32, 0, s>>>(c->d_slabs, (const C*)c->coef, (C*)c->th_buf, c->n_tot, c->d_err);
    rc = lss_check_cuda(c, cudaGetLastError(), "block LU factorization launch");
    if (!rc) c->th_valid = true;
    return rc;
}

// One run of nsl 16-wide slabs (from A.slab0) solved by the block LU; its
// q scratch at tq_buf + q_off bytes.
template <typename T, int MODE, int NRB>
int launch_thomas_nrb(lss_ctx* c, const CrArgs<cx<T>>& A, int nsl, int R, cudaStream_t s, size_t q_off) {
    using C = cx<T>;
    const size_t sh = sizeof(C) * th_smem_entries<NRB>() + (MODE == CR_E ? sizeof(C) * 16 * NRB * kThYS : 0);
    int rc = set_smem(c, th_solve_kernel<T, MODE, NRB>, sh);
    if (rc) return rc;
    th_solve_kernel<T, MODE, NRB><<<dim3((R + NRB - 1) / NRB, nsl), kThThreads, sh, s>>>(
        A, (const C*)c->th_buf, (C*)((char*)c->tq_buf + q_off));
    return lss_check_cuda(c, cudaGetLastError(), "block LU solve launch");
}

template <typename T, int MODE>
int launch_thomas(lss_ctx* c, const CrArgs<cx<T>>& A, int nsl, int R, cudaStream_t s, size_t q_off) {
    return launch_thomas_nrb<T, MODE, 16>(c, A, nsl, R, s, q_off);
}

// q scratch bytes of one run's block LU solves.
template <typename T>
size_t thomas_scratch(const lss_ctx* c, int nsl, int R) {
    const int nrb = th_nrb(R);
    return sizeof(cx<T>) * (size_t)((R + nrb - 1) / nrb) * nsl * c->n_tot * 16 * nrb;
}

template <typename T, int MODE>
int sweep_pass(lss_ctx* c, CrArgs<cx<T>> A, int R, cudaStream_t s, bool thomas = false) {
    const std::vector<SweepRun> runs = sweep_runs(c);
    int rc = lss_ensure_aux(c, runs.size());
    if (rc) return rc;
    // 16-wide runs by the block LU when the caller prepared its factors
    auto th_run = [&](const SweepRun& u) { return thomas && u.ldw == 16; };
    size_t qtot = 0;
    std::vector<size_t> qoff(runs.size());
    for (size_t ri = 0; ri < runs.size(); ++ri) {
        qoff[ri] = qtot;
        if (th_run(runs[ri])) qtot += thomas_scratch<T>(c, runs[ri].n, R);
    }
    if (qtot && (rc = lss_grow(c, &c->tq_buf, &c->tq_cap, qtot))) return rc;
    // global right-hand-side scratch of every run, grown before any launch so
    // that concurrent runs use disjoint parts of one buffer
    // right-hand sides per CTA: two on 16-wide runs when the autotuner chose so
    auto nr_of = [&](const SweepRun& u) { return (c->tune.solve_nr == 2 && u.ldw == 16 && R >= 2) ? 2 : 1; };
    size_t ztot = 0;
    std::vector<size_t> zoff(runs.size());
    for (size_t ri = 0; ri < runs.size(); ++ri) {
        const int nr = nr_of(runs[ri]);
        zoff[ri] = ztot;
        ztot += sizeof(cx<T>) * (size_t)c->n_tot * runs[ri].ldw * nr * ((R + nr - 1) / nr) * runs[ri].n;
    }
    if ((rc = lss_grow(c, &c->z_buf, &c->z_cap, ztot))) return rc;
    if (runs.size() > 1) cudaEventRecord(c->fork_event, s);
    for (size_t ri = 0; ri < runs.size() && !rc; ++ri) {
        const SweepRun& u = runs[ri];
        cudaStream_t su = ri == 0 ? s : c->aux_stream[ri - 1];
        if (ri > 0) cudaStreamWaitEvent(su, c->fork_event, 0);
        CrArgs<cx<T>> Ar = A;
        Ar.slab0 = u.s0;
        if (th_run(u))
            rc = launch_thomas<T, MODE>(c, Ar, u.n, R, su, qoff[ri]);
        else if (nr_of(u) == 2)
            rc = launch_solve<T, MODE, 2>(c, Ar, dim3((R + 1) / 2, u.n), 2LL * c->n_tot * u.ldw, nullptr, 0, su, u.ldw,
                                          zoff[ri]);
        else
            rc = launch_solve<T, MODE>(c, Ar, dim3(R, u.n), (long long)c->n_tot * u.ldw, nullptr, 0, su, u.ldw,
                                       zoff[ri]);
        if (ri > 0) {
            cudaEventRecord(c->aux_event[ri - 1], su);
            cudaStreamWaitEvent(s, c->aux_event[ri - 1], 0);
        }
    }
    return rc;
}

template <typename T>
int factor_impl(lss_ctx* c, cudaStream_t s) {
    int rc0 = prepare_chunk_tables<T>(c, s);
    if (rc0) return rc0;
    using C = cx<T>;
    const int K0 = c->n_tot, ns = c->n_slabs, nlev = cr_levels(K0);
    C* fac = (C*)c->fac;
    C* work = (C*)c->cr_work;
    // runs of consecutive slabs with the same block width: each run's launches
    // size their shared memory for the run's widest slab (occupancy)
    struct Run { int s0, n, w; };
    std::vector<Run> runs;
    for (int i = 0; i < ns; ++i) {
        if (runs.empty() || c->slabs[i].ldw != c->slabs[runs.back().s0].ldw) runs.push_back({i, 0, 0});
        runs.back().n += 1;
        runs.back().w = std::max(runs.back().w, c->slabs[i].w);
    }
    auto shgw_of = [](int w) { return sizeof(C) * (size_t)w * (4 * w + 1); };
    const size_t shew = sizeof(C) * (size_t)6 * 32 * 33;
    int rc = set_smem(c, cr_gjw_kernel<T>, shgw_of(32));
    if (!rc) rc = set_smem(c, cr_evenw_kernel<T>, shew);
    if (rc) return rc;
    // slabs factor independently: run 0 on s, every other run on an auxiliary
    // stream of its own, forked after the level-0 blocks are built and joined
    // before the interface maps
    if ((rc = lss_ensure_aux(c, runs.size() + 1))) return rc;
    // the block LU factors (when this context's sweeps use them) on the last
    // auxiliary stream, joined at the end of the factorization
    const bool chain = c->th_wanted && thomas_enabled();
    cudaStream_t sch = c->aux_stream[runs.size() - 1];
    if (chain) {
        if ((rc = lss_grow(c, &c->th_buf, &c->th_cap, sizeof(C) * (size_t)ns * 3 * K0 * 256))) return rc;
        cudaEventRecord(c->fork_event, s);
        cudaStreamWaitEvent(sch, c->fork_event, 0);
        th_chain_kernel<T><<<ns, 32, 0, sch>>>(c->d_slabs, (const C*)c->coef, (C*)c->th_buf, K0, c->d_err);
        if ((rc = lss_check_cuda(c, cudaGetLastError(), "block LU factorization launch"))) return rc;
    }
    {
        ProfScope ps(c, s, LSS_PROF_FACTOR, 2 + (2 * nlev) * (int)runs.size() + (chain ? 1 : 0));
        cr_build0_kernel<T><<<dim3(K0, ns), 128, 0, s>>>(c->d_slabs, (const C*)c->coef, work, fac, K0);
        cudaEventRecord(c->fork_event, s);
        for (size_t ri = 0; ri < runs.size(); ++ri) {
            const Run& u = runs[ri];
            cudaStream_t su = ri == 0 ? s : c->aux_stream[ri - 1];
            if (ri > 0) cudaStreamWaitEvent(su, c->fork_event, 0);
            for (int l = 0; l < nlev; ++l) {
                const int K = cr_level(K0, l).K;
                const int nodd = K / 2, nev = (K + 1) / 2;
                if (l == 0)
                    cr_gj0_kernel<T><<<(nodd * u.n + kGj0Warps - 1) / kGj0Warps, 32 * kGj0Warps, 0, su>>>(
                        c->d_slabs, (const C*)c->coef, fac, work, K0, nodd, u.s0, u.n, c->d_err);
                else
                    cr_gjw_kernel<T><<<nodd * u.n, kWideThreads, shgw_of(u.w), su>>>(
                        c->d_slabs, fac, work, c->work_len, K0, l, nodd, u.s0, 0, 4 * u.w + 1, c->d_err);
                cr_evenw_kernel<T><<<nev * u.n, kWideThreads, shew, su>>>(c->d_slabs, fac, work, c->work_len, K0,
                                                                         l, nev, u.s0, nlev);
            }
            cr_gjw_kernel<T><<<u.n, kWideThreads, shgw_of(u.w), su>>>(c->d_slabs, fac, work, c->work_len, K0, nlev, 1,
                                                                      u.s0, 1, 4 * u.w + 1, c->d_err);
            if (ri > 0) {
                cudaEventRecord(c->aux_event[ri - 1], su);
                cudaStreamWaitEvent(s, c->aux_event[ri - 1], 0);
            }
        }
    }
    rc = lss_check_cuda(c, cudaGetLastError(), "factor launch");
    if (!rc && ns > 1) rc = lss_iface_maps(c, s);
    if (chain) {   // join the block LU chain (also on an error, so that nothing is left in flight)
        cudaEventRecord(c->aux_event[runs.size() - 1], sch);
        cudaStreamWaitEvent(s, c->aux_event[runs.size() - 1], 0);
        if (!rc) c->th_valid = true;
    }
    return rc;
}

// Cluster size for the recurrence kernels: 16 CTAs when the GPU can
// co-schedule them (non-portable size), else 8.  Returns LSS_ERR_UNSUPPORTED
// when a warp would own more rows than its prefetch registers hold, so the
// caller uses the grid kernel.
template <typename T, int RW, int CW, int NT>
int launch_chain_cfg(lss_ctx* c, const ChainPair<cx<T>>& P, int nchains, int R, cudaStream_t s) {
    const size_t sh = 2 * (size_t)c->n_tot * R * sizeof(cx<T>);
    auto kern = recur_chain_kernel<T, RW, CW, NT>;
    std::unique_lock<std::mutex> lock(lss_config_mutex());
    long long& configured = lss_dev_cache((const void*)kern, 0);   // shared memory opted into
    long long& cl_size = lss_dev_cache((const void*)kern, 1);      // cluster size that co-schedules
    if ((long long)sh > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sh, 48 * 1024));
        if (!e) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e) return lss_check_cuda(c, e, "recurrence attribute");
        configured = (long long)sh;
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
    const int cl = (int)cl_size;
    lock.unlock();
    const int rows_per = (c->n_tot + cl - 1) / cl;
    if ((rows_per * R + NT / 32 - 1) / (NT / 32) > RW || c->n_tot > 32 * CW) return LSS_ERR_UNSUPPORTED;
    attr[0].val.clusterDim.x = cl;
    cfg.gridDim = dim3(cl * nchains);
    int nt = c->n_tot;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, nt, R, P);
    return lss_check_cuda(c, e, "recurrence cluster launch");
}

// TMA-ring version: 16-CTA clusters (8 when 16 cannot be co-scheduled), as
// many ring stages (2..3) as fit beside the vectors.  LSS_ERR_UNSUPPORTED when
// even two stages do not fit.
template <typename T>
int launch_chain_tma(lss_ctx* c, const ChainPair<cx<T>>& P, int nchains, int R, cudaStream_t s) {
    using C = cx<T>;
    constexpr int NT = sizeof(T) == 8 ? 512 : 1024;   // a warp per (row, rhs) task where possible
    auto kern = recur_tma_kernel<T, NT>;
    std::unique_lock<std::mutex> lock(lss_config_mutex());
    long long& attr_done = lss_dev_cache((const void*)kern, 0);
    long long& cl_size = lss_dev_cache((const void*)kern, 1);   // cluster size that co-schedules
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (!e) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e) return lss_check_cuda(c, e, "recurrence attribute");
        attr_done = 1;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(NT);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto smem_for = [&](int cls, int nb) {
        const int rows_per = (c->n_tot + cls - 1) / cls;
        return sizeof(C) * (size_t)(nb * recur_stage_ent(rows_per, c->n_tot) + 2LL * c->n_tot * R);
    };
    if (!cl_size) {
        for (int cand : {16, 8}) {
            attr[0].val.clusterDim.x = cand;
            cfg.gridDim = dim3(cand);
            cfg.dynamicSmemBytes = smem_for(cand, 2);
            int nclusters = 0;
            cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, (void*)kern, &cfg);
            if (!e && nclusters > 0) { cl_size = cand; break; }
            cudaGetLastError();
        }
        if (!cl_size) return LSS_ERR_UNSUPPORTED;
    }
    const int cl = (int)cl_size;
    lock.unlock();
    int nb = c->tune.rec_nb ? std::min(c->tune.rec_nb, 4) : 3;   // full[] holds at most 4 stages
    while (nb >= 2 && smem_for(cl, nb) > (size_t)220 * 1024) --nb;
    if (nb < 2) return LSS_ERR_UNSUPPORTED;
    attr[0].val.clusterDim.x = cl;
    cfg.gridDim = dim3(cl * nchains);
    cfg.dynamicSmemBytes = smem_for(cl, nb);
    int nt = c->n_tot;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, nt, R, P, nb, c->d_err);
    return lss_check_cuda(c, e, "recurrence cluster launch");
}

// One launch running nchains (1 or 2) independent chains, one cluster each.
template <typename T>
int launch_chains(lss_ctx* c, const ChainPair<cx<T>>& P, int nchains, int R, cudaStream_t s) {
    const int rc = launch_chain_tma<T>(c, P, nchains, R, s);
    if (rc != LSS_ERR_UNSUPPORTED) return rc;
    if constexpr (sizeof(T) == 4) {
        if (c->n_tot <= 384) return launch_chain_cfg<T, 3, 12, 256>(c, P, nchains, R, s);
        return launch_chain_cfg<T, 3, 20, 384>(c, P, nchains, R, s);
    } else {
        return launch_chain_cfg<T, 3, 9, 256>(c, P, nchains, R, s);
    }
}

template <typename T>
int launch_chain(lss_ctx* c, const cx<T>* maps, const cx<T>* base, const cx<T>* init, cx<T>* out, int backward, int R,
                 cudaStream_t s) {
    const int ns = c->n_slabs;
    ChainPair<cx<T>> P{};
    P.c[0] = ChainSpec<cx<T>>{maps, base, init, out, backward ? ns - 2 : 1, ns - 2, backward ? -1 : 1};
    return launch_chains<T>(c, P, 1, R, s);
}

template <typename T>
int launch_products(lss_ctx* c, int i_lo, int i_hi, const cx<T>* maps, const cx<T>* base, const cx<T>* x, int dx,
                    cx<T>* out, int R, cudaStream_t s) {
    if (i_hi < i_lo) return LSS_OK;
    const long long warps = (long long)(i_hi - i_lo + 1) * c->n_tot * R;
    recur_mu_kernel<T><<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(i_lo, i_hi, c->n_tot, R, maps, base, x, dx, out);
    return lss_check_cuda(c, cudaGetLastError(), "recurrence products launch");
}

// The two-front recurrences (see recur_grid2_kernel) with the cluster chains:
// both forward chains in one launch, the middle slab and mu / nu, both
// backward chains in one launch.
template <typename T>
int launch_recur2_chains(lss_ctx* c, const cx<T>* ifc, cx<T>* lam, cx<T>* phi, const cx<T>* a_first,
                         const cx<T>* a_last, int R, cudaStream_t s) {
    using C = cx<T>;
    const long long nt2 = (long long)c->n_tot * c->n_tot;
    const long long vec = (long long)c->n_tot * R;
    const int ns = c->n_slabs, m = c->mid;
    const C* LAM = ifc;
    const C* GAM = ifc + ns * nt2;
    const C* PHI = ifc + 2LL * ns * nt2;
    const C* PSI = ifc + 3LL * ns * nt2;
    ChainPair<C> F{};
    F.c[0] = ChainSpec<C>{LAM, a_last, a_last, lam, 1, std::max(0, m - 1), 1};
    F.c[1] = ChainSpec<C>{PHI, a_first, a_first + (ns - 1) * vec, phi, ns - 2, ns - 2 - m, -1};
    int rc = launch_chains<T>(c, F, 2, R, s);
    if (rc) return rc;
    if (m > 0) {
        rc = launch_products<T>(c, 1, m - 1, GAM, a_first, lam, -1, phi, R, s);                  // mu
        if (!rc) rc = launch_products<T>(c, m, m, GAM, a_first, lam, -1, phi, R, s);
        if (!rc) rc = launch_products<T>(c, m, m, LAM, a_last, lam, -1, lam, R, s);
    } else {
        rc = lss_check_cuda(c, cudaMemcpyAsync(phi, a_first, vec * sizeof(C), cudaMemcpyDeviceToDevice, s),
                            "recurrence copy");
    }
    if (!rc) rc = launch_products<T>(c, m + 1, ns - 2, PSI, a_last, phi, 1, lam, R, s);          // nu
    if (!rc) rc = launch_products<T>(c, m, m, PHI, phi, phi, 1, phi, R, s);
    if (!rc) rc = launch_products<T>(c, m, m, PSI, lam, phi, 1, lam, R, s);
    if (rc) return rc;
    ChainPair<C> B{};
    B.c[0] = ChainSpec<C>{PHI, phi, phi + m * vec, phi, m - 1, std::max(0, m - 1), -1};
    B.c[1] = ChainSpec<C>{LAM, lam, lam + m * vec, lam, m + 1, ns - 2 - m, 1};
    return launch_chains<T>(c, B, 2, R, s);
}

// lambda chain, mu for every slab, phi chain (three launches), or the
// cooperative grid kernel when the vectors do not fit the cluster kernels.
template <typename T>
int launch_recur(lss_ctx* c, const cx<T>* ifc, cx<T>* lam, cx<T>* phi, const cx<T>* a_first, const cx<T>* a_last,
                 int R, cudaStream_t s) {
    using C = cx<T>;
    const long long nt2 = (long long)c->n_tot * c->n_tot;
    const long long vec = (long long)c->n_tot * R;
    const int ns = c->n_slabs;
    const bool two = c->fronts == 2;
    const size_t sh = 2 * (size_t)c->n_tot * R * sizeof(C);
    if (sh <= (size_t)200 * 1024) {
        if (two) {
            const int m = c->mid;
            const int nl = 4 + (m > 0 ? 2 + (m > 1) : 0) + (ns - 2 >= m + 1);
            ProfScope ps(c, s, LSS_PROF_RECUR, nl);
            const int rc = launch_recur2_chains<T>(c, ifc, lam, phi, a_first, a_last, R, s);
            if (rc != LSS_ERR_UNSUPPORTED) return rc;
        } else {
            ProfScope ps(c, s, LSS_PROF_RECUR, 3);
            int rc = launch_chain<T>(c, ifc, a_last, a_last, lam, 0, R, s);
            if (rc == LSS_OK) {
                rc = launch_products<T>(c, 1, ns - 1, ifc + ns * nt2, a_first, lam, -1, phi, R, s);   // mu
                if (rc) return rc;
                return launch_chain<T>(c, ifc + 2LL * ns * nt2, phi, phi + (long long)(ns - 1) * vec, phi, 1, R, s);
            }
            if (rc != LSS_ERR_UNSUPPORTED) return rc;
        }
    }
    // a grid-synchronised kernel is not put into a captured graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap != cudaStreamCaptureStatusNone) return LSS_ERR_UNSUPPORTED;
    // tiles of the widest step (lambda and mu with one front, both fronts' two
    // products with two): with up to 8 right-hand sides, 16-row tiles of every
    // column (recur_rows); else 64 x 16 tiles when they cover at least half the
    // SMs (two 32-row tiles on one SM take longer than one 64-row tile), else 32 x 16
    const long long prods = two ? 4 : 2;
    const int RM = R == 1 ? 1 : R == 2 ? 2 : R <= 4 ? 4 : R <= 8 ? 8 : 0;
    const long long nct = RM ? 1 : (R + kGtC - 1) / kGtC;
    const int TR = RM ? 16 : 2 * prods * ((c->n_tot + 63) / 64) * nct >= c->num_sms ? 64 : 32;
    const size_t smem = RM ? 0 : (size_t)kGtS * (TR == 64 ? gt_stage_ent<64>() : gt_stage_ent<32>()) * sizeof(C);
    const int var = RM ? 2 + (RM == 1 ? 0 : RM == 2 ? 1 : RM == 4 ? 2 : 3) : TR == 64;
    using KernPtr = const void*;
    const KernPtr k1[6] = {(KernPtr)recur_grid_kernel<T, 32, 0>, (KernPtr)recur_grid_kernel<T, 64, 0>,
                           (KernPtr)recur_grid_kernel<T, 16, 1>, (KernPtr)recur_grid_kernel<T, 16, 2>,
                           (KernPtr)recur_grid_kernel<T, 16, 4>, (KernPtr)recur_grid_kernel<T, 16, 8>};
    const KernPtr k2[6] = {(KernPtr)recur_grid2_kernel<T, 32, 0>, (KernPtr)recur_grid2_kernel<T, 64, 0>,
                           (KernPtr)recur_grid2_kernel<T, 16, 1>, (KernPtr)recur_grid2_kernel<T, 16, 2>,
                           (KernPtr)recur_grid2_kernel<T, 16, 4>, (KernPtr)recur_grid2_kernel<T, 16, 8>};
    const void* k = two ? k2[var] : k1[var];
    int grid_now;
    {
        std::lock_guard<std::mutex> lock(lss_config_mutex());
        long long& g = lss_dev_cache(k, 0);   // co-resident CTAs on this device
        if (!g) {
            if (smem) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e) return lss_check_cuda(c, e, "recurrence attribute");
            }
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 256, smem);
            g = (long long)std::max(1, per) * c->num_sms;
        }
        grid_now = (int)g;
    }
    const long long tiles = prods * ((c->n_tot + TR - 1) / TR) * nct;
    int nb = (int)std::min<long long>(grid_now, std::max<long long>(1, tiles));
    int nsl = c->n_slabs, nt = c->n_tot, mid = c->mid;
    unsigned* bar = c->d_bar;
    int* err = c->d_err;
    ProfScope ps(c, s, LSS_PROF_RECUR, 1);
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);   // the barriers' arrival counter
    if (e) return lss_check_cuda(c, e, "recurrence barrier");
    if (two) {
        void* args[] = {&nsl, &mid, &nt, &R, &ifc, (void*)&a_first, (void*)&a_last, &lam, &phi, &bar, &err};
        e = cudaLaunchCooperativeKernel(k, dim3(nb), dim3(256), args, smem, s);
    } else {
        void* args[] = {&nsl, &nt, &R, &ifc, (void*)&a_first, (void*)&a_last, &lam, &phi, &bar, &err};
        e = cudaLaunchCooperativeKernel(k, dim3(nb), dim3(256), args, smem, s);
    }
    return lss_check_cuda(c, e, "recurrence launch");
}

__global__ void grid_to_working(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// The sweep of Algorithm 2: on r (vectors on I: f = Q r, result restricted to
// I), or, with grid_in, on a right-hand side given on the grid, the result
// then on the grid too (every point of every D_i, x2 slowest).
template <typename T>
int sweep_impl(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s, const double2* grid_in = nullptr) {
    using C = cx<T>;
    const long long nt2 = (long long)c->n_tot * c->n_tot;
    int rc = lss_grow(c, &c->f_buf, &c->f_cap, (size_t)R * nt2 * sizeof(C));
    if (rc) return rc;
    const long long vec = (long long)c->n_tot * R;
    rc = lss_grow(c, &c->side_buf, &c->side_cap, 4 * (size_t)c->n_slabs * vec * sizeof(C));
    if (rc) return rc;
    if (grid_in) {
        ProfScope ps(c, s, LSS_PROF_SPARSIFY, 1);
        if constexpr (sizeof(T) == 8)
            rc = lss_check_cuda(c, cudaMemcpyAsync(c->f_buf, grid_in, (size_t)R * nt2 * sizeof(double2),
                                                   cudaMemcpyDeviceToDevice, s), "grid right-hand side");
        else {
            grid_to_working<<<4 * c->num_sms, 256, 0, s>>>(grid_in, (float2*)c->f_buf, (long long)R * nt2);
            rc = lss_check_cuda(c, cudaGetLastError(), "grid right-hand side");
        }
    } else {
        rc = lss_sparsify(c, r, c->f_buf, R, s);
    }
    if (rc) return rc;
    C* side = (C*)c->side_buf;
    CrArgs<C> A = base_args<C>(c);
    A.R = R;
    A.f = (const C*)c->f_buf;
    A.a_first = side;
    A.a_last = side + c->n_slabs * vec;
    C* lam = side + 2 * c->n_slabs * vec;
    C* phi = side + 3 * c->n_slabs * vec;
    A.lam = lam;
    A.phi = phi;
    A.y = y;
    A.y_grid = grid_in ? 1 : 0;
    const int nrun = (int)sweep_runs(c).size();
    // block LU solves for the 16-wide slabs with many right-hand sides; their
    // factors are computed here when missing, but never inside a stream
    // capture (a captured sweep without them uses the cyclic reduction)
    bool thomas = R >= kThMinR && thomas_enabled();
    if (thomas && !c->th_valid) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cap);
        if (cap != cudaStreamCaptureStatusNone) thomas = false;
        else if ((rc = thomas_prepare_t<T>(c, s))) return rc;
    }
    if (c->n_slabs > 1) {
        {
            ProfScope ps(c, s, LSS_PROF_SLAB_A, nrun);
            rc = sweep_pass<T, CR_A>(c, A, R, s, thomas);
        }
        if (rc) return rc;
        rc = launch_recur<T>(c, (const C*)c->iface, lam, phi, A.a_first, A.a_last, R, s);
        if (rc) return rc;
    }
    ProfScope ps(c, s, LSS_PROF_SLAB_E, nrun);
    return sweep_pass<T, CR_E>(c, A, R, s, thomas);
}

template <typename T>
int slab_apply_impl(lss_ctx* c, int slab, const double2* v, double2* w, int R, void* scratch, size_t scratch_bytes,
                    cudaStream_t s) {
    using C = cx<T>;
    CrArgs<C> A = base_args<C>(c);
    A.R = R;
    A.slab = slab;
    A.v_in = v;
    A.w_out = w;
    const long long per_cta = (long long)c->n_tot * ldwmax_of(c);
    if (scratch) return launch_solve<T, CR_TEST>(c, A, dim3(R), per_cta, scratch, scratch_bytes, s);
    ProfScope ps(c, s, LSS_PROF_SLAB_E, 1);
    return launch_solve<T, CR_TEST>(c, A, dim3(R), per_cta, nullptr, 0, s);
}

}  // namespace

// Auxiliary streams (and their events) for n concurrent runs.
int lss_ensure_aux(lss_ctx* c, size_t n) {
    while (c->aux_stream.size() + 1 < n) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e) {
            if (st) cudaStreamDestroy(st);
            return lss_check_cuda(c, e, "auxiliary streams");
        }
        c->aux_stream.push_back(st);
        c->aux_event.push_back(ev);
    }
    if (!c->fork_event)
        return lss_check_cuda(c, cudaEventCreateWithFlags(&c->fork_event, cudaEventDisableTiming), "auxiliary streams");
    return LSS_OK;
}

int lss_thomas_prepare(lss_ctx* c, int R, cudaStream_t s) {
    if (c->dim != 2 || R < kThMinR || !thomas_enabled() || c->th_valid) return LSS_OK;
    return c->prec == LSS_FP64 ? thomas_prepare_t<double>(c, s) : thomas_prepare_t<float>(c, s);
}

int lss_prepare_solve_tables(lss_ctx* c, cudaStream_t s) {
    return c->prec == LSS_FP64 ? prepare_chunk_tables<double>(c, s) : prepare_chunk_tables<float>(c, s);
}

int lss_factor_slabs(lss_ctx* c, cudaStream_t s) {
    c->iface_t_valid = false;
    c->th_valid = false;
    return c->prec == LSS_FP64 ? factor_impl<double>(c, s) : factor_impl<float>(c, s);
}

int lss_recurrences(lss_ctx* c, const void* maps, void* lam, void* phi, const void* a_first, const void* a_last,
                    int R, cudaStream_t s) {
    if (c->prec == LSS_FP64)
        return launch_recur<double>(c, (const double2*)maps, (double2*)lam, (double2*)phi, (const double2*)a_first,
                                    (const double2*)a_last, R, s);
    return launch_recur<float>(c, (const float2*)maps, (float2*)lam, (float2*)phi, (const float2*)a_first,
                               (const float2*)a_last, R, s);
}

int lss_sweep(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s) {
    if (c->dim == 3) return lss3_sweep(c, r, y, R, s);
    return c->prec == LSS_FP64 ? sweep_impl<double>(c, r, y, R, s) : sweep_impl<float>(c, r, y, R, s);
}

int lss_sweep_grid(lss_ctx* c, const double2* F, double2* y, int R, cudaStream_t s) {
    if (c->dim != 2) return lss_fail(c, LSS_ERR_UNSUPPORTED, "grid sweep: 2D grids only");
    return c->prec == LSS_FP64 ? sweep_impl<double>(c, nullptr, y, R, s, F) : sweep_impl<float>(c, nullptr, y, R, s, F);
}

int lss_slab_apply(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s) {
    if (c->dim == 3) return lss3_slab_apply(c, slab, v, w, R, s);
    return c->prec == LSS_FP64 ? slab_apply_impl<double>(c, slab, v, w, R, nullptr, 0, s)
                               : slab_apply_impl<float>(c, slab, v, w, R, nullptr, 0, s);
}

// ---------------------------------------------------------------- fixed-scratch slab operator
// lss_apply_slab_noalloc: the slab operator of lss_apply_slab with its
// right-hand-side scratch in a fixed device array instead of the context's
// growable workspace, so that the call never reaches the device allocator.
namespace {

constexpr size_t kFixedScratchBytes = size_t(8) << 20;   // 8 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_fixed_mu;
void* g_fixed_ptr[kMaxDevices] = {};

// Device address of g_fixed_scratch for the current device.  In host code the
// symbol names a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  The cached
// address stays valid while the device's primary context lives; after
// cudaDeviceReset the process must not call this entry point again.
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

}  // namespace

extern "C" int lss_apply_slab_noalloc(lss_ctx* c, int slab, const void* v_dev, void* w_dev, int R, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!c->inst.empty())
        return lss_fail(c, LSS_ERR_ARG, "apply_slab_noalloc: not defined on a batch context; call it on an "
                                         "instance (lss_batch_instance)");
    if (c->dim != 2) return lss_fail(c, LSS_ERR_UNSUPPORTED, "apply_slab_noalloc: 2D contexts only");
    if (!v_dev || !w_dev || R < 1 || slab < 0 || slab >= c->n_slabs)
        return lss_fail(c, LSS_ERR_ARG, "apply_slab_noalloc: bad arguments");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "apply_slab_noalloc before lss_factor");
    void* scratch = nullptr;
    int rc = fixed_scratch(c, &scratch);
    if (rc) return rc;
    // Every scratch entry a CTA reads is written by that CTA first, so
    // nothing has to start at zero and no clearing is needed.
    cudaStream_t s = (cudaStream_t)stream;
    return c->prec == LSS_FP64
               ? slab_apply_impl<double>(c, slab, (const double2*)v_dev, (double2*)w_dev, R, scratch,
                                         kFixedScratchBytes, s)
               : slab_apply_impl<float>(c, slab, (const double2*)v_dev, (double2*)w_dev, R, scratch,
                                        kFixedScratchBytes, s);
}
