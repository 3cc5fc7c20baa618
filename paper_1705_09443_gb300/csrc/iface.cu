// Interface maps of the slab-parallel sweep (Sec. 2.3, Algorithm 2), all
// columns of a slab at once.
//
// For slab i and pin layer q (q = first layer of D_i for Lambda_i and Gamma_i,
// q = last layer for Phi_i) the maps need W = S_i^{-1} [e_{(q,j)}]_j restricted
// to two layers, for every block row j.  The n_tot unit right-hand sides of a
// slab go through the cyclic reduction together.  Forward: the right-hand side
// of column j starts in block row j, and the reduction of level l mixes rows
// 2^l apart, so at level l block row k is non-zero only in the columns
// [k - (2^l - 1), k + (2^l - 1)]; the forward pass touches only those windows.
// The top row and the back substitution are dense in the columns: at level l
// every odd row gets x_k = y_k - (D^{-1}C)_k x_{k-2^l} - (D^{-1}B)_k x_{k+2^l}
// for all n_tot columns, a (G x 2G)(2G x columns) product; level 0 keeps only
// the first and last layers.  The maps then apply the coupling H_{[i,i-1]}
// (resp. H_{[i,i+1]}), tridiagonal in the columns:
//   Lambda_i[k][j] = sum_{j'} W_last[k][j'] H(j', j),  Gamma_i with W_first,
//   Phi_i with W_first and H_{[i,i+1]}.
// One launch per phase covers every slab and side: grid (column tiles, block
// rows of the level, problems); lane p of a column group owns layer p.  The
// column blocks live in a scratch array X[problem][k][j][layer] (n_tot x n_tot
// x G entries per problem).
#include <algorithm>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

constexpr int kIfT = 256;   // threads per CTA: G lanes per column (one per layer) x column groups
constexpr int kIfTN = 16;   // columns per CTA (a short chain per thread: 1 column of 16-wide blocks, 2 of 32-wide)

struct IfProb {
    int slab, side, G, pad;
    long long xoff;   // entries of X before this problem
    long long woff;   // entries of W before this problem (2 n_tot^2 each)
};

template <typename C>
struct IfArgs {
    const SlabDev* slabs;
    int n_slabs, K;
    const C* fac;
    const C* coef;
    const IfProb* probs;
    C* X;
    C* W;             // layers na and w-1 of the solution columns: 2 x n_tot x n_tot per problem
    C* maps;
    int psi;          // also write Psi_i (last layer from the last-layer pin): two fronts
};

__device__ __forceinline__ double2 cfnma_i(double2 a, double2 b, double2 acc) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfnma_i(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(-a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}

// Window of block row k at level l: [k - (2^l - 1), k + (2^l - 1)] within [0, K).
__device__ __forceinline__ int win_lo(int k, int l) { return max(0, k - ((1 << l) - 1)); }
__device__ __forceinline__ int win_hi(int k, int l, int K) { return min(K - 1, k + ((1 << l) - 1)); }

// Copies n entries (blocks or bands) into shared memory.
template <typename C>
__device__ __forceinline__ void stage(C* dst, const C* src, int n) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}

// Forward phase of level l over the windows: phase 0 = odd rows
// (y = D^{-1} b in place), 1 = even rows (b -= C y_{k-s} + B y_{k+s}, into the
// window of level l+1), 2 = the top row (all columns, in place).  Lane p of a
// column group owns layer p of CPT columns.
template <typename T, int G>
__device__ void fwd_body(const IfArgs<cx<T>>& A, const IfProb& pr, int l, int phase) {
    using C = cx<T>;
    extern __shared__ __align__(16) unsigned char smi[];
    C* Ms = reinterpret_cast<C*>(smi);   // up to 2 blocks, or the bands of one row
    const int K = A.K;
    const SlabDev sd = A.slabs[pr.slab];
    const int bs = G * G;
    const C* F = A.fac + sd.fac_off;
    const int pin = pr.side == 0 ? sd.na : sd.ll;
    const int s = 1 << l;
    const CrLevelOffs lv = cr_level(K, l);
    const int r = blockIdx.y;
    int k, lo, hi;
    if (phase == 0) {
        if (r >= lv.K / 2) return;
        k = (2 * r + 1) * s;
        lo = win_lo(k, l);
        hi = win_hi(k, l, K);
    } else if (phase == 1) {
        if (r >= (lv.K + 1) / 2) return;
        k = 2 * r * s;
        lo = win_lo(k, l + 1);
        hi = win_hi(k, l + 1, K);
    } else {
        if (r > 0) return;
        k = 0;
        lo = 0;
        hi = K - 1;
    }
    const int j0 = lo + blockIdx.x * kIfTN;
    if (j0 > hi) return;
    C* X = A.X + pr.xoff;
    auto at = [&](int kk, int j) { return X + ((long long)kk * K + j) * G; };
    const int p = threadIdx.x % G, cg = threadIdx.x / G;
    constexpr int NCG = kIfT / G, CPT = kIfTN / NCG;
    if (phase == 0 || phase == 2) {
        const C* D = phase == 0 ? F + (lv.dinv + r) * bs : F + cr_level(K, cr_levels(K)).dinv * bs;
        stage(Ms, D, bs);
        __syncthreads();
        if (phase == 0 && l == 0) {   // b_k = e_(pin, k): y_k = column pin of D^{-1}, in column k only
            if (threadIdx.x < G) at(k, k)[threadIdx.x] = Ms[pin * G + threadIdx.x];
            return;
        }
        C acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int j = j0 + cg * CPT + q;
            acc[q] = czero<C>();
            if (j <= hi && j < j0 + kIfTN) {
                const C* x = at(k, j);
#pragma unroll
                for (int a = 0; a < G; ++a) acc[q] = cfma(Ms[a * G + p], x[a], acc[q]);
            }
        }
        __syncthreads();   // every column of the tile read before it is overwritten
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int j = j0 + cg * CPT + q;
            if (j <= hi && j < j0 + kIfTN) at(k, j)[p] = acc[q];
        }
        return;
    }
    // even rows: b_k -= C_k y_{k-s} + B_k y_{k+s}; a row that is odd at level
    // l+1 (index r odd there) or the top row then applies its next-level
    // D^{-1} in place (the phase 0 of level l+1, or phase 2, fused: the
    // layers of a column are the G lanes of one column group)
    const bool hasL = k - s >= 0, hasR = k + s < K;
    const int L = cr_levels(K);
    const bool top_next = l + 1 == L && r == 0;
    // (single precision only: in double precision the shuffles cost more than
    // the separate launches they save)
    const bool fuse = sizeof(T) == 4 && (top_next || (l + 1 < L && (r & 1)));
    C* Dn = Ms + 2 * bs;   // the next-level D^{-1} (2 bs >= 6G for the bands of level 0)
    if (l == 0) {
        const C* t0 = F + cr_t0_off(K, bs) + (long long)r * 6 * G;   // even row r's bands
        stage(Ms, t0, 6 * G);
    } else {
        stage(Ms, F + (lv.cbe + 2LL * r) * bs, 2 * bs);
    }
    if (fuse)
        stage(Dn, F + (top_next ? cr_level(K, L).dinv : cr_level(K, l + 1).dinv + (r - 1) / 2) * bs, bs);
    __syncthreads();
    const int llo = win_lo(k, l), lhi = win_hi(k, l, K);
    const int mlo = win_lo(k - s, l), mhi = hasL ? win_hi(k - s, l, K) : -1;
    const int plo = hasR ? win_lo(k + s, l) : K, phi = hasR ? win_hi(k + s, l, K) : -1;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int j = j0 + cg * CPT + q;
        const bool valid = j <= hi && j < j0 + kIfTN;   // uniform over the column group
        C acc = czero<C>();
        if (!valid) {
            // nothing to compute; the group still takes part in the shuffles below
        } else if (l == 0) {
            if (j == k && p == pin) acc.x = T(1);
        } else if (j >= llo && j <= lhi) {
            acc = at(k, j)[p];
        }
        if (valid && hasL && j >= mlo && j <= mhi) {
            const C* x = at(k - s, j);
            if (l == 0) {
#pragma unroll
                for (int da = -1; da <= 1; ++da)
                    if (p + da >= 0 && p + da < G) acc = cfnma_i(Ms[(da + 1) * G + p], x[p + da], acc);
            } else {
#pragma unroll
                for (int a = 0; a < G; ++a) acc = cfnma_i(Ms[a * G + p], x[a], acc);
            }
        }
        if (valid && hasR && j >= plo && j <= phi) {
            const C* x = at(k + s, j);
            if (l == 0) {
#pragma unroll
                for (int da = -1; da <= 1; ++da)
                    if (p + da >= 0 && p + da < G) acc = cfnma_i(Ms[(3 + da + 1) * G + p], x[p + da], acc);
            } else {
#pragma unroll
                for (int a = 0; a < G; ++a) acc = cfnma_i(Ms[bs + a * G + p], x[a], acc);
            }
        }
        if (fuse) {   // y = D^{-1} b over the layers of the column
            C y = czero<C>();
#pragma unroll
            for (int a = 0; a < G; ++a) {
                C ba;
                ba.x = __shfl_sync(0xffffffffu, acc.x, a, G);
                ba.y = __shfl_sync(0xffffffffu, acc.y, a, G);
                y = cfma(Dn[a * G + p], ba, y);
            }
            acc = y;
        }
        if (valid) at(k, j)[p] = acc;
    }
}

// Back substitution of level 0 for the odd rows, layers na and w-1 only:
// x_k[q] = y_k[q] - (D^{-1})_k[q,:] (C_k x_{k-1} + B_k x_{k+1}) for q = na, w-1.
// The two kept rows of D^{-1} are folded into the bands once per CTA,
// u_q = (D^{-1})_k[q,:] C_k and v_q = (D^{-1})_k[q,:] B_k (G-vectors, C and B
// tridiagonal in the layers), so each column is four dot products of length G;
// one thread per column, results into the compact arrays W0 (layer na) and W1
// (layer w-1).  The thread also copies those layers of the even row k-1 (and
// of row K-1 when it is an unpaired even row).
constexpr int kB0N = 128;   // columns (threads) per CTA

template <typename T, int G>
__device__ void bwd0_body(const IfArgs<cx<T>>& A, const IfProb& pr) {
    using C = cx<T>;
    __shared__ C sb[8 * 32];     // bands of row k (6G), rows na and w-1 of its D^{-1} (2G)
    __shared__ C uv[4][32];      // u_na, v_na, u_{w-1}, v_{w-1}
    const int K = A.K;
    const SlabDev sd = A.slabs[pr.slab];
    const int bs = G * G;
    const C* F = A.fac + sd.fac_off;
    const int r = blockIdx.y;
    const int k = 2 * r + 1;
    const int j0 = blockIdx.x * kB0N;
    if (k >= K || j0 >= K) return;   // uniform over the CTA
    const int tid = threadIdx.x;
    const C* bands = F + cr_t0_off(K, bs) + ((long long)(K + 1) / 2 + r) * 6 * G;
    const C* p0 = F + cr_p0_off(K, bs, G) + (long long)r * 2 * G;
    for (int e = tid; e < 8 * G; e += kB0N) sb[e] = e < 6 * G ? bands[e] : p0[e - 6 * G];
    __syncthreads();
    if (tid < G) {   // coefficient of x[a]: sum over p = a - da of D^{-1}[q][p] band[(da+1)G + p]
        const int a = tid;
        C u0 = czero<C>(), v0 = czero<C>(), u1 = czero<C>(), v1 = czero<C>();
#pragma unroll
        for (int da = -1; da <= 1; ++da) {
            const int p = a - da;
            if (p < 0 || p >= G) continue;
            const C cC = sb[(da + 1) * G + p], cB = sb[3 * G + (da + 1) * G + p];
            const C q0 = sb[6 * G + p], q1 = sb[7 * G + p];
            u0 = cfma(q0, cC, u0);
            v0 = cfma(q0, cB, v0);
            u1 = cfma(q1, cC, u1);
            v1 = cfma(q1, cB, v1);
        }
        uv[0][a] = u0;
        uv[1][a] = v0;
        uv[2][a] = u1;
        uv[3][a] = v1;
    }
    __syncthreads();
    // the neighbours' column tiles go through shared memory (coalesced loads,
    // rows padded to G + 1 entries so that each thread's column reads are
    // conflict-free), one neighbour at a time
    extern __shared__ __align__(16) unsigned char smb[];
    C* tile = reinterpret_cast<C*>(smb);   // kB0N x (G + 1)
    const int na = sd.na, wl = sd.ll;
    const bool hasR = k + 1 < K;
    const int nj = min(kB0N, K - j0);
    C* X = A.X + pr.xoff;
    const int j = j0 + tid;
    const bool on = tid < nj;
    C d0 = czero<C>(), d1 = czero<C>(), em0 = czero<C>(), em1 = czero<C>(), ep0 = czero<C>(), ep1 = czero<C>();
    // (double precision reads its columns directly: its 16-byte entries already
    // make the per-thread column walk efficient, and the tile costs occupancy)
    constexpr bool staged = sizeof(T) == 4;
    for (int side = 0; side < (hasR ? 2 : 1); ++side) {
        const C* src = X + ((long long)(side == 0 ? k - 1 : k + 1) * K + j0) * G;
        if (staged) {
            if (side) __syncthreads();   // the previous tile is consumed
            for (int e = tid; e < nj * G; e += kB0N) tile[(e / G) * (G + 1) + e % G] = src[e];
            __syncthreads();
        }
        if (on) {
            const C* x = staged ? tile + tid * (G + 1) : src + (long long)tid * G;
            const C* u = uv[side == 0 ? 0 : 1];
            const C* v = uv[side == 0 ? 2 : 3];
            C c0 = czero<C>(), c1 = czero<C>();
#pragma unroll
            for (int a = 0; a < G; ++a) {
                const C xa = x[a];
                d0 = cfma(u[a], xa, d0);
                d1 = cfma(v[a], xa, d1);
                if (a == na) c0 = xa;
                if (a == wl) c1 = xa;
            }
            if (side == 0) { em0 = c0; em1 = c1; }
            else { ep0 = c0; ep1 = c1; }
        }
    }
    if (!on) return;
    C* W0 = A.W + pr.woff;
    C* W1 = W0 + (long long)K * K;
    const long long o = (long long)k * K + j;
    C y0 = czero<C>(), y1 = czero<C>();
    if (j == k) {   // y_k is non-zero in column k only
        const C* yk = X + ((long long)k * K + j) * G;
        y0 = yk[na];
        y1 = yk[wl];
    }
    W0[o] = y0 - d0;
    W1[o] = (wl == na) ? y0 - d0 : y1 - d1;
    W0[o - K] = em0;
    W1[o - K] = em1;
    if (k + 1 == K - 1) {
        W0[o + K] = ep0;
        W1[o + K] = ep1;
    }
}

// Back substitution of level l >= 1, register-tiled: the CTA stages
// (D^{-1}C)_k, (D^{-1}B)_k and the column tiles of x_{k-s}, x_{k+s} (transposed
// to [layer][column], rows padded to kBtN + 1 entries: conflict-free for both
// the transposing store and the column reads) in shared memory; thread
// (row group rg, column group cg) owns layers rg*TP .. rg*TP+TP-1 of columns
// cg + 16 t, t < TJ, and subtracts the products from y in the same order as
// the untiled loop (block C then B, layer a ascending).
constexpr int kBtN = 64;                 // columns per CTA
constexpr int kBtThreads = 128;          // 8 row groups x 16 column groups
constexpr int kBtNP = kBtN + 1;

template <typename T, int G>
__device__ void bwd_tiled_body(const IfArgs<cx<T>>& A, const IfProb& pr, int l) {
    using C = cx<T>;
    constexpr int RG = 8, CGN = 16, TP = G / RG, TJ = kBtN / CGN;
    extern __shared__ __align__(16) unsigned char smi[];
    C* Ms = reinterpret_cast<C*>(smi);   // [2][G * G], column-major blocks
    C* Xs = Ms + 2 * G * G;              // [2][G][kBtNP]
    const int K = A.K;
    const SlabDev sd = A.slabs[pr.slab];
    const int bs = G * G;
    const C* F = A.fac + sd.fac_off;
    const int s = 1 << l;
    const CrLevelOffs lv = cr_level(K, l);
    const int r = blockIdx.y;
    if (r >= lv.K / 2) return;
    const int k = (2 * r + 1) * s;
    const int j0 = blockIdx.x * kBtN;
    if (j0 >= K) return;
    const int nj = min(kBtN, K - j0);
    const int nb = k + s < K ? 2 : 1;
    C* X = A.X + pr.xoff;
    const int tid = threadIdx.x;
    const C* Mg = F + (lv.dcdb + 2LL * r) * bs;
    for (int e = tid; e < nb * bs; e += kBtThreads) Ms[e] = Mg[e];
    for (int b = 0; b < nb; ++b) {
        const C* src = X + ((long long)(b == 0 ? k - s : k + s) * K + j0) * G;
        C* dst = Xs + b * G * kBtNP;
        for (int e = tid; e < nj * G; e += kBtThreads) dst[(e % G) * kBtNP + e / G] = src[e];
    }
    const int rg = tid / CGN, cg = tid % CGN;
    const int ylo = win_lo(k, l), yhi = win_hi(k, l, K);
    C acc[TP][TJ];
#pragma unroll
    for (int t = 0; t < TJ; ++t) {
        const int jj = cg + CGN * t, j = j0 + jj;
        const bool iny = jj < nj && j >= ylo && j <= yhi;
        const C* y = X + ((long long)k * K + j) * G + rg * TP;
#pragma unroll
        for (int q = 0; q < TP; ++q) acc[q][t] = iny ? y[q] : czero<C>();
    }
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
        const C* M = Ms + b * bs + rg * TP;
        const C* Xb = Xs + b * G * kBtNP + cg;
#pragma unroll 4
        for (int a = 0; a < G; ++a) {
            C m[TP], x[TJ];
#pragma unroll
            for (int q = 0; q < TP; ++q) m[q] = M[a * G + q];
#pragma unroll
            for (int t = 0; t < TJ; ++t) x[t] = Xb[a * kBtNP + CGN * t];
#pragma unroll
            for (int q = 0; q < TP; ++q)
#pragma unroll
                for (int t = 0; t < TJ; ++t) acc[q][t] = cfnma_i(m[q], x[t], acc[q][t]);
        }
    }
#pragma unroll
    for (int t = 0; t < TJ; ++t) {
        const int jj = cg + CGN * t;
        if (jj >= nj) continue;
        C* xo = X + ((long long)k * K + j0 + jj) * G + rg * TP;
#pragma unroll
        for (int q = 0; q < TP; ++q) xo[q] = acc[q][t];
    }
}

template <typename T>
__global__ void __launch_bounds__(kBtThreads) if_bwdt_kernel(IfArgs<cx<T>> A, int l, int zoff) {
    const IfProb pr = A.probs[zoff + blockIdx.z];
    if (pr.G == 16) bwd_tiled_body<T, 16>(A, pr, l);
    else bwd_tiled_body<T, 32>(A, pr, l);
}

template <typename T>
__global__ void __launch_bounds__(kIfT) if_fwd_kernel(IfArgs<cx<T>> A, int l, int phase) {
    const IfProb pr = A.probs[blockIdx.z];
    if (pr.G == 16) fwd_body<T, 16>(A, pr, l, phase);
    else fwd_body<T, 32>(A, pr, l, phase);
}

template <typename T>
__global__ void __launch_bounds__(kB0N) if_bwd0_kernel(IfArgs<cx<T>> A) {
    const IfProb pr = A.probs[blockIdx.z];
    if (pr.G == 16) bwd0_body<T, 16>(A, pr);
    else bwd0_body<T, 32>(A, pr);
}

// Maps from the two kept layers and the coupling, tridiagonal in the columns.
template <typename T>
__global__ void __launch_bounds__(256) if_maps_kernel(IfArgs<cx<T>> A) {
    using C = cx<T>;
    const IfProb pr = A.probs[blockIdx.y];
    const int K = A.K, i = pr.slab;
    const SlabDev sd = A.slabs[i];
    const C* cf = A.coef + sd.coef_off;
    const long long nt2 = (long long)K * K;
    const C* W0 = A.W + pr.woff;
    const C* W1 = W0 + nt2;
    const int ns = A.n_slabs;
    const int pin = pr.side == 0 ? sd.na : sd.ll;
    const int base = pr.side == 0 ? 0 : 6;   // coupling slot of layer offset -1 / +1
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nt2; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / K), j = (int)(e % K);
        C v0 = czero<C>(), v1 = czero<C>();
        for (int jp = max(0, j - 1); jp <= min(K - 1, j + 1); ++jp) {
            const C h = cf[(long long)jp * sd.cstride + pin * 9 + base + (j - jp) + 1];
            const long long o = (long long)k * K + jp;
            v0 = cfma(W1[o], h, v0);
            v1 = cfma(W0[o], h, v1);
        }
        if (pr.side == 0) {
            A.maps[(0LL * ns + i) * nt2 + e] = v0;
            A.maps[(1LL * ns + i) * nt2 + e] = v1;
        } else {
            A.maps[(2LL * ns + i) * nt2 + e] = v1;
            if (A.psi) A.maps[(3LL * ns + i) * nt2 + e] = v0;   // Psi_i (two fronts)
        }
    }
}

template <typename T>
int iface_impl(lss_ctx* c, cudaStream_t s) {
    using C = cx<T>;
    const int K = c->n_tot, ns = c->n_slabs;
    if (ns == 1) return LSS_OK;
    // problems: side 0 for slabs 1..l-1, side 1 for slabs 1..l-2 (from slab 0
    // when two fronts meet in slab 0, whose Psi_0 the meeting step needs)
    // (16-wide blocks first, then 32-wide, so that the tiled back substitution
    // can size its shared memory per block width)
    std::vector<IfProb> probs;
    long long xoff = 0, woff = 0;
    int gmax = 16, n16 = 0;
    const int side1_first = (c->fronts == 2 && c->mid == 0) ? 0 : 1;
    for (int g : {16, 32})
        for (int side = 0; side < 2; ++side)
            for (int i = side == 0 ? 1 : side1_first; i <= (side == 0 ? ns - 1 : ns - 2); ++i) {
                if (c->slabs[i].ldw != g) continue;
                IfProb p{i, side, g, 0, xoff, woff};
                xoff += (long long)K * K * p.G;
                woff += 2LL * K * K;
                gmax = std::max(gmax, p.G);
                n16 += g == 16;
                probs.push_back(p);
            }
    const int np = (int)probs.size();
    int rc = lss_grow(c, &c->ifx_buf, &c->ifx_cap, (size_t)(xoff + woff) * sizeof(C));
    if (rc) return rc;
    if (c->ifp_n != np) {   // the table depends on the slab layout only: uploaded once
        rc = lss_grow(c, &c->ifp_buf, &c->ifp_cap, probs.size() * sizeof(IfProb));
        // on the context's stream (ordered before the map kernels), and finished
        // before the host table goes out of scope
        if (!rc) rc = lss_check_cuda(c, cudaMemcpyAsync(c->ifp_buf, probs.data(), probs.size() * sizeof(IfProb),
                                                        cudaMemcpyHostToDevice, s), "interface problems");
        if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "interface problems");
        if (rc) return rc;
        c->ifp_n = np;
    }
    IfArgs<C> A{};
    A.slabs = c->d_slabs;
    A.n_slabs = ns;
    A.K = K;
    A.fac = (const C*)c->fac;
    A.coef = (const C*)c->coef;
    A.probs = (const IfProb*)c->ifp_buf;
    A.X = (C*)c->ifx_buf;
    A.W = A.X + xoff;
    A.maps = (C*)c->iface;
    A.psi = c->fronts == 2;
    const size_t sh = sizeof(C) * ((size_t)3 * gmax * gmax + (size_t)8 * gmax);
    std::unique_lock<std::mutex> lock(lss_config_mutex());
    long long& cfg_f = lss_dev_cache((const void*)if_fwd_kernel<T>, 0);
    if ((long long)sh > cfg_f) {
        cudaError_t e = cudaFuncSetAttribute(if_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sh, 48 * 1024));
        if (e) return lss_check_cuda(c, e, "interface attribute");
        cfg_f = (long long)sh;
    }
    const size_t sht = sizeof(C) * ((size_t)2 * gmax * gmax + (size_t)2 * gmax * kBtNP);
    const size_t sh0 = sizeof(T) == 4 ? sizeof(C) * (size_t)kB0N * (gmax + 1) : 0;
    long long& cfg_t = lss_dev_cache((const void*)if_bwdt_kernel<T>, 0);
    long long& cfg_0 = lss_dev_cache((const void*)if_bwd0_kernel<T>, 0);
    if (sizeof(T) == 4 && (long long)sh0 > cfg_0) {
        cudaError_t e = cudaFuncSetAttribute(if_bwd0_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sh0, 48 * 1024));
        if (e) return lss_check_cuda(c, e, "interface attribute");
        cfg_0 = (long long)sh0;
    }
    if ((long long)sht > cfg_t) {
        cudaError_t e = cudaFuncSetAttribute(if_bwdt_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(sht, 48 * 1024));
        if (e) return lss_check_cuda(c, e, "interface attribute");
        cfg_t = (long long)sht;
    }
    lock.unlock();
    const int L = cr_levels(K);
    const int kt = (K + kIfTN - 1) / kIfTN;
    const int ncls = (n16 > 0) + (np > n16);
    ProfScope ps(c, s, LSS_PROF_IFACE, (sizeof(T) == 4 ? L + 3 : 2 * L + 3) + (L - 1) * ncls);
    // level 0's odd rows, then per level the even rows; in single precision the
    // next level's odd rows (and finally the top row) are fused into them
    constexpr bool fused = sizeof(T) == 4;
    for (int l = 0; l < L; ++l) {
        const int Kl = cr_level(K, l).K;
        const int wt0 = ((1 << (l + 1)) - 1 + kIfTN - 1) / kIfTN;   // tiles of a level-l window
        const int wt1 = ((1 << (l + 2)) - 1 + kIfTN - 1) / kIfTN;   // tiles of a level-(l+1) window
        if (l == 0 || !fused)
            if_fwd_kernel<T><<<dim3(std::min(wt0, kt), std::max(1, Kl / 2), np), kIfT, sh, s>>>(A, l, 0);
        if_fwd_kernel<T><<<dim3(std::min(wt1, kt), (Kl + 1) / 2, np), kIfT, sh, s>>>(A, l, 1);
    }
    if (!fused) if_fwd_kernel<T><<<dim3(kt, 1, np), kIfT, sh, s>>>(A, L, 2);
    // back substitution, levels L-1..1: the 16-wide problems on s, the 32-wide
    // ones (few, each a long chain of levels) concurrently on an auxiliary
    // stream; level 0 over all problems after the join
    const int ktt = (K + kBtN - 1) / kBtN;
    const bool two = n16 > 0 && np > n16;
    if (two) {
        if (int rc2 = lss_ensure_aux(c, 2)) return rc2;
        cudaEventRecord(c->fork_event, s);
        cudaStreamWaitEvent(c->aux_stream[0], c->fork_event, 0);
    }
    cudaStream_t s32 = two ? c->aux_stream[0] : s;
    const size_t sh16 = sizeof(C) * ((size_t)2 * 16 * 16 + (size_t)2 * 16 * kBtNP);
    for (int l = L - 1; l > 0; --l) {
        const int Kl = cr_level(K, l).K;
        if (n16 > 0) if_bwdt_kernel<T><<<dim3(ktt, std::max(1, Kl / 2), n16), kBtThreads, sh16, s>>>(A, l, 0);
        if (np > n16)
            if_bwdt_kernel<T><<<dim3(ktt, std::max(1, Kl / 2), np - n16), kBtThreads, sht, s32>>>(A, l, n16);
    }
    if (two) {
        cudaEventRecord(c->aux_event[0], s32);
        cudaStreamWaitEvent(s, c->aux_event[0], 0);
    }
    if_bwd0_kernel<T><<<dim3((K + kB0N - 1) / kB0N, std::max(1, K / 2), np), kB0N, sh0, s>>>(A);
    if_maps_kernel<T><<<dim3((unsigned)std::min<long long>(((long long)K * K + 255) / 256, 1024), np), 256, 0,
                        s>>>(A);
    return lss_check_cuda(c, cudaGetLastError(), "interface launch");
}

}  // namespace

int lss_iface_maps(lss_ctx* c, cudaStream_t s) {
    return c->prec == LSS_FP64 ? iface_impl<double>(c, s) : iface_impl<float>(c, s);
}
