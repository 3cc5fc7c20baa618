// The recursive approach of Sec. 3.1: every quasi-2D slab subproblem S_i of
// the 3D sweep is itself swept along x2 over quasi-1D sub-slab problems
// instead of being factored whole.
//
// Sub-slab problem (i, j): x2 layers E_j (the partition of x2 that the slabs
// use of x1) after b_aux auxiliary x2 layers (none for j = 0), x1 over S_i's
// layers, x3 over the whole range.  Its rows on E_j are S_i's rows; its rows
// on the auxiliary x2 layers are PML stencils with the auxiliary profile
// along x2 (the left profile of width b_aux translated so that E_j's first
// layer plays the role of index 0), the layer's own profile along x1 (the
// physical one, or the slab's auxiliary one on S_i's auxiliary layers) and the
// physical one along x3, at the sampled local frequency nearest
// omega^2 (1 - m).  Each problem is block tridiagonal along x3 with n_tot
// blocks of M = w2 * w1 unknowns (x2 layer a, x1 layer c), factored by the
// same block Gaussian elimination as the slabs (dense Gauss-Jordan inverses of
// the pivot blocks).
//
// Application: one CTA per right-hand side walks the outer sweep (Algorithm 2
// over the slabs); each slab solve forms the slab's input, runs the inner
// sweep (Algorithm 2 along x2 over the sub-slab problems, each a forward and
// backward block substitution along x3) and writes the slab's layers back.
// Nothing waits on another CTA.
//
// Layouts (complex entries):
//  - sub-slab coefficient table: block k (X3 = k), part p = d3+1, row
//    q = a * w1 + c, 9 entries (d2+1)*3 + (d1+1): ((k*3 + p) * M + q) * 9 + ...
//  - slab vectors (the inner sweep's right-hand side V and solution U):
//    [X2][X3][c], c over S_i's x1 layers.
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"
#include "stencil3.cuh"

namespace {

constexpr int kRecThreads = 512;
constexpr int kRecStages = 4;                     // ring of factor-row chunks in shared memory
constexpr unsigned kRecStageMax = 48 * 1024;      // bytes per stage (less when the step vectors need the room)
constexpr size_t kRecSmem = 220 * 1024;
enum { R3_FWD = 1, R3_CL = 2, R3_CR = 4 };   // as the flags of the slab sweep's steps

// Inner auxiliary stencils: per (sample k, auxiliary x2 layer t2, x1 kind,
// class x3).  x1 kinds: [0, nc) the physical classes, [nc, nc + b_aux) the
// left auxiliary layers t1 = 1..b_aux, [nc + b_aux, nc + 2 b_aux) the right
// ones (two fronts).
__global__ void __launch_bounds__(32 * kGamWarps) gamma3_aux2_kernel(double2* out, int n, int b, int baux, int ns,
                                                                      double s_lo, double s_hi, double Cw, double h,
                                                                      int nkind1) {
    __shared__ GamSmem S[kGamWarps];
    const int nc = 2 * b + 1;
    const int wid = threadIdx.x / 32;
    const long long e = (long long)blockIdx.x * kGamWarps + wid;
    const long long tot = (long long)ns * baux * nkind1 * nc;
    if (e >= tot) return;
    const int c3 = (int)(e % nc);
    const int kind = (int)((e / nc) % nkind1);
    const int t2 = (int)((e / ((long long)nc * nkind1)) % baux) + 1;
    const int k = (int)(e / ((long long)nc * nkind1 * baux));
    const double sk = (ns == 1) ? s_lo : (k == ns - 1 ? s_hi : s_lo + k * ((s_hi - s_lo) / (ns - 1)));
    double sig[3][3];
    const int q3 = class_index3(c3, n, b);
    for (int u = 0; u < 3; ++u) {
        double v1 = 0;
        if (kind < nc) {
            v1 = sigma_phys3(class_index3(kind, n, b) - 1 + u, n, b, Cw);
        } else if (kind < nc + baux) {   // offset q1 from D_i's first layer
            const int q1 = -(kind - nc + 1) - 1 + u;
            if (q1 <= -1) { const double tt = (q1 + 1.0) / baux; v1 = -Cw * tt * tt; }
        } else {                         // offset d from D_i's last layer
            const int d = (kind - nc - baux + 1) - 1 + u;
            if (d >= 1) { const double tt = (d - 1.0) / baux; v1 = Cw * tt * tt; }
        }
        double v2 = 0;
        const int q2 = -t2 - 1 + u;      // offset from E_j's first layer
        if (q2 <= -1) { const double tt = (q2 + 1.0) / baux; v2 = -Cw * tt * tt; }
        sig[0][u] = v1;
        sig[1][u] = v2;
        sig[2][u] = sigma_phys3(q3 - 1 + u, n, b, Cw);
    }
    gamma3_warp(sig, sqrt(sk), h, S[wid], out + (size_t)e * 27);
}

__device__ __forceinline__ int nearest_sample(double v, int ns, double s_lo, double s_hi) {
    if (ns <= 1) return 0;
    const double x = (v - s_lo) / ((s_hi - s_lo) / (ns - 1));
    int kk = (int)ceil(x - 0.5);   // nearest sample, ties to the lower one
    return kk < 0 ? 0 : (kk > ns - 1 ? ns - 1 : kk);
}

// Row coefficients of every sub-slab problem.  grid (blocks, problems);
// thread per row (k, q).
__global__ void assemble_rec_kernel(const Slab3* __restrict__ probs, const Slab3* __restrict__ oslabs,
                                    const double* __restrict__ m, const double2* __restrict__ gphys,
                                    const double2* __restrict__ gaux, const double2* __restrict__ gaux_r,
                                    const double2* __restrict__ gam2, Stencil27 st, double2* __restrict__ coef, int n,
                                    int b, int baux, int n_tot, int ns, double s_lo, double s_hi, double omega,
                                    int nkind1) {
    const Slab3 P = probs[blockIdx.y];
    const Slab3 O = oslabs[P.oi];
    const long long rows = (long long)n_tot * P.M;
    const int nc = 2 * b + 1;
    const double w2 = omega * omega;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / P.M), q = (int)(e % P.M);
        const int a2 = q / P.nc, a1 = q % P.nc;
        const int x1 = O.s - O.na + a1, x2 = P.s - P.na + a2, x3 = k - b;
        double2 row[27];
        if (a2 < P.na) {   // inner auxiliary x2 layer t2 before E_j
            const int t2 = P.na - a2;
            const int kind = a1 < O.na ? nc + (O.na - a1) - 1
                                       : (a1 > O.ll ? nc + baux + (a1 - O.ll) - 1 : pml_class3(x1, n, b));
            const int kk = nearest_sample(w2 * (1.0 - m3_at(m, n, x1, x2, x3)), ns, s_lo, s_hi);
            const double2* g =
                gam2 + ((((size_t)kk * baux + (t2 - 1)) * nkind1 + kind) * nc + pml_class3(x3, n, b)) * 27;
            for (int o = 0; o < 27; ++o) row[o] = g[o];
        } else if (a1 < O.na || a1 > O.ll) {   // S_i's auxiliary x1 layer t1
            const bool rgt = a1 > O.ll;
            const int t1 = rgt ? a1 - O.ll : O.na - a1;
            const int kk = nearest_sample(w2 * (1.0 - m3_at(m, n, x1, x2, x3)), ns, s_lo, s_hi);
            const double2* g = (rgt ? gaux_r : gaux) +
                               ((((size_t)kk * baux + (t1 - 1)) * nc + pml_class3(x2, n, b)) * nc + pml_class3(x3, n, b)) *
                                   27;
            for (int o = 0; o < 27; ++o) row[o] = g[o];
        } else if (x1 >= 0 && x1 <= n + 1 && x2 >= 0 && x2 <= n + 1 && x3 >= 0 && x3 <= n + 1) {
            for (int o = 0; o < 27; ++o) {
                const double mm = m3_at(m, n, x1 + o / 9 - 1, x2 + (o / 3) % 3 - 1, x3 + o % 3 - 1);
                row[o] = st.a_conj[o] + (w2 * mm) * st.b_conj[o];
            }
        } else {
            const double2* g =
                gphys + (((size_t)pml_class3(x1, n, b) * nc + pml_class3(x2, n, b)) * nc + pml_class3(x3, n, b)) * 27;
            for (int o = 0; o < 27; ++o) row[o] = g[o];
        }
        double2* out = coef + P.cf_off;
        for (int o = 0; o < 27; ++o) {
            const int d1 = o / 9, d2 = (o / 3) % 3, d3 = o % 3;
            out[(((long long)k * 3 + d3) * P.M + q) * 9 + d2 * 3 + d1] = row[o];
        }
    }
}

__global__ void cast_rec_kernel(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

struct RecArgs {
    const Slab3* oslabs;   // the slabs (outer sweep)
    const Slab3* probs;    // sub-slab problems, (i, j) at i * n_slabs + j
    int n_slabs, n_tot, b, Mmax;
    const void* ocoef;     // the slabs' coefficient tables (couplings between slabs)
    const void* icoef;     // sub-slab coefficient tables
    const void* ifac;      // sub-slab factors: per problem n_tot dense M x M inverses
    const void* f;         // sparsified right-hand sides on the grid
    void* ut;              // sweep solution on the grid
    long long G;           // n_tot^3
    void* scr;             // per right-hand side: V, U (n_tot^2 x w1max each), Y (n_tot x Mmax)
    long long vsz, sstride;
    const int2* steps;     // outer steps: (slab, flags)
    int nsteps;
    int* err;
    unsigned sb;           // bytes per ring stage (a multiple of 16, at least one row + 32)
};

// Rows of a pivot-block inverse (M columns) per chunk of the factor stream.
__host__ __device__ __forceinline__ int rec_rows(int M, int esz, unsigned sb) {
    const int r = (int)((sb - 32) / ((unsigned)M * esz));
    return r < 1 ? 1 : r;
}

// The factor stream in the order the walk consumes it: for every outer step,
// inner solve, direction and block row k, the rows of D_k^{-1} in chunks.
// Thread 0 keeps one cursor kRecStages chunks ahead of the consumers.
struct RecCursor {
    int st, pass, jj, dir, kk, r0;
    bool done;
};

template <typename C>
__device__ __forceinline__ void cursor_chunk(const RecArgs& A, const RecCursor& cu, const C** src, int* rows, int* M) {
    const int ns = A.n_slabs, K = A.n_tot;
    const int i = A.steps[cu.st].x;
    const int j = cu.pass == 0 ? cu.jj : ns - 2 - cu.jj;
    const Slab3 P = A.probs[(long long)i * ns + j];
    const int k = cu.dir == 0 ? cu.kk : K - 2 - cu.kk;
    *M = P.M;
    *rows = min(P.M - cu.r0, rec_rows(P.M, (int)sizeof(C), A.sb));
    *src = (const C*)A.ifac + P.fac_off + (long long)k * P.M * P.M + (long long)cu.r0 * P.M;
}

template <typename C>
__device__ __forceinline__ void cursor_advance(const RecArgs& A, RecCursor& cu) {
    const int ns = A.n_slabs, K = A.n_tot;
    const int i = A.steps[cu.st].x;
    const int j = cu.pass == 0 ? cu.jj : ns - 2 - cu.jj;
    const int M = A.probs[(long long)i * ns + j].M;
    cu.r0 += rec_rows(M, (int)sizeof(C), A.sb);
    if (cu.r0 < M) return;
    cu.r0 = 0;
    if (++cu.kk < (cu.dir == 0 ? K : K - 1)) return;
    cu.kk = 0;
    if (++cu.dir < 2) return;
    cu.dir = 0;
    if (++cu.jj < (cu.pass == 0 ? ns : ns - 1)) return;
    cu.jj = 0;
    if (++cu.pass == 1 && ns - 1 > 0) return;
    cu.pass = 0;
    if (++cu.st >= A.nsteps) cu.done = true;
}

// Issue the cursor's chunk into ring stage stg (16-byte aligned window).
template <typename C>
__device__ __forceinline__ void cursor_issue(const RecArgs& A, RecCursor& cu, unsigned char* ring, uint64_t* full,
                                             int stg) {
    const C* src;
    int rows, M;
    cursor_chunk<C>(A, cu, &src, &rows, &M);
    const unsigned long long a = (unsigned long long)src;
    const unsigned long long e = a + (unsigned long long)rows * M * sizeof(C);
    const unsigned long long lo = a & ~15ull;
    const unsigned bytes = (unsigned)(((e + 15ull) & ~15ull) - lo);
    mbar_expect_tx(&full[stg], bytes);
    tma_load_1d(ring + (size_t)stg * A.sb, (const void*)lo, bytes, &full[stg]);
    cursor_advance<C>(A, cu);
}

// x1-coupling of the slab's row (a1, X3 = x3) in block X2 = x2 with the
// neighbouring slab's layer at grid x1-index X1o (slot d1s = 0 for x1-1, 2 for
// x1+1): sum over the (x2, x3) neighbours.
template <typename C>
__device__ __forceinline__ C outer_coupling(const RecArgs& A, const Slab3& O, const C* ocoef, const C* ut, int a1,
                                            int x2, int x3, int d1s, int X1o) {
    const int nt = A.n_tot;
    const int qo = a1 * nt + x3;
    C v = czero<C>();
    for (int d2s = 0; d2s < 3; ++d2s) {
        const int y2 = x2 + d2s - 1;
        if (y2 < 0 || y2 >= nt) continue;
        const C* rc = ocoef + O.cf_off + (((long long)x2 * 3 + d2s) * O.M + qo) * 9 + d1s * 3;
        for (int d3s = 0; d3s < 3; ++d3s) {
            const int y3 = x3 + d3s - 1;
            if (y3 < 0 || y3 >= nt) continue;
            v = cfma(rc[d3s], ut[((long long)X1o * nt + y2) * nt + y3], v);
        }
    }
    return v;
}

// One CTA per right-hand side: the outer sweep over the slab steps, each slab
// solve an inner sweep over the sub-slab problems, each of those a forward and
// backward block substitution along x3.
template <typename C>
__global__ void __launch_bounds__(kRecThreads, 1) rec3_kernel(RecArgs A) {
    extern __shared__ __align__(128) unsigned char smr[];
    unsigned char* ring = smr;                                                  // kRecStages x A.sb
    uint64_t* full = reinterpret_cast<uint64_t*>(smr + (size_t)kRecStages * A.sb);
    C* tb = reinterpret_cast<C*>(full + kRecStages);   // step input t [Mmax]
    C* yb = tb + A.Mmax;                               // [2][Mmax]: the previous step's result, this step's
    C* ab = yb + 2 * A.Mmax;                           // D_k^{-1} t [Mmax]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    RecCursor cu{0, 0, 0, 0, 0, 0, A.nsteps == 0};
    if (tid == 0) {
        for (int q = 0; q < kRecStages; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
        for (int q = 0; q < kRecStages && !cu.done; ++q) cursor_issue<C>(A, cu, ring, full, q);
    }
    __syncthreads();
    unsigned g = 0;        // chunks consumed
    bool stop = false;     // a wait expired: the walk ends (LSS_DERR_TIMEOUT is set)
    const int nt = A.n_tot, K = A.n_tot, ns = A.n_slabs, b = A.b;
    const int r = blockIdx.x;
    const C* f = (const C*)A.f + r * A.G;
    C* ut = (C*)A.ut + r * A.G;
    C* V = (C*)A.scr + r * A.sstride;
    C* U = V + A.vsz;
    C* Y = U + A.vsz;
    const C* ocoef = (const C*)A.ocoef;
    const C* icoef = (const C*)A.icoef;
    const C* ifac = (const C*)A.ifac;
    for (int st = 0; st < A.nsteps && !stop; ++st) {
        const int i = A.steps[st].x, fl = A.steps[st].y;
        const Slab3 O = A.oslabs[i];
        const int w1 = O.w;
        const long long X1s = O.s + b;
        // ---- the slab's input V: f_i (forward) minus / the couplings (backward)
        for (long long e = tid; e < (long long)nt * nt * w1; e += blockDim.x) {
            const int a1 = (int)(e % w1), x3 = (int)((e / w1) % nt), x2 = (int)(e / ((long long)w1 * nt));
            C v = czero<C>();
            if (a1 >= O.na && a1 <= O.ll) {
                const long long x1g = X1s + a1 - O.na;
                C cpl = czero<C>();
                if ((fl & R3_CL) && a1 == O.na) cpl = cpl + outer_coupling<C>(A, O, ocoef, ut, a1, x2, x3, 0, x1g - 1);
                if ((fl & R3_CR) && a1 == O.ll) cpl = cpl + outer_coupling<C>(A, O, ocoef, ut, a1, x2, x3, 2, x1g + 1);
                v = (fl & R3_FWD) ? f[(x1g * nt + x2) * nt + x3] - cpl : cpl;
            }
            V[e] = v;
        }
        __syncthreads();
        // ---- inner sweep along x2: forward over the sub-slabs, then backward
        for (int pass = 0; pass < 2 && !stop; ++pass) {
            const int nsol = pass == 0 ? ns : ns - 1;
            for (int jj = 0; jj < nsol && !stop; ++jj) {
                const int j = pass == 0 ? jj : ns - 2 - jj;
                const int ifl = pass == 0 ? (R3_FWD | (j > 0 ? R3_CL : 0)) : R3_CR;
                const Slab3 P = A.probs[(long long)i * ns + j];
                const int M = P.M, w2 = P.w;
                const C* cf = icoef + P.cf_off;
                int cur = 0;
                for (int dir = 0; dir < 2 && !stop; ++dir) {
                    for (int kk = 0; kk < (dir == 0 ? K : K - 1) && !stop; ++kk) {
                        const int k = dir == 0 ? kk : K - 2 - kk;
                        const C* yp = yb + cur * A.Mmax;   // y_{k-1} (forward) or x_{k+1} (backward)
                        C* yn = yb + (cur ^ 1) * A.Mmax;
                        // t
                        for (int q = tid; q < M; q += blockDim.x) {
                            const int a2 = q / w1, a1 = q % w1;
                            C v = czero<C>();
                            if (dir == 0) {
                                if (a2 >= P.na && a2 <= P.ll) {
                                    const long long x2 = P.s + b + (a2 - P.na);
                                    C cpl = czero<C>();
                                    const int side = ((ifl & R3_CL) && a2 == P.na) ? 0
                                                     : (((ifl & R3_CR) && a2 == P.ll) ? 2 : -1);
                                    if (side >= 0) {   // S_i's coupling with the neighbouring x2 layer
                                        const long long x2o = x2 + side - 1;
                                        for (int d3s = 0; d3s < 3; ++d3s) {
                                            const int y3 = k + d3s - 1;
                                            if (y3 < 0 || y3 >= nt) continue;
                                            const C* rc = cf + (((long long)k * 3 + d3s) * M + q) * 9 + side * 3;
                                            for (int d1s = 0; d1s < 3; ++d1s) {
                                                const int c1 = a1 + d1s - 1;
                                                if (c1 < 0 || c1 >= w1) continue;
                                                cpl = cfma(rc[d1s], U[(x2o * nt + y3) * w1 + c1], cpl);
                                            }
                                        }
                                    }
                                    v = (ifl & R3_FWD) ? V[(x2 * nt + k) * w1 + a1] - cpl : cpl;
                                }
                                if (k > 0) {   // - C_k y_{k-1}
                                    const C* cc = cf + (((long long)k * 3 + 0) * M + q) * 9;
                                    for (int d2s = 0; d2s < 3; ++d2s) {
                                        const int c2 = a2 + d2s - 1;
                                        if (c2 < 0 || c2 >= w2) continue;
                                        for (int d1s = 0; d1s < 3; ++d1s) {
                                            const int c1 = a1 + d1s - 1;
                                            if (c1 < 0 || c1 >= w1) continue;
                                            v = v - cc[d2s * 3 + d1s] * yp[c2 * w1 + c1];
                                        }
                                    }
                                }
                            } else {           // B_k x_{k+1}
                                const C* bc = cf + (((long long)k * 3 + 2) * M + q) * 9;
                                for (int d2s = 0; d2s < 3; ++d2s) {
                                    const int c2 = a2 + d2s - 1;
                                    if (c2 < 0 || c2 >= w2) continue;
                                    for (int d1s = 0; d1s < 3; ++d1s) {
                                        const int c1 = a1 + d1s - 1;
                                        if (c1 < 0 || c1 >= w1) continue;
                                        v = cfma(bc[d2s * 3 + d1s], yp[c2 * w1 + c1], v);
                                    }
                                }
                            }
                            tb[q] = v;
                        }
                        __syncthreads();
                        // D_k^{-1} t, a warp per row, the rows streamed through the ring
                        const C* D = ifac + P.fac_off + (long long)k * M * M;
                        const int rpc = rec_rows(M, (int)sizeof(C), A.sb);
                        for (int r0 = 0; r0 < M && !stop; r0 += rpc) {
                        const int r1 = min(M, r0 + rpc), stg = (int)(g % kRecStages);
                        const bool ok = mbar_wait(&full[stg], (g / kRecStages) & 1u, A.err);
                        if (__syncthreads_or(!ok)) { stop = true; break; }
                        const unsigned off = (unsigned)((unsigned long long)(D + (long long)r0 * M) & 15ull);
                        const C* Sg = reinterpret_cast<const C*>(ring + (size_t)stg * A.sb + off);
                        for (int row = r0 + wid; row < r1; row += nw) {
                            const C* Dr = Sg + (long long)(row - r0) * M;
                            C a0 = czero<C>(), a1v = czero<C>();
                            int p = lane;
                            for (; p + 32 < M; p += 64) {
                                a0 = cfma(Dr[p], tb[p], a0);
                                a1v = cfma(Dr[p + 32], tb[p + 32], a1v);
                            }
                            if (p < M) a0 = cfma(Dr[p], tb[p], a0);
                            C acc = a0 + a1v;
                            for (int o = 16; o > 0; o >>= 1) {
                                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                            }
                            if (lane == 0) ab[row] = acc;
                        }
                        __syncthreads();   // the stage is consumed
                        if (tid == 0 && !cu.done) {
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            cursor_issue<C>(A, cu, ring, full, stg);
                        }
                        ++g;
                        }
                        if (stop) break;
                        // outputs, a thread per row (their global reads overlap)
                        const bool final_x = dir == 1 || k == K - 1;
                        for (int row = tid; row < M; row += blockDim.x) {
                            C* yk = Y + (long long)k * A.Mmax + row;
                            const C val = dir == 0 ? ab[row] : *yk - ab[row];
                            *yk = val;
                            yn[row] = val;
                            const int a2 = row / w1, a1 = row % w1;
                            if (final_x && a2 >= P.na && a2 <= P.ll) {
                                C* uu = U + ((long long)(P.s + b + (a2 - P.na)) * nt + k) * w1 + a1;
                                *uu = (ifl & R3_FWD) ? val : *uu - val;
                            }
                        }
                        __syncthreads();
                        cur ^= 1;
                    }
                }
            }
        }
        // ---- the slab's layers of the inner sweep's solution into the grid
        const int nd = O.nl;
        for (long long e = tid; e < (long long)nt * nt * nd; e += blockDim.x) {
            const int x3 = (int)(e % nt), x2 = (int)((e / nt) % nt), a = (int)(e / ((long long)nt * nt));
            const int a1 = O.na + a;
            const C uval = U[((long long)x2 * nt + x3) * w1 + a1];
            C* up = ut + ((X1s + a) * nt + x2) * nt + x3;
            *up = (fl & R3_FWD) ? uval : *up - uval;
        }
        __syncthreads();
    }
    if (stop && tid == 0) {
        // a wait expired: give the copies already issued a bounded chance to land
        const long long t0 = clock64();
        while (clock64() - t0 < 2000000ll) __nanosleep(1000);
    }
}

}  // namespace

// ---------------------------------------------------------------- host side

void lss3r_free(lss_ctx* c) {
    Rec3* q = c->d3 ? c->d3->rec : nullptr;
    if (!q) return;
    void* ptrs[] = {q->d_probs, q->gam2, q->coef64, q->coef == q->coef64 ? nullptr : q->coef, q->fac, q->W, q->X,
                    q->T, q->piv, q->rowid, q->scr, q->steps};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete q;
    c->d3->rec = nullptr;
}

int lss3r_setup(lss_ctx* c, cudaStream_t s) {
    Ctx3* d = c->d3;
    Rec3* q = new Rec3();
    d->rec = q;
    const int ns = c->n_slabs, K = c->n_tot;
    long long cf = 0, fo = 0, wo = 0;
    for (int i = 0; i < ns; ++i) {
        const Slab3& O = d->slabs[i];
        q->w1max = std::max(q->w1max, O.w);
        for (int j = 0; j < ns; ++j) {
            const Slab3& E = d->slabs[j];   // the same partition along x2
            Slab3 P{};
            P.oi = i;
            P.s = E.s;
            P.nl = E.nl;
            P.na = j > 0 ? c->b_aux : 0;
            P.nr = 0;
            P.ll = P.na + P.nl - 1;
            P.w = P.na + P.nl;
            P.nc = O.w;
            P.M = P.w * P.nc;
            P.cf_off = cf;
            P.fac_off = fo;
            P.w_off = wo;
            cf += (long long)K * 3 * P.M * 9;
            fo += (long long)K * P.M * P.M;
            wo += (long long)P.M * P.M;
            q->Mmax = std::max(q->Mmax, P.M);
            q->probs.push_back(P);
        }
    }
    if (q->Mmax > 1760) return lss_fail(c, LSS_ERR_UNSUPPORTED, "3D recursive: a sub-slab block exceeds 1760 unknowns");
    q->coef_len = cf;
    q->fac_len = fo;
    q->w_len = wo;
    const int nc = 2 * c->b + 1;
    q->nkind1 = nc + c->b_aux * (c->fronts == 2 ? 2 : 1);
    const size_t cs = c->csize();
    const int NB = c->prec == LSS_FP64 ? 8 : 16;
    const int np = ns * ns;
    int rc = LSS_OK;
    rc = rc ? rc : lss3_dalloc(c, (void**)&q->d_probs, np * sizeof(Slab3), "sub-slab problems");
    rc = rc ? rc : lss3_dalloc(c, (void**)&q->gam2,
                               (size_t)c->n_samples * c->b_aux * q->nkind1 * nc * 27 * sizeof(double2),
                               "inner auxiliary stencils");
    rc = rc ? rc : lss3_dalloc(c, (void**)&q->coef64, (size_t)cf * sizeof(double2), "sub-slab coefficients");
    if (!rc) {
        if (c->prec == LSS_FP64) q->coef = q->coef64;
        else rc = lss3_dalloc(c, &q->coef, (size_t)cf * cs, "sub-slab coefficients fp32");
    }
    // 64 bytes of slack: the factor stream copies 16-byte aligned windows that
    // may end up to 15 bytes past the last factor entry
    rc = rc ? rc : lss3_dalloc(c, &q->fac, (size_t)fo * cs + 64, "sub-slab factors");
    rc = rc ? rc : lss3_dalloc(c, &q->W, (size_t)wo * cs, "sub-slab pivot blocks");
    rc = rc ? rc : lss3_dalloc(c, &q->X, (size_t)wo * cs, "sub-slab Schur scratch");
    rc = rc ? rc : lss3_dalloc(c, &q->T, (size_t)np * NB * q->Mmax * cs, "sub-slab panel rows");
    rc = rc ? rc : lss3_dalloc(c, (void**)&q->piv, (size_t)np * NB * sizeof(int), "sub-slab pivots");
    rc = rc ? rc : lss3_dalloc(c, (void**)&q->rowid, (size_t)np * q->Mmax * sizeof(int), "sub-slab row ids");
    if (rc) return rc;
    return lss_check_cuda(c, cudaMemcpyAsync(q->d_probs, q->probs.data(), np * sizeof(Slab3), cudaMemcpyHostToDevice,
                                             s),
                          "sub-slab problems");
}

namespace {
Stencil27 rec_stencil_args(const Ctx3* d) {
    Stencil27 st;
    for (int o = 0; o < 27; ++o) {
        st.a_conj[o] = make_double2(d->alpha[o].real(), -d->alpha[o].imag());
        st.b_conj[o] = make_double2(d->beta[o].real(), -d->beta[o].imag());
    }
    return st;
}
}  // namespace

int lss3r_set_medium(lss_ctx* c, cudaStream_t s) {
    Ctx3* d = c->d3;
    Rec3* q = d->rec;
    const int n = c->n, b = c->b, nc = 2 * b + 1;
    const long long tot = (long long)c->ns_eff * c->b_aux * q->nkind1 * nc;
    const int np = c->n_slabs * c->n_slabs;
    ProfScope ps(c, s, LSS_PROF_SETUP, c->prec == LSS_MIXED ? 3 : 2);
    gamma3_aux2_kernel<<<(unsigned)((tot + kGamWarps - 1) / kGamWarps), 32 * kGamWarps, 0, s>>>(
        q->gam2, n, b, c->b_aux, c->ns_eff, c->s_lo, c->s_hi, c->pml.C / c->omega, c->h, q->nkind1);
    const int per = (int)std::min<long long>(64, ((long long)c->n_tot * q->Mmax + 255) / 256);
    assemble_rec_kernel<<<dim3(per, np), 256, 0, s>>>(q->d_probs, d->d_slabs, c->m, d->gam_phys, d->gam_aux,
                                                      d->gam_aux_r, q->gam2, rec_stencil_args(d), q->coef64, n, b,
                                                      c->b_aux, c->n_tot, c->ns_eff, c->s_lo, c->s_hi, c->omega,
                                                      q->nkind1);
    if (c->prec == LSS_MIXED)
        cast_rec_kernel<<<4 * c->num_sms, 256, 0, s>>>(q->coef64, (float2*)q->coef, q->coef_len);
    return lss_check_cuda(c, cudaGetLastError(), "3D recursive set_medium");
}

int lss3r_factor(lss_ctx* c, cudaStream_t s) {
    Rec3* q = c->d3->rec;
    FactorSet3 fs{q->d_probs, c->n_slabs * c->n_slabs, q->Mmax, q->coef, q->fac, q->W, q->X, q->T, nullptr,
                  q->piv, q->rowid, false};
    return lss3_factor_set(c, fs, s);
}

namespace {
template <typename C>
int rec_sweep_t(lss_ctx* c, const double2* r, double2* y, int R, int only, const double2* fin, cudaStream_t s) {
    Ctx3* d = c->d3;
    Rec3* q = d->rec;
    const int ns = c->n_slabs, nt = c->n_tot;
    const long long G = (long long)nt * nt * nt;
    const size_t cs = sizeof(C);
    // outer steps (device, cached per key): Algorithm 2 over the slabs, or one slab solve
    std::vector<int2> tab;
    if (only >= 0) {
        tab.push_back(make_int2(only, R3_FWD));
    } else if (c->fronts != 2) {
        for (int i = 0; i < ns; ++i) tab.push_back(make_int2(i, R3_FWD | (i > 0 ? R3_CL : 0)));
        for (int i = ns - 2; i >= 0; --i) tab.push_back(make_int2(i, R3_CR));
    } else {   // two fronts toward the middle slab, one slab solve at a time
        const int m = c->mid;
        for (int i = 0; i < m; ++i) tab.push_back(make_int2(i, R3_FWD | (i > 0 ? R3_CL : 0)));
        for (int i = ns - 1; i > m; --i) tab.push_back(make_int2(i, R3_FWD | (i < ns - 1 ? R3_CR : 0)));
        tab.push_back(make_int2(m, R3_FWD | (m > 0 ? R3_CL : 0) | (m < ns - 1 ? R3_CR : 0)));
        for (int i = m - 1; i >= 0; --i) tab.push_back(make_int2(i, R3_CR));
        for (int i = m + 1; i < ns; ++i) tab.push_back(make_int2(i, R3_CL));
    }
    int rc = LSS_OK;
    if (q->steps_key != only || !q->steps) {
        rc = lss_grow(c, &q->steps, &q->steps_cap, tab.size() * sizeof(int2));
        if (!rc) rc = lss_check_cuda(c, cudaMemcpyAsync(q->steps, tab.data(), tab.size() * sizeof(int2),
                                                        cudaMemcpyHostToDevice, s), "recursive step table");
        if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "recursive step table");
        if (rc) return rc;
        q->steps_key = only;
    }
    const long long vsz = (long long)nt * nt * q->w1max;
    const long long sstride = 2 * vsz + (long long)nt * q->Mmax;
    rc = lss_grow(c, &d->f, &d->f_cap, (size_t)R * G * cs);
    if (!rc) rc = lss_grow(c, &d->ut, &d->ut_cap, (size_t)R * G * cs);
    if (!rc) rc = lss_grow(c, &q->scr, &q->scr_cap, (size_t)R * sstride * cs);
    if (rc) return rc;
    lss3_grid_in(c, r, fin, only, 0, d->f, R, s);
    cudaMemsetAsync(d->ut, 0, (size_t)R * G * cs, s);
    RecArgs a{};
    a.oslabs = d->d_slabs;
    a.probs = q->d_probs;
    a.n_slabs = ns;
    a.n_tot = nt;
    a.b = c->b;
    a.Mmax = q->Mmax;
    a.ocoef = d->coef;
    a.icoef = q->coef;
    a.ifac = q->fac;
    a.f = d->f;
    a.ut = d->ut;
    a.G = G;
    a.scr = q->scr;
    a.vsz = vsz;
    a.sstride = sstride;
    a.steps = (const int2*)q->steps;
    a.nsteps = (int)tab.size();
    a.err = c->d_err;
    {
        ProfScope ps(c, s, LSS_PROF_SLAB_A, 1);
        const size_t vec = 4 * (size_t)q->Mmax * cs + kRecStages * sizeof(uint64_t);
        size_t sb = std::min<size_t>(kRecStageMax, vec < kRecSmem ? (kRecSmem - vec) / kRecStages : 0) & ~(size_t)15;
        if (sb < (size_t)q->Mmax * cs + 32)
            return lss_fail(c, LSS_ERR_UNSUPPORTED, "3D recursive: a sub-slab block row does not fit a stage");
        a.sb = (unsigned)sb;
        const size_t smem = (size_t)kRecStages * sb + vec;
        rc = lss_check_cuda(c, cudaFuncSetAttribute(rec3_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem), "recursive sweep attribute");
        if (rc) return rc;
        rec3_kernel<C><<<R, kRecThreads, smem, s>>>(a);
        rc = lss_check_cuda(c, cudaGetLastError(), "3D recursive sweep launch");
        if (rc) return rc;
    }
    lss3_grid_out(c, d->ut, y, only, fin != nullptr, 0, R, s);
    return lss_check_cuda(c, cudaGetLastError(), "3D recursive sweep");
}
}  // namespace

int lss3r_sweep(lss_ctx* c, const double2* r, double2* y, int R, int only, const double2* fin, cudaStream_t s) {
    if (c->prec == LSS_FP64) return rec_sweep_t<double2>(c, r, y, R, only, fin, s);
    return rec_sweep_t<float2>(c, r, y, R, only, fin, s);
}
