// Internal context of the C ABI and the host-side launchers shared between
// translation units.  Not part of the public interface (include/lss.h is).
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>
#include <array>
#include <complex>
#include <mutex>

#include "../../include/lss.h"

// One slab of the sweep (Sec. 2.3): D_i = x1 layers [s, s+nl), preceded in its
// subproblem by na virtual auxiliary layers (Eq. Hwv_approx); w = na + nl.
struct SlabDev {
    int s;          // first x1 index of D_i
    int nl;         // layers of D_i
    int na;         // auxiliary layers left of D_i (0 for the first slab)
    int nr;         // auxiliary layers right of D_i (two fronts: the middle slab and those right of it)
    int ll;         // index of D_i's last layer within the subproblem: na + nl - 1
    int w;          // subproblem width in layers: na + nl + nr
    int ldw;        // padded block size: 16 when w <= 16, else 32 (blocks are ldw x ldw, zero outside w x w)
    int cstride;    // complex entries per block row of the coefficient table (w*9 rounded up to even)
    int bs;         // complex entries per stored block (ldw x ldw, column-major)
    long long coef_off;  // offset (complex entries) of this slab's coefficient table
    long long fac_off;   // offset (complex entries) of this slab's cyclic-reduction factors
    long long work_off;  // offset (complex entries) of this slab's factorization work blocks (per parity)
};

// Cyclic reduction along x2 (block rows k = 0..n_tot-1): level l has K_l rows,
// K_0 = n_tot, K_{l+1} = ceil(K_l / 2); the odd rows of level l are eliminated
// and its even rows form level l+1, until one row is left (L levels with more
// than one row).  Per slab the factors are stored in the order a solve reads
// them, in blocks of bs entries:
//   forward part, level l = 0..L-1: D^{-1} of the odd rows (K_l / 2 blocks),
//     then for l >= 1 the blocks C, B of the even rows (2 ceil(K_l / 2));
//   the top row's D^{-1};
//   backward part, level l = L-1..1: D^{-1}C, D^{-1}B of the odd rows
//     (2 (K_l / 2) blocks);
// then, in entries: level 0's off-diagonal bands, 6 ldw per block row (C then
// B, layer offsets -1, 0, +1; even rows first, then odd rows), and rows na and
// w-1 of level 0's D^{-1} (2 ldw per odd row).
#ifdef __CUDACC__
#define LSS_HD __host__ __device__
#else
#define LSS_HD
#endif
struct CrLevelOffs {
    int K;              // rows of the level
    long long dinv;     // block offset of the odd rows' D^{-1}
    long long cbe;      // block offset of the even rows' C, B (l >= 1)
    long long dcdb;     // block offset of the odd rows' D^{-1}C, D^{-1}B (l >= 1)
};
LSS_HD inline int cr_levels(int K0) {
    int L = 0;
    for (int K = K0; K > 1; K = (K + 1) / 2) ++L;
    return L;
}
// Level l's offsets; for l = L, K = 1 and dinv is the top inverse's block.
LSS_HD inline CrLevelOffs cr_level(int K0, int l) {
    const int L = cr_levels(K0);
    CrLevelOffs o{K0, 0, 0, 0};
    long long off = 0;   // forward part
    int k = K0;
    for (int t = 0; t <= L; ++t) {
        if (t == l) {
            o.K = k;
            o.dinv = off;
            o.cbe = t >= 1 ? off + k / 2 : 0;
        }
        if (t == L) break;
        off += k / 2;
        if (t >= 1) off += 2LL * ((k + 1) / 2);
        k = (k + 1) / 2;
    }
    if (l >= 1 && l < L) {   // backward part starts after the top block
        long long d = off + 1;
        k = K0;
        for (int t = 0; t < L; ++t) {
            if (t > l) d += 2LL * (k / 2);
            k = (k + 1) / 2;
        }
        o.dcdb = d;
    }
    return o;
}
LSS_HD inline long long cr_top_block(int K0) { return cr_level(K0, cr_levels(K0)).dinv; }
LSS_HD inline long long cr_nblocks(int K0) {
    const int L = cr_levels(K0);
    long long nb = cr_top_block(K0) + 1;
    int k = K0;
    for (int t = 0; t < L; ++t) {
        if (t >= 1) nb += 2LL * (k / 2);
        k = (k + 1) / 2;
    }
    return nb;
}
// Entries of one slab's factor area (blocks, level-0 bands, level-0 D^{-1} rows).
LSS_HD inline long long cr_fac_entries(int K0, int bs, int ldw) {
    return cr_nblocks(K0) * bs + 6LL * ldw * K0 + 2LL * ldw * (K0 / 2);
}
// Entry offsets (from a slab's factor base) of level 0's bands and of level
// 0's D^{-1} rows na and w-1.
LSS_HD inline long long cr_t0_off(int K0, int bs) { return cr_nblocks(K0) * bs; }
LSS_HD inline long long cr_p0_off(int K0, int bs, int ldw) { return cr_t0_off(K0, bs) + 6LL * ldw * K0; }
// Factorization work blocks per slab and parity: A (K_0), C and B (2 K_0) of
// every row, D^{-1}C and D^{-1}B of the odd rows (2 (K_0 / 2)).
LSS_HD inline long long cr_work_blocks(int K0) { return 4LL * K0; }

struct Ctx3;

struct lss_ctx {
    // problem
    int dim = 2, n = 0, prec = LSS_FP64;
    double omega = 0, h = 0;
    lss_pml pml{};
    lss_slab slab{};
    int b = 0, b_aux = 0, n_tot = 0, n_slabs = 0, L = 0, lgL = 0, n_samples = 0;
    int fronts = 1;               // sweeping fronts: 1 (Algorithm 2) or 2 (toward the middle slab)
    int mid = 0;                  // the middle slab (n_slabs - 1) / 2 where the two fronts meet
    int ns_eff = 0;               // samples used for the current medium (1 if m is constant)
    long long coef_len = 0;       // complex entries of the coefficient table
    double s_lo = 0, s_hi = 0;   // squared-frequency sample range
    bool factored = false;
    std::string err;

    // stencils (host copies)
    std::complex<double> alpha[9], beta[9];
    std::vector<SlabDev> slabs;

    // device data
    double* m = nullptr;          // n*n
    double2* khatT = nullptr;     // L*L, transposed (column k2 contiguous), scaled by omega^2/L^2
    double2* tw = nullptr;        // L twiddles exp(-2 pi i k / L)
    double2* gam_phys = nullptr;  // (2b+1)^2 x 9 PML stencils (row coefficients)
    double2* gam_aux = nullptr;   // n_samples x b_aux x (2b+1) x 9
    double2* gam_aux_r = nullptr; // the same for the auxiliary PML right of D_i (two fronts)
    double2* coef64 = nullptr;    // slab row coefficients, complex128
    void* coef = nullptr;         // working-precision coefficients (== coef64 for FP64)
    void* fac = nullptr;          // cyclic-reduction factors of every slab (working precision)
    void* cr_work = nullptr;      // factorization work blocks, two parities (levels alternate)
    void* iface = nullptr;        // interface maps Lambda, Gamma, Phi (and Psi with two fronts): 3 (4) x n_slabs x n_tot^2
    void* iface_t = nullptr;      // maps of the transposed sweep (built on the first adjoint use)
    bool iface_t_valid = false;
    SlabDev* d_slabs = nullptr;
    int* d_err = nullptr;
    unsigned* d_bar = nullptr;    // grid barrier words

    // workspaces (grown on demand)
    double2* mv_buf = nullptr; size_t mv_cap = 0;      // n x L x R FFT scratch
    void* f_buf = nullptr; size_t f_cap = 0;           // R x n_tot^2 sparsified rhs
    void* side_buf = nullptr; size_t side_cap = 0;     // 4 x n_slabs x n_tot x R interface vectors
    void* z_buf = nullptr; size_t z_cap = 0;           // slab-solve right-hand sides in global memory
    double2* kr_buf = nullptr; size_t kr_cap = 0;      // Krylov basis storage
    double2* red_buf = nullptr; size_t red_cap = 0;    // reduction partials
    long long work_len = 0;       // complex entries of one level work buffer
    void* io_buf = nullptr; size_t io_cap = 0;         // host-buffer solve staging
    void* dir_buf = nullptr; size_t dir_cap = 0;       // plane-wave directions
    void* gr_buf = nullptr; size_t gr_cap = 0;         // -omega^2 K mu for the medium gradient
    void* hz_buf = nullptr; size_t hz_cap = 0;         // direct Helmholtz solve: beta^* f and u on the grid
    void* ifx_buf = nullptr; size_t ifx_cap = 0;       // interface-map column blocks (all slabs, both sides)
    void* ifp_buf = nullptr; size_t ifp_cap = 0;       // interface-map problem table
    int ifp_n = 0;                                     // problems uploaded to ifp_buf
    // slab-solve chunk tables: key (first/last layers only, stage entries, chunks
    // of 16-wide blocks, chunks of 32-wide blocks) and two device arrays per key
    std::vector<std::array<long long, 4>> chunk_keys;
    std::vector<void*> chunk_dev;
    int num_sms = 0;

    // auxiliary streams (and their completion events) on which slabs of other
    // block widths factor concurrently with the first run of slabs
    std::vector<cudaStream_t> aux_stream;
    std::vector<cudaEvent_t> aux_event;
    cudaEvent_t fork_event = nullptr;

    // launch parameters picked by lss_autotune (0 / -1: the built-in choice)
    struct Tune {
        int fft_C = 0;        // columns per CTA of the FFT column pass
        int solve_bsm = -1;   // 0: slab-solve right-hand sides in global memory even when they fit shared
        int solve_nst = 0;    // slab-solve ring stages (the stages then share the free shared memory)
        int solve_nst_w = 0;  // the same for launches of 32-wide slabs only (0: as solve_nst)
        int solve_half = 0;   // 1: slab solves keep to half the shared memory (two CTAs per SM)
        int solve_nr = 1;     // right-hand sides per slab-solve CTA on 16-wide slabs (1 or 2)
        int rec_nb = 0;       // ring stages of the TMA recurrence
    } tune;

    // CUDA graphs of the FGMRES iteration body (preconditioner, operator,
    // CGS2 of basis vector j), one per (j, R, transpose), captured on
    // cap_stream once a first uncaptured solve with the same R and transpose
    // has grown every workspace; a graph is dropped when a workspace moves
    // (buf_gen changes).
    struct GraphRec { int j, R, transpose, m; unsigned long long gen; cudaGraphExec_t exec; };
    bool graphs_on = true;
    unsigned long long buf_gen = 0;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphRec> graphs;
    std::vector<std::array<long long, 4>> graph_warm;   // (R, transpose, buf_gen, m) solved once uncaptured
    void* gm_buf = nullptr; size_t gm_cap = 0;          // device GMRES state (Hessenberg, rotations, masks)
    void* seg_buf = nullptr; size_t seg_cap = 0;        // ragged batch in lockstep: the right-hand sides' segments
    void* th_buf = nullptr; size_t th_cap = 0;          // block LU of the 16-wide slabs: T_k^{-1}, V_k, Y_k per block row
    void* tq_buf = nullptr; size_t tq_cap = 0;          // block LU solves: q_k per CTA
    bool th_valid = false;                              // th_buf holds the factors of the current medium
    bool th_wanted = false;                             // a sweep used them: factorizations compute them
    int* host_flags = nullptr;                          // pinned host copies of the "RHS active" flag per iteration
    cudaEvent_t iter_ev[8] = {};                        // completion of the last iterations' flag copies

    // ragged batch (lss_setup_batch): one full context per instance, each with
    // its own stream and completion event; empty for an ordinary context
    std::vector<lss_ctx*> inst;
    std::vector<cudaStream_t> inst_stream;
    std::vector<cudaEvent_t> inst_done;
    std::vector<long long> inst_off;   // prefix sums of n_q^2 (elements per right-hand side)
    cudaEvent_t fork_ev = nullptr;

    // profiling: event pairs per kernel group, launch counters
    struct ProfRec { int cat; cudaEvent_t a, b; int launches; };
    bool prof_on = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    long long launches[LSS_PROF_NCAT] = {};

    // the 3D path's data (lss3d.cu); null for a 2D context
    Ctx3* d3 = nullptr;

    size_t csize() const { return prec == LSS_FP64 ? sizeof(double2) : sizeof(float2); }
    // points of I: n^dim
    long long npts() const { return dim == 3 ? (long long)n * n * n : (long long)n * n; }
};

// Records CUDA events around a kernel group when profiling is on and counts
// the group's launches.
struct ProfScope {
    lss_ctx* c;
    cudaStream_t s;
    int cat, n;
    cudaEvent_t a = nullptr;
    ProfScope(lss_ctx* c_, cudaStream_t s_, int cat_, int n_launch);
    ~ProfScope();
};

// Guards the once-per-kernel launch configuration (shared memory and cluster
// attributes, cached occupancy) when instances of a batch are driven from
// several host threads.
std::mutex& lss_config_mutex();
// The launch configuration applied or measured for (key, slot) on the current
// device (kernel attributes are per device, and so are cluster sizes and
// occupancy-derived grids); zero until a caller sets it.  Callers hold
// lss_config_mutex().
long long& lss_dev_cache(const void* key, int slot);

// batch.cu: ragged instances (contexts made by lss_setup_batch)
void lss_batch_free(lss_ctx* c);
int lss_batch_factor(lss_ctx* c, cudaStream_t s);
int lss_batch_plane_wave_rhs(lss_ctx* c, const double* dirs, int R, double2* g, double2* uI, cudaStream_t s);
int lss_batch_apply(lss_ctx* c, int which, const double2* x, double2* y, int R, int transpose, cudaStream_t s);
int lss_batch_solve(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
                    cudaStream_t s, int adjoint);
int lss_batch_gradient(lss_ctx* c, const double2* mu, const double2* u, const double* dirs, int R, double* grad,
                       cudaStream_t s);

// status helpers
int lss_fail(lss_ctx* c, int code, const std::string& msg);
int lss_check_cuda(lss_ctx* c, cudaError_t e, const char* what);
int lss_check_device_err(lss_ctx* c, cudaStream_t s);
int lss_grow(lss_ctx* c, void** p, size_t* cap, size_t bytes);

// greens.cu: Nystrom weights, FFT of the kernel, alpha/beta
std::complex<double> lss_cell_integral_G(int d, double omega, double h);
int lss_build_kernel(lss_ctx* c, cudaStream_t s);
int lss_build_interior_stencils(lss_ctx* c, cudaStream_t s);

// fft.cu: LS operator
enum MvIn { MV_IN_MU = 0, MV_IN_U = 1, MV_IN_PLANEWAVE = 2, MV_IN_RAW = 3 };
enum MvOut { MV_OUT_A = 0, MV_OUT_AT = 1, MV_OUT_NEG = 2 };
int lss_matvec(lss_ctx* c, const double2* x, double2* y, int R, int in_mode, int out_mode,
               const double* dirs_dev, double2* uI, cudaStream_t s);
int lss_fft_kernel_table(lss_ctx* c, const double2* kc, cudaStream_t s);  // kc: L x L -> khatT
int lss_fft_configure(lss_ctx* c);
std::vector<int> lss_fft_col_candidates(const lss_ctx* c);   // admissible column groups (autotuner)
// slab.cu: chunk tables of every solve plan under the current launch parameters
int lss_prepare_solve_tables(lss_ctx* c, cudaStream_t s);
// slab.cu: at least n - 1 auxiliary streams (with events) and the fork event
int lss_ensure_aux(lss_ctx* c, size_t n);

// stencil.cu: gamma tables, slab assembly, Q
int lss_build_gamma_phys(lss_ctx* c, cudaStream_t s);
int lss_build_gamma_aux(lss_ctx* c, cudaStream_t s);
int lss_assemble_slabs(lss_ctx* c, cudaStream_t s);
int lss_sparsify(lss_ctx* c, const double2* r, void* f, int R, cudaStream_t s);

// slab.cu: factorization, sweep
int lss_factor_slabs(lss_ctx* c, cudaStream_t s);
int lss_sweep(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s);
int lss_slab_apply(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s);
// iface.cu: interface maps Lambda, Gamma, Phi of every slab (all columns at once)
int lss_iface_maps(lss_ctx* c, cudaStream_t s);
// the three interface recurrences with the maps at `maps` (Lambda, Gamma, Phi blocks)
int lss_recurrences(lss_ctx* c, const void* maps, void* lam, void* phi, const void* a_first, const void* a_last,
                    int R, cudaStream_t s);

// adjoint.cu: the transposed preconditioner P^T = Q^T Sweep^T E^T
int lss_sweep_t(lss_ctx* c, const double2* y, double2* r, int R, cudaStream_t s);
// builds the transposed interface maps now if the factorization changed (the
// sweep would otherwise build them on first use)
int lss_prepare_sweep_t(lss_ctx* c, cudaStream_t s);
// gradient of a data misfit with respect to m from adjoint states mu (stencil.cu)
int lss_gradient_m(lss_ctx* c, const double2* Kmu, const double2* u, const double* dirs_dev, double* grad, int R,
                   cudaStream_t s);
int lss_sparsify_t(lss_ctx* c, const void* X, double2* r, int R, cudaStream_t s);
// Sec. 4 direct solver (2D): beta^* f on the grid, H on grid vectors, the sweep
// on a grid right-hand side, grid -> I
int lss_sparsify_beta(lss_ctx* c, const double2* f, double2* F, int R, cudaStream_t s);
int lss_apply_H(lss_ctx* c, const double2* x, double2* y, int R, cudaStream_t s);
int lss_sweep_grid(lss_ctx* c, const double2* F, double2* y, int R, cudaStream_t s);
int lss_extract_grid(lss_ctx* c, const double2* U, double2* u, int R, cudaStream_t s);

// krylov.cu: FGMRES
int lss_set_medium_impl(lss_ctx* c, const double* m_dev, cudaStream_t s);
int lss_fgmres(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
               cudaStream_t s, int transpose = 0);
// slab.cu: the block LU factors of the 16-wide slabs for solves with R >= 16
// right-hand sides (nothing to do for fewer, or when they are current)
int lss_thomas_prepare(lss_ctx* c, int R, cudaStream_t s);
int lss_fgmres_batch(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
                     cudaStream_t s, int transpose = 0);
// batch.cu: the operator (which = 0) or the preconditioner (1) of every
// instance of a batch, issued from the calling thread on the instances' streams
int lss_batch_op(lss_ctx* c, int which, const double2* x, double2* y, int R, int transpose, cudaStream_t s);
