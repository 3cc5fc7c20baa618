// Internal declarations of the 3D path (lss3d.cu).  Not part of the public
// interface (include/lss.h is).
#pragma once
#include <complex>
#include <vector>
#include <cuda_runtime.h>

struct lss_ctx;

// One slab of the 3D sweep: D_i = x1 layers [s, s+nl), preceded in its
// subproblem by na auxiliary layers; the subproblem is block tridiagonal along
// x2 with n_tot blocks of M = w * nc unknowns (layer a, x3 index c < nc =
// n_tot).  The recursive approach reuses the record for the sub-slab problems
// of a slab subproblem: E_j = x2 layers [s, s+nl) after na auxiliary x2
// layers, block tridiagonal along x3 with n_tot blocks of M = w * nc unknowns
// (x2 layer a, x1 layer c of the slab subproblem, nc of them).
struct Slab3 {
    int s, nl, na, w, M;
    int nr;              // auxiliary layers right of D_i (two fronts)
    int ll;              // index of D_i's last layer within the subproblem: na + nl - 1
    int nc;              // extent of the second in-block index c
    int oi;              // sub-slab problems: the slab whose subproblem they split
    long long cf_off;    // coefficient table offset (complex entries)
    long long fac_off;   // factor offset: n_tot dense M x M inverses
    long long w_off;     // work-matrix offset (M x M)
};

// A batch of block-tridiagonal problems factored together (block LU along the
// block index with dense Gauss-Jordan inverses of the pivot blocks): the
// slabs, or the sub-slab problems of the recursive approach.
struct FactorSet3 {
    const Slab3* d_slabs;
    int count, Mmax;
    const void* coef;
    void* fac;
    void *W, *X, *T, *T64;
    int* piv;
    int* rowid;
    bool tc;             // rank-64 updates on the tensor cores (mixed precision, the slabs only)
};

// The recursive approach (Sec. 3.1): every slab subproblem swept along x2
// over sub-slab problems (i, j) stored at i * n_slabs + j.
struct Rec3 {
    std::vector<Slab3> probs;
    Slab3* d_probs = nullptr;
    int Mmax = 0, w1max = 0, nkind1 = 0;
    double2* gam2 = nullptr;      // inner auxiliary stencils: n_samples x b_aux x nkind1 x (2b+1) x 27
    double2* coef64 = nullptr;    // sub-slab coefficient tables, complex128
    void* coef = nullptr;         // working precision (== coef64 for FP64)
    long long coef_len = 0, fac_len = 0, w_len = 0;
    void* fac = nullptr;
    void *W = nullptr, *X = nullptr, *T = nullptr;
    int* piv = nullptr;
    int* rowid = nullptr;
    void* scr = nullptr; size_t scr_cap = 0;       // per right-hand side: slab vectors V, U and substitution vectors
    void* steps = nullptr; size_t steps_cap = 0; int steps_key = -2;   // outer step table
};

struct Ctx3 {
    std::vector<Slab3> slabs;
    Slab3* d_slabs = nullptr;
    int Mmax = 0;
    std::complex<double> alpha[27], beta[27];
    double2* khat = nullptr;      // L^3 kernel transform, [k2][k3][k1], scaled by omega^2 / L^3
    double2* gam_phys = nullptr;  // (2b+1)^3 x 27 physical PML stencils
    double2* gam_aux = nullptr;   // n_samples x b_aux x (2b+1)^2 x 27 moving-PML stencils
    double2* gam_aux_r = nullptr; // the same right of D_i (two fronts)
    double2* coef64 = nullptr;    // slab coefficient tables, complex128
    void* coef = nullptr;         // working precision (== coef64 for FP64)
    long long coef_len = 0;
    void* fac = nullptr;          // dense inverses of the pivot blocks (working precision)
    long long fac_len = 0;
    void* W = nullptr;            // pivot block being inverted, one per slab
    void* X = nullptr;            // Schur scratch D_{k-1}^{-1} B_{k-1}, one per slab
    void* T = nullptr;            // pivot rows of the current panel, per slab NB x Mmax
    void* T64 = nullptr;          // pivot rows of the current outer panel (tensor-core path), per slab 64 x Mmax
    int* piv = nullptr;           // pivot rows of the current panel, per slab NB
    int* rowid = nullptr;         // original row of each position, per slab Mmax
    long long w_len = 0;
    void* f = nullptr; size_t f_cap = 0;          // sparsified right-hand sides on the n_tot^3 grid
    void* ut = nullptr; size_t ut_cap = 0;        // sweep solution on the n_tot^3 grid
    void* Y = nullptr; size_t Y_cap = 0;          // block substitution vectors n_tot x Mmax per RHS
    double2* mvA = nullptr; size_t mvA_cap = 0;   // FFT scratch n^2 x L per RHS
    double2* mvB = nullptr; size_t mvB_cap = 0;   // FFT scratch n x L^2 per RHS
    void* TB = nullptr; size_t TB_cap = 0;        // sweep step input exchanged between CTAs (FP64)
    void* steps_all = nullptr; size_t steps_all_cap = 0; int steps_all_key = -2;   // step table, whole sweep
    void* steps_one = nullptr; size_t steps_one_cap = 0; int steps_one_key = -2;   // step table, one slab
    Rec3* rec = nullptr;          // the recursive approach's sub-slab problems (null: non-recursive)
};

void lss3_free(lss_ctx* c);
long long lss3_N(const lss_ctx* c);
int lss3_setup(lss_ctx* c, const double* m_dev, cudaStream_t s);
int lss3_set_medium(lss_ctx* c, cudaStream_t s);
int lss3_factor(lss_ctx* c, cudaStream_t s);
int lss3_sweep(lss_ctx* c, const double2* r, double2* y, int R, cudaStream_t s);
int lss3_slab_apply(lss_ctx* c, int slab, const double2* v, double2* w, int R, cudaStream_t s);
int lss3_matvec(lss_ctx* c, const double2* x, double2* y, int R, int in_mode, int out_mode, const double* dirs_dev,
                double2* uI, cudaStream_t s);
int lss3_get_stencils(const lss_ctx* c, double* alpha, double* beta);
int lss3_factor_set(lss_ctx* c, const FactorSet3& fs, cudaStream_t s);
int lss3_dalloc(lss_ctx* c, void** p, size_t bytes, const char* what);
// the sweep's grid right-hand sides (f = Q r, or a slab's layers given directly)
// and its output (restriction to I, or a slab's layers), vectors r0.. of Rc
void lss3_grid_in(lss_ctx* c, const double2* r, const double2* fin, int only, int r0, void* f, int Rc,
                  cudaStream_t s);
void lss3_grid_out(lss_ctx* c, const void* ut, double2* y, int only, bool fin, int r0, int Rc, cudaStream_t s);
// recursive3d.cu: the recursive approach
int lss3r_setup(lss_ctx* c, cudaStream_t s);
int lss3r_set_medium(lss_ctx* c, cudaStream_t s);
int lss3r_factor(lss_ctx* c, cudaStream_t s);
int lss3r_sweep(lss_ctx* c, const double2* r, double2* y, int R, int only, const double2* fin, cudaStream_t s);
void lss3r_free(lss_ctx* c);
// tc_update.cu: rank-16 Gauss-Jordan update of the FP32 pivot blocks on the tensor cores (3xTF32)
int lss3_update_tc(lss_ctx* c, float2* W, const float2* T64, int J0, int NO, cudaStream_t s);
bool lss3_use_tc();

// greens.cu: cyclic Jacobi eigen-decomposition of a real symmetric matrix
void lss_jacobi_eigen(std::vector<double> A, int n, std::vector<double>& d, std::vector<double>& V);
