// Internal declarations of the 3D path (lss3d.cu).  Not part of the public
// interface (include/lss.h is).
#pragma once
#include <complex>
#include <vector>
#include <cuda_runtime.h>

struct lss_ctx;

// One slab of the 3D sweep: D_i = x1 layers [s, s+nl), preceded in its
// subproblem by na auxiliary layers; the subproblem is block tridiagonal along
// x2 with n_tot blocks of M = w * n_tot unknowns (layer a, x3 index c).
struct Slab3 {
    int s, nl, na, w, M;
    int nr;              // auxiliary layers right of D_i (two fronts)
    int ll;              // index of D_i's last layer within the subproblem: na + nl - 1
    long long cf_off;    // coefficient table offset (complex entries)
    long long fac_off;   // factor offset: n_tot dense M x M inverses
    long long w_off;     // work-matrix offset (M x M)
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
// tc_update.cu: rank-16 Gauss-Jordan update of the FP32 pivot blocks on the tensor cores (3xTF32)
int lss3_update_tc(lss_ctx* c, float2* W, const float2* T64, int J0, int NO, cudaStream_t s);
bool lss3_use_tc();

// greens.cu: cyclic Jacobi eigen-decomposition of a real symmetric matrix
void lss_jacobi_eigen(std::vector<double> A, int n, std::vector<double>& d, std::vector<double>& V);
