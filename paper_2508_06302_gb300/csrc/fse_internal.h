// Internal declarations of the FSE-Shooting CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fse.h"

#define FSE_MAX_D 4

namespace fse {

// Banded storage used by every kernel (b = half-bandwidth, detected at setup):
//  full band  A[i*(2b+1) + (j - i + b)],  |j - i| <= b      (M, D, K, S in FP64)
//  col band   C[j*(b+1) + (i - j)],      j <= i <= j + b    (lower factor, by columns)
//  row band   R[i*(b+1) + (j - i + b)],  i - b <= j <= i    (lower factor, by rows)
// Entries outside [0, n) are stored as exact zeros.
// Sensitivities of trajectory s: X[s][i][t], i < n dofs, t < P = 2n + 1 tangent
// directions (dz0 for t < 2n, d w_1 for t = 2n), row-major so that consecutive t
// are contiguous.

struct Dev {
    // model
    double* Mb = nullptr;    // n x (2b+1)
    double* Db = nullptr;
    double* Kb = nullptr;
    double* Sb = nullptr;    // effective stiffness S of Eq. (E7), rebuilt per w_1
    double* F = nullptr;     // e x n
    int* el_type = nullptr;  // elements sorted by colour
    int* el_dof = nullptr;   // 6 per element
    double* el_p = nullptr;  // 6 per element
    int* col_off = nullptr;  // ncolors + 1
    // AFT tables
    double* phis = nullptr;  // N x (d-1)
    double* G = nullptr;     // N x U   (Eq. D2)
    double* Gi = nullptr;    // U x N   (Eq. D3)
    double* RG = nullptr;    // U x N   R(rho) Gamma^-1
    double* rc = nullptr;    // L rotation cos
    double* rs = nullptr;    // L rotation sin
    int* ktab = nullptr;     // L x (d-1)
    // factor of M (FP64) and its copy in the sensitivity precision
    double* LMc = nullptr;
    double* LMr = nullptr;
    double* LMinv = nullptr;
    void* LMc_t = nullptr;
    void* LMr_t = nullptr;
    void* LMinv_t = nullptr;
    // trajectory state (FP64)
    double* q = nullptr;     // N x n
    double* u = nullptr;
    double* a = nullptr;
    double* zb = nullptr;    // N x 2n  (start / end points)
    double* Kt0 = nullptr;   // N x n x (b+1) col band of K_t(q_0)
    // per-trajectory factor of K_eff (sensitivity precision)
    void* Lc = nullptr;      // N x n x (b+1)
    void* Lr = nullptr;      // N x n x (b+1)
    void* Linv = nullptr;    // N x n
    // sensitivities (sensitivity precision)
    void* X = nullptr;       // N x n x P
    void* V = nullptr;
    void* W = nullptr;
    void* Y = nullptr;       // right-hand side / forward-substitution buffer
    // vectors
    double* Z0 = nullptr;    // 2nU
    double* R = nullptr;     // 2nU
    double* vec = nullptr;   // scratch 2nU
    double* vec2 = nullptr;  // scratch 2nU
    double* yb = nullptr;    // N x 2n scratch
    int* status = nullptr;   // N
    int* iters = nullptr;    // N
};

struct Params {
    int n = 0, b = 0, d = 0, e = 0, N = 0, U = 0, L = 0, S1 = 0, P = 0;
    int maxit = 0, prec = 0, ncolors = 0, n_el = 0;
    double tol = 0;
    size_t smem_state = 0;
};

}  // namespace fse

struct fse_ctx {
    fse::Params p;
    fse::Dev d;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<int> ktab_host;
    std::vector<double> rho;
    double omega_S = -1.0;       // w_1 the effective stiffness was built for
    bool have_jac = false;
    bool jac_fp64 = false;
    double omega_jac = 0.0;
    cudaEvent_t ev[8] = {};
    double timing[5] = {0, 0, 0, 0, 0};
    // scratch for the dense Newton solve
    double* Jd = nullptr;
    int* piv = nullptr;
    size_t Jd_cap = 0;
};

namespace fse {

// launchers (fse_kernels.cu)
void launch_fill_tables(fse_ctx* c);
void launch_build_S(fse_ctx* c, double omega1);
int launch_factor_M(fse_ctx* c);
void launch_idft(fse_ctx* c, const double* Z, double* zb, int nvec);
void launch_init_state(fse_ctx* c, double omega1, int want_sens);
void launch_state_step(fse_ctx* c, int k, double omega1, int want_sens);
void launch_sens_init(fse_ctx* c, double omega1);
void launch_sens_step(fse_ctx* c, double omega1, int phase);
void launch_collect_end(fse_ctx* c);
void launch_dft_residual(fse_ctx* c, const double* zb, const double* Z0, double* R, int subtract);
void launch_phi_apply(fse_ctx* c, const double* zin, double* zout);
void launch_domega(fse_ctx* c, double* zout);
void launch_phi_copy(fse_ctx* c, double* Phi_dev, double* dzdw_dev);
void launch_dense_jac(fse_ctx* c, double* J);
int dense_lu_solve(fse_ctx* c, double* A, double* bvec, int m);
int lyapunov_run(fse_ctx* c, double omega1, int N_Ly, int h, double* sigma);

}  // namespace fse
