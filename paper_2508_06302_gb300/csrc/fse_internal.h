// Internal declarations of the FSE-Shooting CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>   // CUtensorMap (types only; the encoder is fetched at run time)
#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/fse.h"

#define FSE_MAX_D 4
#define FSE_BLK 32        // row block of the blocked triangular solves
#define FSE_NBUF_F 2      // factor buffers (step parity)
#define FSE_NBUF_KT 3     // tangent-value buffers (step index mod 3)
#define FSE_RHS_GPS 16    // row groups per pass of the right-hand-side kernel (one per warp)
#define FSE_RHS_MAXR 4    // rows per group of the right-hand-side kernel, at most
// passes of the right-hand-side kernel in flight ahead of the one computed (FP32 / FP64 tangents)
#define FSE_RHS_DEPTH_F32 3
#define FSE_RHS_DEPTH_F64 2
#define FSE_MAX_BAND 224  // half-bandwidth limit of the blocked solves

namespace fse {

// Storage used by the kernels (b = half-bandwidth, detected at setup):
//  * M, D, K, S and the sensitivity operators are CSR on the union of the
//    exact nonzero patterns of M, D, K (sorted columns, shared by all
//    trajectories); the M factor of setup uses the diagonal-major full band
//    A[c*n + i] = A(i, i+c-b).
//  * K_t(q) of the nonlinear elements is CSR on its own pattern; its values
//    are per trajectory, summed from per-element tangents in a fixed order.
//  * factor of K_eff, per trajectory: column band Lc[j*(b+1) + (i-j)], row band
//    Lr[i*(b+1) + (j-i+b)], 1/L_jj, and the inverses of the 32x32 diagonal
//    blocks Dinv[B][r][c] (lower triangular, identity padding past n).
//  * tangents of trajectory s: X[s][i][t], V[s][i][t], i < n, t < P = 2n+1
//    (d/dz0 for t < 2n, d/dw_1 for t = 2n), consecutive t contiguous.

struct Dev {
    // model (FP64)
    double* Mb = nullptr;    // full band of M (setup factor)
    double* F = nullptr;     // e x n
    int* el_type = nullptr;  // nonlinear elements sorted by colour
    int* el_dof = nullptr;   // 6 per element
    double* el_p = nullptr;  // 6 per element
    int* col_off = nullptr;  // ncolors + 1
    // CSR of the union pattern of M, D, K
    int* cs_ptr = nullptr;
    int* cs_col = nullptr;
    double* cs_m = nullptr;
    double* cs_d = nullptr;
    double* cs_k = nullptr;
    double* cs_s = nullptr;  // S of Eq. (E7) for the current w_1 (FP64)
    void* cs_A = nullptr;    // w^2 4/D^2 M + w 2/D D - K (sensitivity precision)
    void* cs_B = nullptr;    // w^2 4/D M
    // CSR of the K_t pattern and the element-tangent sources of each entry
    int* kt_ptr = nullptr;
    int* kt_col = nullptr;
    // panel factor: the lower band of S in FP32 (column band, shared by all trajectories, rebuilt
    // with the operators) and the K_t entries of the lower triangle by column: entry ktc_e[k] of the
    // CSR, column ktc_c[k], row offset ktc_r[k], k in ktc_ptr[j] .. ktc_ptr[j + 1]
    void* Sband = nullptr;
    int *ktc_ptr = nullptr, *ktc_e = nullptr, *ktc_c = nullptr, *ktc_r = nullptr;
    int* kt_slot = nullptr;  // kt_col mod RW
    // row groups of the right-hand-side kernel (rows with identical column patterns)
    int* g_pass = nullptr;   // 8 per pass: rows to stage, entry range, K_t slice (first, count), first group
    int* g_info = nullptr;   // 2 per group (even count): first entry relative to its pass, entries
    int* g_rr = nullptr;     // ng x R row records {row, K_t begin, K_t end, 0} (row -1 = padding; the
                             // K_t range relative to the pass's slice)
    int* g_map = nullptr;    // E x R CSR index of entry and row (-1 = none)
    int* g_slot = nullptr;   // E ring slot (column mod RW)
    void* g_rec = nullptr;   // E records of RB bytes: slot, then A values (R), B values (R)
    int* kt_soff = nullptr;
    int* kt_src = nullptr;   // element * 36 + a * 6 + b
    double* ke = nullptr;    // N x n_el x 36 element tangents (scratch of k_state)
    void* kt_val = nullptr;  // FSE_NBUF_KT x N x kt_ld
    // velocity tangents C_t = d f_nl / d qdot of the velocity-dependent elements (only when the
    // model has some): element scratch N x n_el x 36 and the values on the K_t pattern, same ring
    double* ce = nullptr;
    void* ct_val = nullptr;  // FSE_NBUF_KT x N x kt_ld
    void* romega = nullptr;  // 2 x N x n   right-hand side of the w_1 column
    // AFT tables
    double* phis = nullptr;  // N x (d-1)
    double* G = nullptr;     // N x U   (Eq. D2)
    double* Gi = nullptr;    // U x N   (Eq. D3)
    double* RG = nullptr;    // U x N   R(rho) Gamma^-1
    double* rc = nullptr;    // L rotation cos
    double* rs = nullptr;    // L rotation sin
    int* ktab = nullptr;     // L x (d-1)
    // factor of M (FP64)
    double* LMc = nullptr;
    double* LMr = nullptr;
    double* LMinv = nullptr;
    // trajectory state (FP64)
    double* q = nullptr;     // N x n
    double* u = nullptr;
    double* a = nullptr;
    double* zb = nullptr;    // N x 2n  (start / end points)
    // factor of K_eff (sensitivity precision), FSE_NBUF_F buffers.  The panel factor (chol_blk)
    // writes the bands, Linv and Dinv only while the tensor-core solves are selected (their records
    // are built from Lr and Dinv); it always writes Rf and Rb, which its chord solves read.  Lc is
    // also the assembled K_eff that the column-by-column factors take as input.
    void* Lc = nullptr;      // NBUF x N x n x (b+1)
    void* Lr = nullptr;
    void* Linv = nullptr;    // NBUF x N x n
    void* Dinv = nullptr;    // NBUF x N x nblk x 32 x 32
    // per 32-row block, contiguous records for the blocked tangent solves (NBUF x N x nblk x RECE):
    // forward Rf = [L(i0 + r, i0 - b + c) at c * 32 + r, c < bpad | Dinv^T], backward
    // Rb = [L(i0 + 32 + c, i0 + r) at c * 32 + r | Dinv]; entries outside the band stay zero
    void* Rf = nullptr;
    void* Rb = nullptr;
    // factor records of the tensor-core solves (FP32 tangents, b <= 96), per direction two
    // buffers (step parity) of N x (nblk + 1) x 8192 floats: record sigma + 1 holds the B operands
    // (hi | lo, K-major) of the MMAs issued after block sigma (fse_tc.cu)
    void* Tf = nullptr;
    void* Tb = nullptr;
    // tangents (sensitivity precision)
    void* X = nullptr;       // N x n x ld (columns P..ld-1 are zero padding)
    void* V = nullptr;
    void* Y = nullptr;       // right-hand side / forward-substitution buffer
    // vectors
    double* Z0 = nullptr;    // 2nU
    double* R = nullptr;     // 2nU
    double* vec = nullptr;   // scratch 2nU
    double* vec2 = nullptr;  // scratch 2nU
    double* yb = nullptr;    // N x 2n scratch
    int* status = nullptr;   // N
    int* iters = nullptr;    // N
    int* nref = nullptr;     // N  in-loop refactorisations of the per-step Newton
    int* flag = nullptr;     // 4 status words: [0] a bounded wait of a kernel gave up, [1] zero pivot of
                             // the dense LU, [2] non-positive pivot of the M factor (0 = fine)
};

struct Params {
    int n = 0, b = 0, d = 0, e = 0, N = 0, U = 0, L = 0, S1 = 0, P = 0;
    // trajectory shard: this context integrates samples s0 .. s0 + N - 1 of an N_glob-sample grid;
    // its DFT sums are then partial and complete only after the reduction across shards
    int N_glob = 0, s0 = 0;
    bool shard = false;
    int maxit = 0, prec = 0, ncolors = 0, n_el = 0, nnz = 0, nnz_kt = 0, nblk = 0;
    int ld = 0;              // row stride of the tangent arrays: P rounded up to a multiple of 4
    int RW = 0;              // ring rows of the right-hand-side kernel (two passes + 2b)
    int R = 1, ng = 0, nE = 0, ME = 0, RB = 16;   // row groups: rows per group, groups, entries,
                                                  // entries per pass (max), record bytes
    int kt_ld = 4;           // per-trajectory stride of the K_t values (nnz_kt rounded up to 4)
    int MK = 0;              // K_t entries of a pass's slice (max, a multiple of 4)
    int RWT = 0;             // ring rows of the blocked solves (power of two >= b + 32)
    int RECE = 0;            // elements of one block record of Rf / Rb: bpad * 32 + 32 * 32
    int ND = 0;              // 32-row blocks coupled to a block through the band: ceil(b / 32)
    bool tc_ok = false;      // the tensor-core solves apply (FP32 tangents, b <= 96)
    bool has_vel = false;    // some element depends on qdot (C_t != 0)
    int chol_blk = 0;        // the state kernel factors K_eff by 32-column panels (FP32, b <= 96)
    double tol = 0;
    size_t smem_state = 0, smem_rhs = 0, smem_trsm = 0;
};

}  // namespace fse

struct fse_ctx {
    fse::Params p;
    fse::Dev d;
    CUtensorMap tmX{};   // TMA maps of the tangent arrays X, V ([N][n][ld], boxes of 32 rows x the
    CUtensorMap tmV{};   // right-hand-side kernel's column tile); the type carries its own alignment
    int device = 0;
    cudaStream_t stream = nullptr;   // state path + everything ordered
    cudaStream_t stream2 = nullptr;  // sensitivity kernels (overlap with the next state step)
    std::string err;
    std::vector<int> ktab_host;
    fse_ctx* fallback = nullptr;   // FP64 context of the same problem for points the mixed form rejects
    std::vector<double> rho;
    double omega_S = -1.0;       // w_1 the operators were built for
    bool have_jac = false;
    double omega_jac = 0.0;
    cudaEvent_t ev[8] = {};
    std::vector<cudaEvent_t> ev_state, ev_sens;   // per-step ordering events
    double timing[6] = {0, 0, 0, 0, 0, 0};
    // optional per-kernel timing: events around every launch of the step loop
    bool prof = false;
    int n_steps = 0;                // 0 = the whole period
    std::vector<cudaEvent_t> pev;   // [phase][k][begin/end], phase 0 state, 1 rhs, 2 fwd, 3 bwd
    bool prof_pending = false;
    bool prof_sens = false;
    int prof_steps = 0;
    // scratch for the dense Newton solve
    double* Jd = nullptr;
    int* piv = nullptr;
    size_t Jd_cap = 0;
    // outer linear solver: FSE_LIN_AUTO / FSE_LIN_DENSE / FSE_LIN_GMRES, GMRES(m) settings,
    // its Krylov basis ((m + 1) x 2nU, allocated on first use) and the last solve's statistics
    int lin_kind = FSE_LIN_AUTO;
    double lin_rtol = 1e-8;
    int lin_restart = 40, lin_maxit = 400;
    double* kry = nullptr;
    double* kdot = nullptr;       // device scratch for the Gram-Schmidt coefficients
    size_t kry_cap = 0;
    int lin_iters = 0;
    double lin_relres = 0.0;
    int solve_kind = FSE_SOLVE_AUTO;   // banded tangent solves: FSE_SOLVE_AUTO / _SIMT / _TC
    // hyper-time form (Sec. 3.4), allocated on first use: start points, residual and two scratch
    // vectors (N x 2n each), a coefficient vector (2n U~) and Gamma R Gamma^-1 (N x N)
    double* ht = nullptr;
    bool ht_pm = false;                // Gamma R Gamma^-1 formed
    // unknown base frequencies (Sec. 3.2), allocated on first use: u border columns, u rows and
    // a GMRES-size solution / right-hand side ((2n U~ + 3) each, u <= 3)
    double* unk = nullptr;
    // reduction of partial DFT sums across trajectory shards (fse_set_reduce), nullable
    fse_reduce_fn reduce = nullptr;
    void* reduce_user = nullptr;
    bool reduce_failed = false;
};

namespace fse {

// dynamic shared memory of the state, right-hand-side and blocked-solve kernels
size_t state_smem(const Params& p);
size_t rhs_smem(const Params& p);
size_t trsm_smem(const Params& p);

// TMA maps of X and V for the right-hand-side kernel (after the allocations)
int make_tangent_maps(fse_ctx* c);

// SM count of the current device (queried once per device and cached)
inline int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int>& slot = cache[dev & 63];
    int v = slot.load();
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        slot.store(v);
    }
    return v;
}

// launchers
void ensure_constants();

// One-time set-up per device (kernel attributes, __constant__ tables): true while the current
// device's bit of `done` is clear.  The caller runs its set-up and then calls mark_device; two
// threads racing on a first use both run the (idempotent) set-up.
inline bool needs_device_setup(const std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaGetDevice(&dev);
    return (done.load() & (1ull << (dev & 63))) == 0;
}
inline void mark_device(std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaGetDevice(&dev);
    done.fetch_or(1ull << (dev & 63));
}
void launch_fill_tables(fse_ctx* c);
void launch_build_ops(fse_ctx* c, double omega1);
void launch_build_groups(fse_ctx* c);
int launch_factor_M(fse_ctx* c);
void launch_idft(fse_ctx* c, const double* Z, double* zb);
void launch_init_state(fse_ctx* c, double omega1);
void launch_state_step(fse_ctx* c, int k, double omega1, cudaStream_t st, bool sens);
void launch_sens_init(fse_ctx* c, cudaStream_t st);
void launch_sens_phase(fse_ctx* c, int k, double omega1, int phase, cudaStream_t st);
void launch_collect_end(fse_ctx* c);
void launch_dft_residual(fse_ctx* c, const double* zb, const double* Z0, double* R, int subtract);
void launch_phi_apply(fse_ctx* c, const double* zin, double* zout);
void launch_domega(fse_ctx* c, double* zout);
void launch_phi_copy(fse_ctx* c, double* Phi_dev, double* dzdw_dev);
void launch_phi_copy_one(fse_ctx* c, int s, double* Phi_dev, double* dzdw_dev);
void launch_dense_jac(fse_ctx* c, double* J);
// unknown base frequency w_{j+2} (Sec. 3.2): its column dR/dw (Eq. 23, 24) and phase-condition row
// (Eq. 18, 19) from R and Z0 (2n U~ each); the dense J bordered by u such columns and rows
void launch_unknown_border(fse_ctx* c, int j, double w, const double* R, const double* Z0, double* col,
                           double* row);
void launch_dense_jac_bordered(fse_ctx* c, int u, const double* cols, const double* rows, double* B);
// hyper-time form (Sec. 3.4): Pm = Gamma R Gamma^-1 (N x N) and the dense Jacobian of Eq. FSES_T
void launch_pmat(fse_ctx* c, double* Pm);
void launch_dense_jac_ht(fse_ctx* c, const double* Pm, double* J);
// (m + 1) x (m + 1) pseudo-arclength matrix [J dR/dw_1; t_Z^T tail] (row-major)
void launch_bordered_jac(fse_ctx* c, const double* Rw, const double* tZ, double tail, double* B);
int dense_lu_solve(fse_ctx* c, double* A, double* bvec, int m);
// tensor-core tangent solves (fse_tc.cu): per-step factor records of both directions from the
// factor of step k (record buffer k % 2, launched on the state stream right after state step k)
// and the forward (phase 1) / backward (phase 2) solve of step k
void launch_tc_records(fse_ctx* c, int k, cudaStream_t st);
void launch_tc_solve(fse_ctx* c, int k, int phase, cudaStream_t st);
// FSE_SOLVE_AUTO keeps the SIMT solves: the tensor cores' truncating FP32 accumulation makes the
// tangents of a long period drift (on the 1872-dof shell the monodromy of a 1000-step period
// differs from the SIMT one by 1e-2, enough to stall Newton's convergence)
inline bool use_tc(const fse_ctx* c) { return c->p.tc_ok && c->solve_kind == FSE_SOLVE_TC; }
int lyapunov_run(fse_ctx* c, double omega1, int N_Ly, int h, double* sigma);
// same propagation with the static device scratch of fse_aft.cu (no allocation)
int lyapunov_run_noalloc(fse_ctx* c, double omega1, int N_Ly, int h, double* sigma);

// vector helpers on the context stream (fse_aft.cu)
void vec_axpby(fse_ctx* c, size_t n, double a, const double* x, double b, double* y);
void vec_norms2(fse_ctx* c, size_t n, const double* x, const double* y, double* out_dev);
// out[i] = V_i . w for i < k (V: k x n row-major), one block per vector
void vec_mdot(fse_ctx* c, size_t n, int k, const double* V, const double* w, double* out_dev);
// w += sum_{i<k} coef[i] V_i  (coef on the device)
void vec_mupdate(fse_ctx* c, size_t n, int k, const double* V, const double* coef_dev, double* w);
void pod_expand(fse_ctx* c, size_t nu, int r, const double* mean, const double* basis, const double* coef,
                double* z);
void pod_project(fse_ctx* c, size_t nu, int r, int m, const double* mean, const double* basis, const double* Z,
                 double* coef);

// POD of m device snapshots (rows of S, m x nu; S is centred in place) on `st`:
// mean (nu), r modes (r x nu) on the device, singular values on the host (fse_mlp.cu)
int pod_build_dev(double* S, int nu, int m, int r, double* mean, double* basis, double* sing_host,
                  cudaStream_t st);

}  // namespace fse
