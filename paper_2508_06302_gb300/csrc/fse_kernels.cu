// CUDA kernels of the FSE-Shooting hot path (sm_103a).
//
// Layouts are described in fse_internal.h.  Every kernel loop has a fixed
// bound; failures are reported through the per-trajectory status array and
// never trap.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "fse_internal.h"

namespace fse {

__constant__ double c_glx[5];   // 5-point Gauss-Legendre nodes on [-1, 1]
__constant__ double c_glw[5];   // and weights (exact for the von Karman element integrands)

static bool g_const_ready = false;

static void ensure_constants() {
    if (g_const_ready) return;
    // closed forms of the 5-point Gauss-Legendre rule
    const double r = 2.0 * sqrt(10.0 / 7.0);
    double x[5] = {-sqrt(5.0 + r) / 3.0, -sqrt(5.0 - r) / 3.0, 0.0, sqrt(5.0 - r) / 3.0,
                   sqrt(5.0 + r) / 3.0};
    const double s70 = 13.0 * sqrt(70.0);
    double w[5] = {(322.0 - s70) / 900.0, (322.0 + s70) / 900.0, 128.0 / 225.0,
                   (322.0 + s70) / 900.0, (322.0 - s70) / 900.0};
    cudaMemcpyToSymbol(c_glx, x, sizeof(x));
    cudaMemcpyToSymbol(c_glw, w, sizeof(w));
    g_const_ready = true;
}

// ----------------------------------------------------------------------------
// nonlinear elements (Eq. 1 / Eq. 25 model)
// ----------------------------------------------------------------------------

__device__ __forceinline__ double qval(const double* q, int g) { return g >= 0 ? q[g] : 0.0; }

// slope of the Hermite cubic (w1, th1, w2, th2) at xi in [-1, 1] of an element of length L
__device__ __forceinline__ void vk_slope(double xi, double L, double Nd[4]) {
    const double s = 0.5 * (xi + 1.0);
    Nd[0] = (-6.0 * s + 6.0 * s * s) / L;
    Nd[1] = 1.0 - 4.0 * s + 3.0 * s * s;
    Nd[2] = (6.0 * s - 6.0 * s * s) / L;
    Nd[3] = -2.0 * s + 3.0 * s * s;
}

// element force fe[6] (local dof order) and, if ke != nullptr, its tangent ke[36]
__device__ void elem_eval(int type, const int* dof, const double* p, const double* q, double fe[6],
                          double* ke) {
    for (int a = 0; a < 6; ++a) fe[a] = 0.0;
    if (ke)
        for (int a = 0; a < 36; ++a) ke[a] = 0.0;
    if (type == FSE_NL_CUBIC_GROUND) {
        const double x = qval(q, dof[0]);
        fe[0] = p[0] * x * x * x;
        if (ke) ke[0] = 3.0 * p[0] * x * x;
    } else if (type == FSE_NL_CUBIC_DIFF) {
        const double s = qval(q, dof[0]) - qval(q, dof[1]);
        const double f = p[0] * s * s * s;
        fe[0] = f;
        fe[1] = -f;
        if (ke) {
            const double k = 3.0 * p[0] * s * s;
            ke[0] = k;
            ke[1] = -k;
            ke[6] = -k;
            ke[7] = k;
        }
    } else if (type == FSE_NL_VK_BEAM) {
        const double EA = p[0], L = p[1];
        double loc[6];
        for (int a = 0; a < 6; ++a) loc[a] = qval(q, dof[a]);
        const double du = (loc[3] - loc[0]) / L;
        const double wb[4] = {loc[1], loc[2], loc[4], loc[5]};
        const int bidx[4] = {1, 2, 4, 5};
        const double bu[2] = {-1.0 / L, 1.0 / L};
        const int uidx[2] = {0, 3};
        for (int g = 0; g < 5; ++g) {
            const double jac = 0.5 * L * c_glw[g];
            double Nd[4];
            vk_slope(c_glx[g], L, Nd);
            const double wp = Nd[0] * wb[0] + Nd[1] * wb[1] + Nd[2] * wb[2] + Nd[3] * wb[3];
            const double fu = jac * 0.5 * EA * wp * wp;
            fe[0] += fu * bu[0];
            fe[3] += fu * bu[1];
            const double fb = jac * EA * (du * wp + 0.5 * wp * wp * wp);
            for (int c = 0; c < 4; ++c) fe[bidx[c]] += fb * Nd[c];
            if (ke) {
                const double kub = jac * EA * wp;
                for (int a = 0; a < 2; ++a)
                    for (int c = 0; c < 4; ++c) {
                        const double v = kub * bu[a] * Nd[c];
                        ke[uidx[a] * 6 + bidx[c]] += v;
                        ke[bidx[c] * 6 + uidx[a]] += v;
                    }
                const double kbb = jac * EA * (du + 1.5 * wp * wp);
                for (int c = 0; c < 4; ++c)
                    for (int c2 = 0; c2 < 4; ++c2) ke[bidx[c] * 6 + bidx[c2]] += kbb * Nd[c] * Nd[c2];
            }
        }
    }
}

__device__ __forceinline__ int elem_ndof(int type) {
    return type == FSE_NL_CUBIC_GROUND ? 1 : (type == FSE_NL_CUBIC_DIFF ? 2 : 6);
}

// ----------------------------------------------------------------------------
// small helpers
// ----------------------------------------------------------------------------

// y_i = sum_{|j-i|<=b} A_ij x_j for a diagonal-major full band A (Ad[c*n + i] = A(i, i+c-b))
__device__ __forceinline__ double band_row(const double* __restrict__ Ad, int n, int b, int i,
                                           const double* x) {
    const int lo = max(0, b - i), hi = min(2 * b, n - 1 - i + b);
    double acc = 0.0;
    for (int c = lo; c <= hi; ++c) acc += Ad[(size_t)c * n + i] * x[i + c - b];
    return acc;
}

template <typename T>
__device__ __forceinline__ double tod(T v) { return (double)v; }

// Block-wide max reduction of two values (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ void block_max2(double& a, double& b) {
    __shared__ double ra[32], rb[32];
    for (int o = 16; o > 0; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        ra[w] = a;
        rb[w] = b;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    a = 0.0;
    b = 0.0;
    for (int k = 0; k < nw; ++k) {
        a = fmax(a, ra[k]);
        b = fmax(b, rb[k]);
    }
}

// Single-warp banded solve (L L^T) x = r in place (r in shared memory, FP64
// arithmetic, factor entries of type T).  Lc: column band, Lr: row band.
template <typename T>
__device__ void warp_band_solve(const T* __restrict__ Lc, const T* __restrict__ Lr,
                                const T* __restrict__ Linv, int n, int b, double* r) {
    const int lane = threadIdx.x & 31;
    const int nb = b + 1;
    // forward, right-looking by columns
    for (int j = 0; j < n; ++j) {
        const double x = r[j] * tod(Linv[j]);
        __syncwarp();
        if (lane == 0) r[j] = x;
        for (int rr = 1 + lane; rr <= b; rr += 32) {
            const int i = j + rr;
            if (i < n) r[i] -= tod(Lc[(size_t)j * nb + rr]) * x;
        }
        __syncwarp();
    }
    // backward (L^T), right-looking by rows of L
    for (int j = n - 1; j >= 0; --j) {
        const double x = r[j] * tod(Linv[j]);
        __syncwarp();
        if (lane == 0) r[j] = x;
        for (int rr = 1 + lane; rr <= b; rr += 32) {
            const int i = j - rr;
            if (i >= 0) r[i] -= tod(Lr[(size_t)j * nb + b - rr]) * x;
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------
// AFT tables (App. D, Eq. 14) -- one kernel, FP64
// ----------------------------------------------------------------------------

__global__ void k_tables(int N, int U, int L, int dm1, const int* __restrict__ ktab,
                         const double* __restrict__ phis, const double* __restrict__ rc,
                         const double* __restrict__ rs, double* G, double* Gi, double* RG) {
    const int s = blockIdx.x;
    for (int c = threadIdx.x; c < U; c += blockDim.x) {
        double g;
        if (c == 0) {
            g = 1.0;
        } else {
            const int l = (c - 1) >> 1;
            double arg = 0.0;
            for (int j = 0; j < dm1; ++j) arg += (double)ktab[l * dm1 + j] * phis[s * dm1 + j];
            g = ((c - 1) & 1) ? sin(arg) : cos(arg);
        }
        G[(size_t)s * U + c] = g;
        Gi[(size_t)c * N + s] = (c == 0 ? 1.0 : 2.0) * g / (double)N;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < U; c += blockDim.x) {
        double v;
        if (c == 0) {
            v = Gi[s];
        } else {
            const int l = (c - 1) >> 1;
            const double gc = Gi[(size_t)(1 + 2 * l) * N + s], gs = Gi[(size_t)(2 + 2 * l) * N + s];
            v = ((c - 1) & 1) ? (rs[l] * gc + rc[l] * gs) : (rc[l] * gc - rs[l] * gs);
        }
        RG[(size_t)c * N + s] = v;
    }
}

// S = w^2 4/D^2 M + w 2/D D + K (Eq. E7), diagonal-major full band
__global__ void k_build_S(int total, double cm, double cd, const double* Mb, const double* Db,
                          const double* Kb, double* Sb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        Sb[i] = cm * Mb[i] + cd * Db[i] + Kb[i];
}

// ----------------------------------------------------------------------------
// in-CTA banded Cholesky of the column band A (global, type T) -> Lc, Lr, Linv
// ----------------------------------------------------------------------------

template <typename T>
__device__ int cta_band_cholesky(T* Ac, T* Lr, T* Linv, int n, int b, T* wnd) {
    const int nb = b + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int idx = tid; idx < nb * nb; idx += nt) {
        const int c = idx / nb;
        wnd[idx] = (c < n) ? Ac[(size_t)c * nb + (idx - c * nb)] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const int slot = j % nb;
        T* colj = wnd + slot * nb;
        const T piv = colj[0];
        if (!(piv > T(0)) || !isfinite((double)piv)) {
            if (tid == 0) bad = 1;
            __syncthreads();
            break;
        }
        const T ljj = sqrt(piv);
        const T inv = T(1) / ljj;
        __syncthreads();
        for (int r = tid; r < nb; r += nt) colj[r] = (r == 0) ? ljj : colj[r] * inv;
        __syncthreads();
        // trailing update of the window triangle
        for (int idx = tid; idx < b * nb; idx += nt) {
            const int cc = 1 + idx / nb, rr = idx % nb;
            if (cc + rr <= b && j + cc < n) {
                T* colc = wnd + ((j + cc) % nb) * nb;
                colc[rr] -= colj[cc + rr] * colj[cc];
            }
        }
        __syncthreads();
        for (int r = tid; r < nb; r += nt) {
            const T v = (j + r < n) ? colj[r] : T(0);
            Ac[(size_t)j * nb + r] = v;
            if (j + r < n) Lr[(size_t)(j + r) * nb + (b - r)] = v;
        }
        if (tid == 0) {
            Linv[j] = inv;
            if (j < b)  // zero the row-band entries left of column 0
                for (int c = 0; c < b - j; ++c) Lr[(size_t)j * nb + c] = T(0);
        }
        __syncthreads();
        const int jn = j + nb;
        for (int r = tid; r < nb; r += nt) colj[r] = (jn < n) ? Ac[(size_t)jn * nb + r] : T(0);
        __syncthreads();
    }
    __syncthreads();
    return bad;
}

// ----------------------------------------------------------------------------
// state step: one CTA per trajectory (App. E, Eq. E2-E7)
// ----------------------------------------------------------------------------

struct StateArgs {
    int n, b, e, dm1, maxit, ncolors, want_sens, init;
    double tol, Dl, a0c, a1c, a2c, w, phi;
    double rho[FSE_MAX_D - 1];
    const double *Mb, *Db, *Kb, *Sb, *F, *phis;
    const int *el_type, *el_dof, *col_off;
    const double* el_p;
    const double *LMc, *LMr, *LMinv;
    double *q, *u, *a, *Kt0;
    void *Lc, *Lr, *Linv;
    int *status, *iters;
};

__device__ __forceinline__ double forcing_i(const StateArgs& A, int s, int i, double phi) {
    double e = A.F[i] * cos(phi);
    for (int j = 1; j < A.e; ++j)
        e += A.F[(size_t)j * A.n + i] * cos(A.phis[s * A.dm1 + (j - 1)] + A.rho[j - 1] * phi);
    return e;
}

// r += f_nl(q), elements processed colour by colour (no two elements of a colour share a dof)
__device__ void add_fnl(const StateArgs& A, const double* q, double* r) {
    for (int c = 0; c < A.ncolors; ++c) {
        const int e0 = A.col_off[c], e1 = A.col_off[c + 1];
        for (int el = e0 + threadIdx.x; el < e1; el += blockDim.x) {
            const int type = A.el_type[el];
            const int* dof = A.el_dof + 6 * el;
            double fe[6];
            elem_eval(type, dof, A.el_p + 6 * el, q, fe, nullptr);
            const int nd = elem_ndof(type);
            for (int a = 0; a < nd; ++a)
                if (dof[a] >= 0) r[dof[a]] += fe[a];
        }
        __syncthreads();
    }
}

// Ac = lower col band of S + K_t(q) (type T); optionally Kt0 = col band of K_t(q) (FP64)
template <typename T>
__device__ void assemble_keff(const StateArgs& A, const double* q, T* Ac, double* Kt0) {
    const int n = A.n, b = A.b, nb = b + 1;
    for (int idx = threadIdx.x; idx < n * nb; idx += blockDim.x) {
        const int j = idx / nb, r = idx - j * nb, i = j + r;
        // S(i, j) with j = i - r  -> diagonal-major index c = j - i + b = b - r
        Ac[idx] = (i < n) ? T(A.Sb[(size_t)(b - r) * n + i]) : T(0);
        if (Kt0) Kt0[idx] = 0.0;
    }
    __syncthreads();
    for (int c = 0; c < A.ncolors; ++c) {
        const int e0 = A.col_off[c], e1 = A.col_off[c + 1];
        for (int el = e0 + threadIdx.x; el < e1; el += blockDim.x) {
            const int type = A.el_type[el];
            const int* dof = A.el_dof + 6 * el;
            double fe[6], ke[36];
            elem_eval(type, dof, A.el_p + 6 * el, q, fe, ke);
            const int nd = elem_ndof(type);
            for (int a = 0; a < nd; ++a) {
                const int ga = dof[a];
                if (ga < 0) continue;
                for (int bb = 0; bb < nd; ++bb) {
                    const int gb = dof[bb];
                    if (gb < 0 || gb > ga) continue;   // lower triangle only
                    const size_t off = (size_t)gb * nb + (ga - gb);
                    Ac[off] = Ac[off] + T(ke[a * 6 + bb]);
                    if (Kt0) Kt0[off] += ke[a * 6 + bb];
                }
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_state(StateArgs A) {
    const int s = blockIdx.x, n = A.n, b = A.b, nb = b + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ double sm[];
    double *sq = sm, *su = sq + n, *sa = su + n, *sqn = sa + n, *sb = sqn + n, *sr = sb + n;
    T* wnd = reinterpret_cast<T*>(sr + n);
    __shared__ int s_conv, s_stat;
    const size_t off = (size_t)s * n;
    T* Lc = reinterpret_cast<T*>(A.Lc) + (size_t)s * n * nb;
    T* Lr = reinterpret_cast<T*>(A.Lr) + (size_t)s * n * nb;
    T* Li = reinterpret_cast<T*>(A.Linv) + off;
    double* Kt0 = (A.init && A.want_sens) ? A.Kt0 + (size_t)s * n * nb : nullptr;
    if (tid == 0) {
        s_stat = A.init ? 0 : A.status[s];
        s_conv = 0;
    }
    for (int i = tid; i < n; i += nt) {
        sq[i] = A.q[off + i];
        su[i] = A.u[off + i];
        if (!A.init) sa[i] = A.a[off + i];
    }
    __syncthreads();
    int it = 0;
    if (A.init) {
        // consistent start: w^2 M a0 = e(0) - w D u0 - K q0 - f_nl(q0)  (Eq. E2 at phi_1 = 0)
        for (int i = tid; i < n; i += nt) sr[i] = 0.0;
        __syncthreads();
        add_fnl(A, sq, sr);
        for (int i = tid; i < n; i += nt)
            sb[i] = forcing_i(A, s, i, 0.0) - A.w * band_row(A.Db, n, b, i, su) -
                    band_row(A.Kb, n, b, i, sq) - sr[i];
        __syncthreads();
        if (tid < 32) warp_band_solve<double>(A.LMc, A.LMr, A.LMinv, n, b, sb);
        __syncthreads();
        const double iw2 = 1.0 / (A.w * A.w);
        for (int i = tid; i < n; i += nt) {
            sa[i] = sb[i] * iw2;
            A.a[off + i] = sa[i];
        }
        __syncthreads();
    } else {
        // b = e_{k+1} + w^2 M (a0 q + a1 u + a) + w D (a2 q + u)   (Eq. E7)
        for (int i = tid; i < n; i += nt) {
            sr[i] = A.a0c * sq[i] + A.a1c * su[i] + sa[i];
            sqn[i] = A.a2c * sq[i] + su[i];
        }
        __syncthreads();
        const double w2 = A.w * A.w;
        for (int i = tid; i < n; i += nt)
            sb[i] = forcing_i(A, s, i, A.phi) + w2 * band_row(A.Mb, n, b, i, sr) +
                    A.w * band_row(A.Db, n, b, i, sqn);
        __syncthreads();
        // predictor: the previous displacement q_k
        for (int i = tid; i < n; i += nt) sqn[i] = sq[i];
        __syncthreads();
        // chord Newton on Eq. (E6) with the factor of K_eff(q_k)
        for (it = 0; it < A.maxit; ++it) {
            for (int i = tid; i < n; i += nt) sr[i] = band_row(A.Sb, n, b, i, sqn) - sb[i];
            __syncthreads();
            add_fnl(A, sqn, sr);
            if (tid < 32) warp_band_solve<T>(Lc, Lr, Li, n, b, sr);
            __syncthreads();
            double dmax = 0.0, qmax = 0.0;
            for (int i = tid; i < n; i += nt) {
                const double v = sqn[i] - sr[i];
                sqn[i] = v;
                dmax = fmax(dmax, fabs(sr[i]));
                qmax = fmax(qmax, fabs(v));
            }
            block_max2(dmax, qmax);
            if (!isfinite(dmax) || !isfinite(qmax)) {
                if (tid == 0) s_stat = FSE_ENAN;
                break;
            }
            if (A.tol > 0.0 && dmax <= A.tol * qmax) {
                if (tid == 0) s_conv = 1;
                ++it;
                break;
            }
        }
        __syncthreads();
        if (tid == 0 && A.tol > 0.0 && !s_conv && s_stat == 0) s_stat = FSE_ENOCONV;
        // corrector (Eq. E5)
        for (int i = tid; i < n; i += nt) {
            const double dq = sqn[i] - sq[i];
            const double un = A.a2c * dq - su[i];
            const double an = A.a0c * dq - A.a1c * su[i] - sa[i];
            sq[i] = sqn[i];
            su[i] = un;
            sa[i] = an;
            A.q[off + i] = sqn[i];
            A.u[off + i] = un;
            A.a[off + i] = an;
        }
        __syncthreads();
    }
    // effective stiffness at the new state and its banded Cholesky factor
    assemble_keff<T>(A, sq, Lc, Kt0);
    const int bad = cta_band_cholesky<T>(Lc, Lr, Li, n, b, wnd);
    if (tid == 0) {
        if (bad && s_stat == 0) s_stat = FSE_ENONPOS_PIVOT;
        A.status[s] = s_stat;
        A.iters[s] = (A.init ? 0 : A.iters[s]) + it;
    }
}

// ----------------------------------------------------------------------------
// sensitivities: right-hand side (banded GEMM), forward and backward solves
// ----------------------------------------------------------------------------

struct SensArgs {
    int n, b, P, mode;            // mode 0: regular step, 1: initial W_0
    double w, a0c, a1c, a2c;
    const double *Mb, *Db, *Kb, *Kt0, *u, *a;
    void *X, *V, *W, *Y;
    const void *Lc, *Lr, *Linv;
    size_t Lstride;               // per-trajectory stride of the factor (0 = shared)
    size_t Lvstride;
};

// RHS[s][i][t] = w^2 sum_j M_ij Yv[j][t] + w sum_j D_ij Zv[j][t]
//   Yv = a0 X + a1 V + W,  Zv = a2 X + V;  t = 2n (the w_1 column) adds -2/w a_{k+1}, -1/w u_{k+1}
// (differentiated Eq. E6-E7).  64 x 64 output tile, 256 threads, 4 x 4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_sens_rhs(SensArgs A) {
    constexpr int BI = 64, BT = 64, KC = 16;
    __shared__ T sM[KC][BI + 1], sD[KC][BI + 1];
    __shared__ T sY[KC][BT], sZ[KC][BT];
    const int n = A.n, b = A.b, P = A.P;
    const int s = blockIdx.z;
    const int i0 = blockIdx.y * BI, t0 = blockIdx.x * BT;
    const int tid = threadIdx.x;
    const int ti = tid / 16, tt = tid % 16;   // 16 x 16 threads, 4 x 4 each
    const T* X = reinterpret_cast<const T*>(A.X) + (size_t)s * n * P;
    const T* V = reinterpret_cast<const T*>(A.V) + (size_t)s * n * P;
    const T* W = reinterpret_cast<const T*>(A.W) + (size_t)s * n * P;
    T* Y = reinterpret_cast<T*>(A.Y) + (size_t)s * n * P;
    const double* us = A.u + (size_t)s * n;
    const double* as = A.a + (size_t)s * n;
    T accM[4][4], accD[4][4];
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) accM[x][y] = accD[x][y] = T(0);
    const int jbeg = max(0, i0 - b), jend = min(n, i0 + BI + b);
    const T aw = T(2.0 / A.w), bw = T(1.0 / A.w);
    for (int j0 = jbeg; j0 < jend; j0 += KC) {
        for (int idx = tid; idx < KC * BI; idx += 256) {
            const int kk = idx / BI, ii = idx % BI;
            const int i = i0 + ii, j = j0 + kk;
            T m = T(0), d = T(0);
            if (i < n && j < jend && abs(j - i) <= b) {
                const size_t o = (size_t)(j - i + b) * n + i;
                m = T(A.Mb[o]);
                d = T(A.Db[o]);
            }
            sM[kk][ii] = m;
            sD[kk][ii] = d;
        }
        for (int idx = tid; idx < KC * BT; idx += 256) {
            const int kk = idx / BT, tq = idx % BT;
            const int j = j0 + kk, t = t0 + tq;
            T yv = T(0), zv = T(0);
            if (j < jend && t < P) {
                const size_t o = (size_t)j * P + t;
                const T x = X[o], v = V[o], wv = W[o];
                yv = T(A.a0c) * x + T(A.a1c) * v + wv;
                zv = T(A.a2c) * x + v;
                if (t == P - 1) {
                    yv -= aw * T(as[j]);
                    zv -= bw * T(us[j]);
                }
            }
            sY[kk][tq] = yv;
            sZ[kk][tq] = zv;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            T m[4], d[4], yv[4], zv[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                m[x] = sM[kk][ti * 4 + x];
                d[x] = sD[kk][ti * 4 + x];
                yv[x] = sY[kk][tt + 16 * x];
                zv[x] = sZ[kk][tt + 16 * x];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    accM[x][y] += m[x] * yv[y];
                    accD[x][y] += d[x] * zv[y];
                }
        }
        __syncthreads();
    }
    const T w2 = T(A.w * A.w), w1 = T(A.w);
    for (int x = 0; x < 4; ++x) {
        const int i = i0 + ti * 4 + x;
        if (i >= n) continue;
        for (int y = 0; y < 4; ++y) {
            const int t = t0 + tt + 16 * y;
            if (t < P) Y[(size_t)i * P + t] = w2 * accM[x][y] + w1 * accD[x][y];
        }
    }
}

// initial right-hand side of w^2 M W_0 = -(K + K_t0) X_0 - w D V_0 [- 2 w M a_0 - D u_0]
// with X_0 = [I 0 0], V_0 = [0 I 0]  (derivative of Eq. E2 at phi_1 = 0)
template <typename T>
__global__ void k_sens_init_rhs(SensArgs A) {
    const int n = A.n, b = A.b, P = A.P, nb = b + 1;
    const int s = blockIdx.y;
    T* Y = reinterpret_cast<T*>(A.Y) + (size_t)s * n * P;
    const double* Kt0 = A.Kt0 + (size_t)s * n * nb;
    const double* us = A.u + (size_t)s * n;
    const double* as = A.a + (size_t)s * n;
    const size_t total = (size_t)n * P;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / P), t = (int)(idx % P);
        double v = 0.0;
        if (t < n) {
            if (abs(t - i) <= b) {
                v = -A.Kb[(size_t)(t - i + b) * n + i];
                v -= (i >= t) ? Kt0[(size_t)t * nb + (i - t)] : Kt0[(size_t)i * nb + (t - i)];
            }
        } else if (t < 2 * n) {
            const int j = t - n;
            if (abs(j - i) <= b) v = -A.w * A.Db[(size_t)(j - i + b) * n + i];
        } else {
            v = -2.0 * A.w * band_row(A.Mb, n, b, i, as) - band_row(A.Db, n, b, i, us);
        }
        Y[idx] = T(v);
    }
}

// forward substitution L y = rhs, in place on Y; one thread per tangent direction
template <typename T>
__global__ void __launch_bounds__(128) k_sens_fwd(SensArgs A) {
    const int n = A.n, b = A.b, P = A.P, nb = b + 1;
    const int s = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    extern __shared__ unsigned char smraw[];
    T* win = reinterpret_cast<T*>(smraw);    // nb x blockDim circular window
    const T* Lr = reinterpret_cast<const T*>(A.Lr) + s * A.Lstride;
    const T* Li = reinterpret_cast<const T*>(A.Linv) + s * A.Lvstride;
    T* Y = reinterpret_cast<T*>(A.Y) + (size_t)s * n * P;
    if (t >= P) return;
    const int tl = threadIdx.x, bd = blockDim.x;
    for (int i = 0; i < n; ++i) {
        T acc = Y[(size_t)i * P + t];
        const int jlo = max(0, i - b);
        const T* Lrow = Lr + (size_t)i * nb + b;   // Lrow[j - i] = L(i, j)
        int slot = jlo % nb;
        for (int j = jlo; j < i; ++j) {
            acc -= Lrow[j - i] * win[slot * bd + tl];
            slot = (slot + 1 == nb) ? 0 : slot + 1;
        }
        const T y = acc * Li[i];
        win[(i % nb) * bd + tl] = y;
        Y[(size_t)i * P + t] = y;
    }
}

// backward substitution L^T x = y, then the Newmark update of the tangents (Eq. E5)
template <typename T>
__global__ void __launch_bounds__(128) k_sens_bwd(SensArgs A) {
    const int n = A.n, b = A.b, P = A.P, nb = b + 1;
    const int s = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    extern __shared__ unsigned char smraw[];
    T* win = reinterpret_cast<T*>(smraw);
    const T* Lc = reinterpret_cast<const T*>(A.Lc) + s * A.Lstride;
    const T* Li = reinterpret_cast<const T*>(A.Linv) + s * A.Lvstride;
    const size_t base = (size_t)s * n * P;
    T* X = reinterpret_cast<T*>(A.X) + base;
    T* V = reinterpret_cast<T*>(A.V) + base;
    T* W = reinterpret_cast<T*>(A.W) + base;
    const T* Y = reinterpret_cast<const T*>(A.Y) + base;
    if (t >= P) return;
    const int tl = threadIdx.x, bd = blockDim.x;
    const T a0 = T(A.a0c), a1 = T(A.a1c), a2 = T(A.a2c);
    const T iw2 = T(1.0 / (A.w * A.w));
    for (int i = n - 1; i >= 0; --i) {
        T acc = Y[(size_t)i * P + t];
        const int khi = min(n - 1, i + b);
        const T* Lcol = Lc + (size_t)i * nb - i;   // Lcol[k] = L(k, i)
        int slot = (i + 1) % nb;
        for (int k = i + 1; k <= khi; ++k) {
            acc -= Lcol[k] * win[slot * bd + tl];
            slot = (slot + 1 == nb) ? 0 : slot + 1;
        }
        const T x = acc * Li[i];
        win[(i % nb) * bd + tl] = x;
        const size_t o = (size_t)i * P + t;
        if (A.mode == 0) {
            const T xo = X[o], vo = V[o], wo = W[o];
            const T dx = x - xo;
            X[o] = x;
            V[o] = a2 * dx - vo;
            W[o] = a0 * dx - a1 * vo - wo;
        } else {
            W[o] = x * iw2;
            X[o] = (t == i) ? T(1) : T(0);
            V[o] = (t == i + n) ? T(1) : T(0);
        }
    }
}

// ----------------------------------------------------------------------------
// AFT: i-DFT (Eq. 20) and DFT + rotation + residual (Eq. 21, 15, 16)
// ----------------------------------------------------------------------------

__global__ void k_idft(int N, int U, int n2, const double* __restrict__ G,
                       const double* __restrict__ Z, double* zb) {
    const int s = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < U; ++c) acc += G[(size_t)s * U + c] * Z[(size_t)i * U + c];
        zb[(size_t)s * n2 + i] = acc;
    }
}

__global__ void k_split(int N, int n, const double* zb, double* q, double* u) {
    const size_t total = (size_t)N * n;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t s = idx / n, i = idx % n;
        q[idx] = zb[s * 2 * n + i];
        u[idx] = zb[s * 2 * n + n + i];
    }
}

__global__ void k_join(int N, int n, const double* q, const double* u, double* zb) {
    const size_t total = (size_t)N * n;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t s = idx / n, i = idx % n;
        zb[s * 2 * n + i] = q[idx];
        zb[s * 2 * n + n + i] = u[idx];
    }
}

// out[i*U + c] = sum_s RG[c][s] zb[s][i] - (subtract ? Z0[i*U + c] : 0); one warp per output
__global__ void k_dft_res(int N, int U, int n2, const double* __restrict__ RG,
                          const double* __restrict__ zb, const double* __restrict__ Z0, double* out,
                          int subtract) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int total = n2 * U;
    if (warp >= total) return;
    const int i = warp / U, c = warp % U;
    double acc = 0.0;
    for (int s = lane; s < N; s += 32) acc += RG[(size_t)c * N + s] * zb[(size_t)s * n2 + i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[warp] = acc - (subtract ? Z0[warp] : 0.0);
}

// ----------------------------------------------------------------------------
// Jacobian products (Eq. 22, 23) from the stored tangents
// ----------------------------------------------------------------------------

// zout[s][i] = sum_{j < 2n} Phi_s[i][j] zin[s][j],  Phi_s = [X[:, :2n]; V[:, :2n]]; one warp per (s, i)
template <typename T>
__global__ void k_phi_apply(int N, int n, int P, const T* X, const T* V, const double* zin,
                            double* zout) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int n2 = 2 * n;
    if (warp >= N * n2) return;
    const int s = warp / n2, i = warp % n2;
    const T* row = (i < n ? X + ((size_t)s * n + i) * P : V + ((size_t)s * n + (i - n)) * P);
    const double* z = zin + (size_t)s * n2;
    double acc = 0.0;
    for (int j = lane; j < n2; j += 32) acc += (double)row[j] * z[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) zout[warp] = acc;
}

template <typename T>
__global__ void k_domega_col(int N, int n, int P, const T* X, const T* V, double* zout) {
    const int n2 = 2 * n;
    const size_t total = (size_t)N * n2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t s = idx / n2;
        const int i = (int)(idx % n2);
        const T* row = (i < n ? X + (s * n + i) * P : V + (s * n + (i - n)) * P);
        zout[idx] = (double)row[P - 1];
    }
}

template <typename T>
__global__ void k_phi_copy(int N, int n, int P, const T* X, const T* V, double* Phi, double* dzdw) {
    const int n2 = 2 * n;
    const size_t total = (size_t)N * n2 * n2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t s = idx / ((size_t)n2 * n2);
        const int r = (int)((idx / n2) % n2), c = (int)(idx % n2);
        const T* row = (r < n ? X + (s * n + r) * P : V + (s * n + (r - n)) * P);
        if (Phi) Phi[idx] = (double)row[c];
        if (dzdw && c == 0) dzdw[s * n2 + r] = (double)row[P - 1];
    }
}

// dense Eq. (22): J[(i,u),(j,v)] = sum_s RG[u][s] Phi_s[i][j] G[s][v] - delta
template <typename T>
__global__ void k_dense_jac(int N, int n, int U, int P, const T* X, const T* V,
                            const double* RG, const double* G, double* J) {
    const int n2 = 2 * n;
    const size_t m = (size_t)n2 * U;
    const size_t total = m * m;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t row = idx / m, col = idx % m;
        const int i = (int)(row / U), uu = (int)(row % U);
        const int j = (int)(col / U), vv = (int)(col % U);
        double acc = 0.0;
        for (int s = 0; s < N; ++s) {
            const T* xr = (i < n ? X + ((size_t)s * n + i) * P : V + ((size_t)s * n + (i - n)) * P);
            acc += RG[(size_t)uu * N + s] * (double)xr[j] * G[(size_t)s * U + vv];
        }
        J[idx] = acc - (row == col ? 1.0 : 0.0);
    }
}

// ----------------------------------------------------------------------------
// dense LU with partial pivoting (FP64) for the outer Newton step
// ----------------------------------------------------------------------------

__global__ void k_lu_pivot(double* A, double* bvec, int* piv, int m, int k, int* flag) {
    __shared__ double sv[1024];
    __shared__ int si[1024];
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
        const double v = fabs(A[(size_t)i * m + k]);
        if (v > best) {
            best = v;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double v2 = sv[threadIdx.x + o];
            const int i2 = si[threadIdx.x + o];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const int p = si[0];
    if (threadIdx.x == 0) {
        piv[k] = p;
        if (!(sv[0] > 0.0)) *flag = 1;
    }
    if (p != k) {
        for (int c = threadIdx.x; c < m; c += blockDim.x) {
            const double t = A[(size_t)k * m + c];
            A[(size_t)k * m + c] = A[(size_t)p * m + c];
            A[(size_t)p * m + c] = t;
        }
        if (threadIdx.x == 0) {
            const double t = bvec[k];
            bvec[k] = bvec[p];
            bvec[p] = t;
        }
    }
}

__global__ void k_lu_update(double* A, double* bvec, int m, int k) {
    const double pv = A[(size_t)k * m + k];
    const int rows = m - k - 1;
    const size_t total = (size_t)rows * (m - k);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = k + 1 + (int)(idx / (m - k));
        const int c = k + (int)(idx % (m - k));
        const double l = A[(size_t)i * m + k] / pv;
        if (c == k) {
            // the multiplier is written after all reads of column k by this row are done
            continue;
        }
        A[(size_t)i * m + c] -= l * A[(size_t)k * m + c];
        if (c == k + 1) bvec[i] -= l * bvec[k];
    }
}

__global__ void k_lu_mult(double* A, int m, int k) {
    const double pv = A[(size_t)k * m + k];
    for (int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        A[(size_t)i * m + k] /= pv;
}

__global__ void k_back_subst(const double* A, double* x, int m) {
    // single block, sequential over rows, parallel dot products
    __shared__ double red[1024];
    for (int i = m - 1; i >= 0; --i) {
        double acc = 0.0;
        for (int c = i + 1 + threadIdx.x; c < m; c += blockDim.x) acc += A[(size_t)i * m + c] * x[c];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) x[i] = (x[i] - red[0]) / A[(size_t)i * m + i];
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Lyapunov exponents (App. F)
// ----------------------------------------------------------------------------

// weights w_s(phi) = sum_c H_c(phi) Gamma^-1[c][s] of the trigonometric interpolant
__global__ void k_lyap_weights(int N, int U, int dm1, const int* ktab, const double* Gi,
                               double phi0, double phi1, double phi2, double* wts) {
    const double ph[3] = {phi0, phi1, phi2};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        double acc = Gi[s];
        for (int c = 1; c < U; ++c) {
            const int l = (c - 1) >> 1;
            double arg = 0.0;
            for (int j = 0; j < dm1; ++j) arg += (double)ktab[l * dm1 + j] * ph[j];
            const double h = ((c - 1) & 1) ? sin(arg) : cos(arg);
            acc += h * Gi[(size_t)c * N + s];
        }
        wts[s] = acc;
    }
}

// A[i][c] = sum_s w_s sum_j Psi_s[i][j] Q[j][c],  Psi = diag(1, w) Phi diag(1, 1/w)  (Eq. F3)
template <typename T>
__global__ void k_lyap_prop(int N, int n, int P, int h, double w, const T* X, const T* V,
                            const double* wts, const double* Q, double* Aout) {
    const int n2 = 2 * n;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n2 * h) return;
    const int i = warp / h, c = warp % h;
    const double si = (i < n) ? 1.0 : w;
    double acc = 0.0;
    for (int s = 0; s < N; ++s) {
        const T* row = (i < n ? X + ((size_t)s * n + i) * P : V + ((size_t)s * n + (i - n)) * P);
        double a2 = 0.0;
        for (int j = lane; j < n2; j += 32) {
            const double sj = (j < n) ? 1.0 : 1.0 / w;
            a2 += (double)row[j] * sj * Q[(size_t)j * h + c];
        }
        acc += wts[s] * a2;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Aout[(size_t)i * h + c] = si * acc;
}

// classical Gram-Schmidt with re-orthogonalisation, one CTA: Q R = A; acc[c] += ln R[c][c]
__global__ void k_lyap_qr(int m, int h, double* A, double* Q, double* acc) {
    __shared__ double red[1024];
    __shared__ double coef[64];
    for (int c = 0; c < h; ++c) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int k = 0; k < c; ++k) {
                double d = 0.0;
                for (int i = threadIdx.x; i < m; i += blockDim.x) d += Q[(size_t)i * h + k] * A[(size_t)i * h + c];
                red[threadIdx.x] = d;
                __syncthreads();
                for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                    __syncthreads();
                }
                if (threadIdx.x == 0) coef[k] = red[0];
                __syncthreads();
            }
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                double v = A[(size_t)i * h + c];
                for (int k = 0; k < c; ++k) v -= coef[k] * Q[(size_t)i * h + k];
                A[(size_t)i * h + c] = v;
            }
            __syncthreads();
        }
        double d = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) d += A[(size_t)i * h + c] * A[(size_t)i * h + c];
        red[threadIdx.x] = d;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        const double nrm = sqrt(red[0]);
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) Q[(size_t)i * h + c] = A[(size_t)i * h + c] / nrm;
        if (threadIdx.x == 0) acc[c] += log(nrm);
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------

static inline int nblk(size_t total, int bs, int cap = 152 * 16) {
    size_t g = (total + bs - 1) / bs;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

void launch_fill_tables(fse_ctx* c) {
    ensure_constants();
    const Params& p = c->p;
    k_tables<<<p.N, 128, 0, c->stream>>>(p.N, p.U, p.L, p.d - 1, c->d.ktab, c->d.phis, c->d.rc,
                                         c->d.rs, c->d.G, c->d.Gi, c->d.RG);
}

void launch_build_S(fse_ctx* c, double w) {
    const Params& p = c->p;
    const double Dl = 2.0 * M_PI / p.S1;
    const double cm = w * w * 4.0 / (Dl * Dl), cd = w * 2.0 / Dl;
    const size_t total = (size_t)p.n * (2 * p.b + 1);
    k_build_S<<<nblk(total, 256), 256, 0, c->stream>>>((int)total, cm, cd, c->d.Mb, c->d.Db,
                                                       c->d.Kb, c->d.Sb);
}

// Cholesky of M (FP64) at setup: reuses the in-CTA band factorisation
__global__ void k_factor_M(int n, int b, const double* Mb, double* LMc, double* LMr, double* LMinv,
                           int* flag) {
    extern __shared__ double wndM[];
    const int nb = b + 1;
    for (int idx = threadIdx.x; idx < n * nb; idx += blockDim.x) {
        const int j = idx / nb, r = idx - j * nb, i = j + r;
        LMc[idx] = (i < n) ? Mb[(size_t)(b - r) * n + i] : 0.0;
    }
    __syncthreads();
    const int bad = cta_band_cholesky<double>(LMc, LMr, LMinv, n, b, wndM);
    if (threadIdx.x == 0) *flag = bad;
}

template <typename Tdst>
__global__ void k_convert(size_t total, const double* src, Tdst* dst) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = Tdst(src[i]);
}

int launch_factor_M(fse_ctx* c) {
    ensure_constants();
    const Params& p = c->p;
    const int nb = p.b + 1;
    int* flag = nullptr;
    cudaMalloc(&flag, sizeof(int));
    const size_t smem = (size_t)nb * nb * sizeof(double);
    cudaFuncSetAttribute(k_factor_M, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_factor_M<<<1, 256, smem, c->stream>>>(p.n, p.b, c->d.Mb, c->d.LMc, c->d.LMr, c->d.LMinv, flag);
    int h = 0;
    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(flag);
    if (p.prec == FSE_MIXED_FP32) {
        const size_t tot = (size_t)p.n * nb;
        k_convert<float><<<nblk(tot, 256), 256, 0, c->stream>>>(tot, c->d.LMc, (float*)c->d.LMc_t);
        k_convert<float><<<nblk(tot, 256), 256, 0, c->stream>>>(tot, c->d.LMr, (float*)c->d.LMr_t);
        k_convert<float><<<nblk(p.n, 256), 256, 0, c->stream>>>(p.n, c->d.LMinv, (float*)c->d.LMinv_t);
    }
    return h;
}

void launch_idft(fse_ctx* c, const double* Z, double* zb, int) {
    const Params& p = c->p;
    dim3 g((2 * p.n + 127) / 128, p.N);
    k_idft<<<g, 128, 0, c->stream>>>(p.N, p.U, 2 * p.n, c->d.G, Z, zb);
}

static StateArgs make_state_args(fse_ctx* c, double w, int want_sens, int init, int k) {
    const Params& p = c->p;
    StateArgs A;
    A.n = p.n;
    A.b = p.b;
    A.e = p.e;
    A.dm1 = p.d - 1;
    A.maxit = p.maxit;
    A.ncolors = p.ncolors;
    A.want_sens = want_sens;
    A.init = init;
    A.tol = p.tol;
    A.Dl = 2.0 * M_PI / p.S1;
    A.a0c = 4.0 / (A.Dl * A.Dl);
    A.a1c = 4.0 / A.Dl;
    A.a2c = 2.0 / A.Dl;
    A.w = w;
    A.phi = (k + 1) * A.Dl;
    for (int j = 0; j < FSE_MAX_D - 1; ++j) A.rho[j] = j < (int)c->rho.size() ? c->rho[j] : 0.0;
    A.Mb = c->d.Mb;
    A.Db = c->d.Db;
    A.Kb = c->d.Kb;
    A.Sb = c->d.Sb;
    A.F = c->d.F;
    A.phis = c->d.phis;
    A.el_type = c->d.el_type;
    A.el_dof = c->d.el_dof;
    A.col_off = c->d.col_off;
    A.el_p = c->d.el_p;
    A.LMc = c->d.LMc;
    A.LMr = c->d.LMr;
    A.LMinv = c->d.LMinv;
    A.q = c->d.q;
    A.u = c->d.u;
    A.a = c->d.a;
    A.Kt0 = c->d.Kt0;
    A.Lc = c->d.Lc;
    A.Lr = c->d.Lr;
    A.Linv = c->d.Linv;
    A.status = c->d.status;
    A.iters = c->d.iters;
    return A;
}

template <typename T>
static void state_launch(fse_ctx* c, const StateArgs& A) {
    static bool attr_set = false;
    const size_t smem = c->p.smem_state;
    if (!attr_set) {
        cudaFuncSetAttribute(k_state<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    k_state<T><<<c->p.N, 256, smem, c->stream>>>(A);
}

void launch_init_state(fse_ctx* c, double w, int want_sens) {
    ensure_constants();
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * p.n;
    k_split<<<nblk(tot, 256), 256, 0, c->stream>>>(p.N, p.n, c->d.zb, c->d.q, c->d.u);
    StateArgs A = make_state_args(c, w, want_sens, 1, -1);
    if (p.prec == FSE_MIXED_FP32)
        state_launch<float>(c, A);
    else
        state_launch<double>(c, A);
}

void launch_state_step(fse_ctx* c, int k, double w, int want_sens) {
    StateArgs A = make_state_args(c, w, want_sens, 0, k);
    if (c->p.prec == FSE_MIXED_FP32)
        state_launch<float>(c, A);
    else
        state_launch<double>(c, A);
}

static SensArgs make_sens_args(fse_ctx* c, double w, int mode) {
    const Params& p = c->p;
    SensArgs A;
    A.n = p.n;
    A.b = p.b;
    A.P = p.P;
    A.mode = mode;
    A.w = w;
    const double Dl = 2.0 * M_PI / p.S1;
    A.a0c = 4.0 / (Dl * Dl);
    A.a1c = 4.0 / Dl;
    A.a2c = 2.0 / Dl;
    A.Mb = c->d.Mb;
    A.Db = c->d.Db;
    A.Kb = c->d.Kb;
    A.Kt0 = c->d.Kt0;
    A.u = c->d.u;
    A.a = c->d.a;
    A.X = c->d.X;
    A.V = c->d.V;
    A.W = c->d.W;
    A.Y = c->d.Y;
    if (mode == 1) {
        const bool f32 = p.prec == FSE_MIXED_FP32;
        A.Lc = f32 ? c->d.LMc_t : (const void*)c->d.LMc;
        A.Lr = f32 ? c->d.LMr_t : (const void*)c->d.LMr;
        A.Linv = f32 ? c->d.LMinv_t : (const void*)c->d.LMinv;
        A.Lstride = 0;
        A.Lvstride = 0;
    } else {
        A.Lc = c->d.Lc;
        A.Lr = c->d.Lr;
        A.Linv = c->d.Linv;
        A.Lstride = (size_t)p.n * (p.b + 1);
        A.Lvstride = (size_t)p.n;
    }
    return A;
}

template <typename T>
static void sens_solves(fse_ctx* c, const SensArgs& A) {
    const Params& p = c->p;
    const int bs = 128;
    const size_t smem = (size_t)(p.b + 1) * bs * sizeof(T);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sens_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_sens_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    dim3 g((p.P + bs - 1) / bs, p.N);
    k_sens_fwd<T><<<g, bs, smem, c->stream>>>(A);
    if (c->ev[3]) cudaEventRecord(c->ev[3], c->stream);
    k_sens_bwd<T><<<g, bs, smem, c->stream>>>(A);
}

template <typename T>
static void sens_init_t(fse_ctx* c, double w) {
    const Params& p = c->p;
    SensArgs A = make_sens_args(c, w, 1);
    dim3 g(nblk((size_t)p.n * p.P, 256, 4096), p.N);
    k_sens_init_rhs<T><<<g, 256, 0, c->stream>>>(A);
    sens_solves<T>(c, A);
}

void launch_sens_init(fse_ctx* c, double w) {
    if (c->p.prec == FSE_MIXED_FP32)
        sens_init_t<float>(c, w);
    else
        sens_init_t<double>(c, w);
}

template <typename T>
static void sens_step_t(fse_ctx* c, double w, int phase) {
    const Params& p = c->p;
    SensArgs A = make_sens_args(c, w, 0);
    if (phase == 0) {
        dim3 g((p.P + 63) / 64, (p.n + 63) / 64, p.N);
        k_sens_rhs<T><<<g, 256, 0, c->stream>>>(A);
    } else {
        sens_solves<T>(c, A);
    }
}

void launch_sens_step(fse_ctx* c, double w, int phase) {
    if (c->p.prec == FSE_MIXED_FP32)
        sens_step_t<float>(c, w, phase);
    else
        sens_step_t<double>(c, w, phase);
}

void launch_collect_end(fse_ctx* c) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * p.n;
    k_join<<<nblk(tot, 256), 256, 0, c->stream>>>(p.N, p.n, c->d.q, c->d.u, c->d.zb);
}

void launch_dft_residual(fse_ctx* c, const double* zb, const double* Z0, double* R, int subtract) {
    const Params& p = c->p;
    const size_t warps = (size_t)2 * p.n * p.U;
    k_dft_res<<<(int)((warps * 32 + 255) / 256), 256, 0, c->stream>>>(p.N, p.U, 2 * p.n, c->d.RG, zb,
                                                                      Z0, R, subtract);
}

void launch_phi_apply(fse_ctx* c, const double* zin, double* zout) {
    const Params& p = c->p;
    const size_t warps = (size_t)p.N * 2 * p.n;
    const int g = (int)((warps * 32 + 255) / 256);
    if (p.prec == FSE_MIXED_FP32)
        k_phi_apply<float><<<g, 256, 0, c->stream>>>(p.N, p.n, p.P, (const float*)c->d.X,
                                                    (const float*)c->d.V, zin, zout);
    else
        k_phi_apply<double><<<g, 256, 0, c->stream>>>(p.N, p.n, p.P, (const double*)c->d.X,
                                                     (const double*)c->d.V, zin, zout);
}

void launch_domega(fse_ctx* c, double* zout) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * 2 * p.n;
    if (p.prec == FSE_MIXED_FP32)
        k_domega_col<float><<<nblk(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.P, (const float*)c->d.X,
                                                                  (const float*)c->d.V, zout);
    else
        k_domega_col<double><<<nblk(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.P, (const double*)c->d.X,
                                                                   (const double*)c->d.V, zout);
}

void launch_phi_copy(fse_ctx* c, double* Phi, double* dzdw) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * 4 * p.n * p.n;
    if (p.prec == FSE_MIXED_FP32)
        k_phi_copy<float><<<nblk(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.P, (const float*)c->d.X,
                                                                (const float*)c->d.V, Phi, dzdw);
    else
        k_phi_copy<double><<<nblk(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.P, (const double*)c->d.X,
                                                                 (const double*)c->d.V, Phi, dzdw);
}

void launch_dense_jac(fse_ctx* c, double* J) {
    const Params& p = c->p;
    const size_t m = (size_t)2 * p.n * p.U;
    if (p.prec == FSE_MIXED_FP32)
        k_dense_jac<float><<<nblk(m * m, 256, 152 * 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.P, (const float*)c->d.X, (const float*)c->d.V, c->d.RG, c->d.G, J);
    else
        k_dense_jac<double><<<nblk(m * m, 256, 152 * 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.P, (const double*)c->d.X, (const double*)c->d.V, c->d.RG, c->d.G, J);
}

int dense_lu_solve(fse_ctx* c, double* A, double* bvec, int m) {
    int* flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return FSE_ENOMEM;
    cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    for (int k = 0; k < m; ++k) {
        k_lu_pivot<<<1, 1024, 0, c->stream>>>(A, bvec, c->piv, m, k, flag);
        if (k + 1 < m) {
            const size_t tot = (size_t)(m - k - 1) * (m - k);
            k_lu_update<<<nblk(tot, 256, 152 * 32), 256, 0, c->stream>>>(A, bvec, m, k);
            k_lu_mult<<<nblk(m - k - 1, 256), 256, 0, c->stream>>>(A, m, k);
        }
    }
    k_back_subst<<<1, 1024, 0, c->stream>>>(A, bvec, m);
    int h = 0;
    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(flag);
    return h ? FSE_ENONPOS_PIVOT : FSE_OK;
}

int lyapunov_run(fse_ctx* c, double w, int N_Ly, int h, double* sigma) {
    const Params& p = c->p;
    const int m = 2 * p.n;
    double *Q = nullptr, *A = nullptr, *acc = nullptr, *wts = nullptr;
    if (cudaMalloc(&Q, sizeof(double) * m * h) != cudaSuccess) return FSE_ENOMEM;
    cudaMalloc(&A, sizeof(double) * m * h);
    cudaMalloc(&acc, sizeof(double) * h);
    cudaMalloc(&wts, sizeof(double) * p.N);
    std::vector<double> Q0((size_t)m * h, 0.0);
    for (int c2 = 0; c2 < h; ++c2) Q0[(size_t)c2 * h + c2] = 1.0;
    cudaMemcpyAsync(Q, Q0.data(), sizeof(double) * m * h, cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(acc, 0, sizeof(double) * h, c->stream);
    const size_t warps = (size_t)m * h;
    const int g = (int)((warps * 32 + 255) / 256);
    for (int i = 1; i <= N_Ly; ++i) {
        double ph[3] = {0, 0, 0};
        for (int j = 0; j < p.d - 1; ++j) ph[j] = 2.0 * (i - 1) * M_PI * c->rho[j];
        k_lyap_weights<<<nblk(p.N, 128), 128, 0, c->stream>>>(p.N, p.U, p.d - 1, c->d.ktab, c->d.Gi,
                                                             ph[0], ph[1], ph[2], wts);
        if (p.prec == FSE_MIXED_FP32)
            k_lyap_prop<float><<<g, 256, 0, c->stream>>>(p.N, p.n, p.P, h, w, (const float*)c->d.X,
                                                        (const float*)c->d.V, wts, Q, A);
        else
            k_lyap_prop<double><<<g, 256, 0, c->stream>>>(p.N, p.n, p.P, h, w, (const double*)c->d.X,
                                                         (const double*)c->d.V, wts, Q, A);
        k_lyap_qr<<<1, 512, 0, c->stream>>>(m, h, A, Q, acc);
    }
    std::vector<double> hacc(h);
    cudaMemcpyAsync(hacc.data(), acc, sizeof(double) * h, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(Q);
    cudaFree(A);
    cudaFree(acc);
    cudaFree(wts);
    if (e != cudaSuccess) return FSE_ECUDA;
    const double T1 = 2.0 * M_PI / w;
    for (int j = 0; j < h; ++j) sigma[j] = hacc[j] / (N_Ly * T1);
    return FSE_OK;
}

}  // namespace fse
