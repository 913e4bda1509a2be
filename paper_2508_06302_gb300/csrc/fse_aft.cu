// AFT (Eq. 20, 21, 15, 16), structured Jacobian products (Eq. 22, 23), the dense
// outer Newton solve and the Lyapunov exponents (App. F).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "fse_common.cuh"

namespace fse {

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
        zout[idx] = (double)row[2 * n];
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
        if (dzdw && c == 0) dzdw[s * n2 + r] = (double)row[2 * n];
    }
}

// dense Eq. (22): J[(i,u),(j,v)] = sum_s RG[u][s] Phi_s[i][j] G[s][v] - delta
template <typename T>
__global__ void k_dense_jac(int N, int n, int U, int P, const T* X, const T* V,
                            const double* RG, const double* G, double* J, size_t lda) {
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
        J[row * lda + col] = acc - (row == col ? 1.0 : 0.0);
    }
}

// hyper-time form (Sec. 3.4, Eq. FSES_T): Pm = Gamma R(rho) Gamma^-1 (N x N), Pm[s][t] =
// sum_c G[s][c] RG[c][t]
__global__ void k_pmat(int N, int U, const double* __restrict__ G, const double* __restrict__ RG, double* Pm) {
    const size_t total = (size_t)N * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t s = idx / N, t = idx % N;
        double acc = 0.0;
        for (int c = 0; c < U; ++c) acc += G[s * U + c] * RG[(size_t)c * N + t];
        Pm[idx] = acc;
    }
}

// dense Jacobian of Eq. FSES_T: J[(s,i),(t,j)] = Pm[s][t] Phi_t[i][j] - delta (unknowns sample-major)
template <typename T>
__global__ void k_dense_jac_ht(int N, int n, int P, const T* X, const T* V, const double* Pm, double* J) {
    const int n2 = 2 * n;
    const size_t m = (size_t)N * n2;
    const size_t total = m * m;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t row = idx / m, col = idx % m;
        const int s = (int)(row / n2), i = (int)(row % n2);
        const int t = (int)(col / n2), j = (int)(col % n2);
        const T* xr = (i < n ? X + ((size_t)t * n + i) * P : V + ((size_t)t * n + (i - n)) * P);
        J[idx] = Pm[(size_t)s * N + t] * (double)xr[j] - (row == col ? 1.0 : 0.0);
    }
}

// border of the pseudo-arclength system: column m = dR/dw_1, row m = (t_Z, tail)
__global__ void k_border(size_t m, const double* __restrict__ Rw, const double* __restrict__ tZ, double tail,
                         double* B) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i <= m; i += (size_t)gridDim.x * blockDim.x) {
        if (i < m) {
            B[i * (m + 1) + m] = Rw[i];
            B[m * (m + 1) + i] = tZ[i];
        } else {
            B[m * (m + 1) + m] = tail;
        }
    }
}

// Unknown base frequency w_{j+2} (Sec. 3.2, Eq. 18, 19, 23, 24), one harmonic row l of the table
// (column j: k = k~_lj) acting on each (cos, sin) coefficient pair (a, b) of the 2n states:
//   col = dR/dw_{j+2} = (2 pi / w_1) (I (x) Upsilon_j) (R + Z0), Upsilon: (a, b) -> (-k b, k a)
//         ((I (x) R(rho)) Z(2 pi) = R + Z0; the trajectories do not move with an unforced w_i);
//   row = (I (x) grad_j) Z0,                         grad:    (a, b) -> (k b, -k a)
// (the phase condition of Eq. 18 on the Newton correction).  The constant coefficient gives 0.
__global__ void k_unknown_border(size_t m, int U, int dm1, int j, const int* __restrict__ ktab, double scale,
                                 const double* __restrict__ R, const double* __restrict__ Z0, double* col,
                                 double* row) {
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < m; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t i = idx / U;
        const int c = (int)(idx % U);
        if (c == 0) {
            col[idx] = 0.0;
            row[idx] = 0.0;
            continue;
        }
        const int l = (c - 1) >> 1;
        const double k = (double)ktab[l * dm1 + j];
        const size_t ci = i * U + 1 + 2 * l, si = ci + 1;
        if (((c - 1) & 1) == 0) {   // cos coefficient
            col[idx] = -scale * k * (R[si] + Z0[si]);
            row[idx] = k * Z0[si];
        } else {                    // sin coefficient
            col[idx] = scale * k * (R[ci] + Z0[ci]);
            row[idx] = -k * Z0[ci];
        }
    }
}

// border of a bordered m x m matrix with u extra columns / rows (lda = m + u): B[i][m + a] =
// cols[a][i], B[m + a][i] = rows[a][i], B[m + a][m + b] = 0
__global__ void k_border_multi(size_t m, int u, const double* __restrict__ cols, const double* __restrict__ rows,
                               double* B) {
    const size_t lda = m + u;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m + u; i += (size_t)gridDim.x * blockDim.x)
        for (int a = 0; a < u; ++a) {
            if (i < m) {
                B[i * lda + m + a] = cols[(size_t)a * m + i];
                B[(m + a) * lda + i] = rows[(size_t)a * m + i];
            } else {
                B[(m + a) * lda + i] = 0.0;
            }
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

void launch_idft(fse_ctx* c, const double* Z, double* zb) {
    const Params& p = c->p;
    dim3 g((2 * p.n + 127) / 128, p.N);
    k_idft<<<g, 128, 0, c->stream>>>(p.N, p.U, 2 * p.n, c->d.G, Z, zb);
}

void launch_collect_end(fse_ctx* c) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * p.n;
    k_join<<<nblocks(tot, 256), 256, 0, c->stream>>>(p.N, p.n, c->d.q, c->d.u, c->d.zb);
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
        k_phi_apply<float><<<g, 256, 0, c->stream>>>(p.N, p.n, p.ld, (const float*)c->d.X,
                                                    (const float*)c->d.V, zin, zout);
    else
        k_phi_apply<double><<<g, 256, 0, c->stream>>>(p.N, p.n, p.ld, (const double*)c->d.X,
                                                     (const double*)c->d.V, zin, zout);
}

void launch_domega(fse_ctx* c, double* zout) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * 2 * p.n;
    if (p.prec == FSE_MIXED_FP32)
        k_domega_col<float><<<nblocks(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.ld, (const float*)c->d.X,
                                                                  (const float*)c->d.V, zout);
    else
        k_domega_col<double><<<nblocks(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.ld, (const double*)c->d.X,
                                                                   (const double*)c->d.V, zout);
}

void launch_phi_copy(fse_ctx* c, double* Phi, double* dzdw) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * 4 * p.n * p.n;
    if (p.prec == FSE_MIXED_FP32)
        k_phi_copy<float><<<nblocks(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.ld, (const float*)c->d.X,
                                                                (const float*)c->d.V, Phi, dzdw);
    else
        k_phi_copy<double><<<nblocks(tot, 256), 256, 0, c->stream>>>(p.N, p.n, p.ld, (const double*)c->d.X,
                                                                 (const double*)c->d.V, Phi, dzdw);
}

void launch_phi_copy_one(fse_ctx* c, int s, double* Phi, double* dzdw) {
    const Params& p = c->p;
    const size_t tot = (size_t)4 * p.n * p.n;
    const size_t off = (size_t)s * p.n * p.ld;
    if (p.prec == FSE_MIXED_FP32)
        k_phi_copy<float><<<nblocks(tot, 256), 256, 0, c->stream>>>(1, p.n, p.ld, (const float*)c->d.X + off,
                                                                (const float*)c->d.V + off, Phi, dzdw);
    else
        k_phi_copy<double><<<nblocks(tot, 256), 256, 0, c->stream>>>(1, p.n, p.ld, (const double*)c->d.X + off,
                                                                 (const double*)c->d.V + off, Phi, dzdw);
}

void launch_dense_jac(fse_ctx* c, double* J) {
    const Params& p = c->p;
    const size_t m = (size_t)2 * p.n * p.U;
    if (p.prec == FSE_MIXED_FP32)
        k_dense_jac<float><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.ld, (const float*)c->d.X, (const float*)c->d.V, c->d.RG, c->d.G, J, m);
    else
        k_dense_jac<double><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.ld, (const double*)c->d.X, (const double*)c->d.V, c->d.RG, c->d.G, J, m);
}

void launch_pmat(fse_ctx* c, double* Pm) {
    const Params& p = c->p;
    k_pmat<<<nblocks((size_t)p.N * p.N, 256), 256, 0, c->stream>>>(p.N, p.U, c->d.G, c->d.RG, Pm);
}

void launch_dense_jac_ht(fse_ctx* c, const double* Pm, double* J) {
    const Params& p = c->p;
    const size_t m = (size_t)2 * p.n * p.N;
    if (p.prec == FSE_MIXED_FP32)
        k_dense_jac_ht<float><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.ld, (const float*)c->d.X, (const float*)c->d.V, Pm, J);
    else
        k_dense_jac_ht<double><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.ld, (const double*)c->d.X, (const double*)c->d.V, Pm, J);
}

void launch_bordered_jac(fse_ctx* c, const double* Rw, const double* tZ, double tail, double* B) {
    const Params& p = c->p;
    const size_t m = (size_t)2 * p.n * p.U;
    if (p.prec == FSE_MIXED_FP32)
        k_dense_jac<float><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.ld, (const float*)c->d.X, (const float*)c->d.V, c->d.RG, c->d.G, B, m + 1);
    else
        k_dense_jac<double><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.ld, (const double*)c->d.X, (const double*)c->d.V, c->d.RG, c->d.G, B, m + 1);
    k_border<<<nblocks(m + 1, 256), 256, 0, c->stream>>>(m, Rw, tZ, tail, B);
}

void launch_unknown_border(fse_ctx* c, int j, double w, const double* R, const double* Z0, double* col,
                           double* row) {
    const Params& p = c->p;
    const size_t m = (size_t)2 * p.n * p.U;
    k_unknown_border<<<nblocks(m, 256), 256, 0, c->stream>>>(m, p.U, p.d - 1, j, c->d.ktab, 2.0 * M_PI / w, R, Z0,
                                                             col, row);
}

void launch_dense_jac_bordered(fse_ctx* c, int u, const double* cols, const double* rows, double* B) {
    const Params& p = c->p;
    const size_t m = (size_t)2 * p.n * p.U;
    if (p.prec == FSE_MIXED_FP32)
        k_dense_jac<float><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.ld, (const float*)c->d.X, (const float*)c->d.V, c->d.RG, c->d.G, B, m + u);
    else
        k_dense_jac<double><<<nblocks(m * m, 256, 64), 256, 0, c->stream>>>(
            p.N, p.n, p.U, p.ld, (const double*)c->d.X, (const double*)c->d.V, c->d.RG, c->d.G, B, m + u);
    k_border_multi<<<nblocks(m + u, 256), 256, 0, c->stream>>>(m, u, cols, rows, B);
}

int dense_lu_solve(fse_ctx* c, double* A, double* bvec, int m) {
    int* flag = c->d.flag + 1;   // zero-pivot flag: the context's second status word
    cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    for (int k = 0; k < m; ++k) {
        k_lu_pivot<<<1, 1024, 0, c->stream>>>(A, bvec, c->piv, m, k, flag);
        if (k + 1 < m) {
            const size_t tot = (size_t)(m - k - 1) * (m - k);
            k_lu_update<<<nblocks(tot, 256, 32), 256, 0, c->stream>>>(A, bvec, m, k);
            k_lu_mult<<<nblocks(m - k - 1, 256), 256, 0, c->stream>>>(A, m, k);
        }
    }
    k_back_subst<<<1, 1024, 0, c->stream>>>(A, bvec, m);
    int h = 0;
    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("dense LU: ") + cudaGetErrorString(e);
        return FSE_ECUDA;
    }
    return h ? FSE_ENONPOS_PIVOT : FSE_OK;
}

int lyapunov_run(fse_ctx* c, double w, int N_Ly, int h, double* sigma) {
    const Params& p = c->p;
    const int m = 2 * p.n;
    double *Q = nullptr, *A = nullptr, *acc = nullptr, *wts = nullptr;
    cudaError_t ea = cudaMalloc(&Q, sizeof(double) * m * h);
    if (ea == cudaSuccess) ea = cudaMalloc(&A, sizeof(double) * m * h);
    if (ea == cudaSuccess) ea = cudaMalloc(&acc, sizeof(double) * h);
    if (ea == cudaSuccess) ea = cudaMalloc(&wts, sizeof(double) * p.N);
    if (ea != cudaSuccess) {
        // nothing has been launched: free what was allocated and report before any kernel runs
        cudaGetLastError();
        for (double* q : {Q, A, acc, wts})
            if (q) cudaFree(q);
        c->err = std::string("Lyapunov scratch allocation failed: ") + cudaGetErrorString(ea);
        return FSE_ENOMEM;
    }
    std::vector<double> Q0((size_t)m * h, 0.0);
    for (int c2 = 0; c2 < h; ++c2) Q0[(size_t)c2 * h + c2] = 1.0;
    cudaMemcpyAsync(Q, Q0.data(), sizeof(double) * m * h, cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(acc, 0, sizeof(double) * h, c->stream);
    const size_t warps = (size_t)m * h;
    const int g = (int)((warps * 32 + 255) / 256);
    for (int i = 1; i <= N_Ly; ++i) {
        double ph[3] = {0, 0, 0};
        for (int j = 0; j < p.d - 1; ++j) ph[j] = 2.0 * (i - 1) * M_PI * c->rho[j];
        k_lyap_weights<<<nblocks(p.N, 128), 128, 0, c->stream>>>(p.N, p.U, p.d - 1, c->d.ktab, c->d.Gi,
                                                             ph[0], ph[1], ph[2], wts);
        if (p.prec == FSE_MIXED_FP32)
            k_lyap_prop<float><<<g, 256, 0, c->stream>>>(p.N, p.n, p.ld, h, w, (const float*)c->d.X,
                                                        (const float*)c->d.V, wts, Q, A);
        else
            k_lyap_prop<double><<<g, 256, 0, c->stream>>>(p.N, p.n, p.ld, h, w, (const double*)c->d.X,
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
    if (e != cudaSuccess) {
        c->err = std::string("Lyapunov run: ") + cudaGetErrorString(e);
        return FSE_ECUDA;
    }
    const double T1 = 2.0 * M_PI / w;
    for (int j = 0; j < h; ++j) sigma[j] = hacc[j] / (N_Ly * T1);
    return FSE_OK;
}

}  // namespace fse

// ----------------------------------------------------------------------------
// Lyapunov propagation with static device scratch (no allocation)
// ----------------------------------------------------------------------------
// Some callers must not allocate device memory while they run: a process that
// hands all of the GPU's memory to its own pool at start-up and allows no
// other allocation, or a latency-bound loop that cannot take the device-wide
// synchronisation that cudaFree implies.  For them the propagation's scratch
// (the Q and A blocks, the ln|R_jj| accumulators and the interpolation
// weights) is one fixed-size array in the library's device image: every GPU
// that loads the library holds its 4.5 MiB until the process exits.  All calls
// share it and it keeps the last call's contents, so each call sets Q and the
// accumulators before use, and calls that overlap on the GPU race on it.

namespace {

constexpr size_t kNoallocQ = FSE_NOALLOC_MAX_QH;   // doubles of Q (and of A)
constexpr size_t kNoallocAcc = 64;                  // ln|R_jj| accumulators (h <= 64)
constexpr size_t kNoallocW = FSE_NOALLOC_MAX_N;     // interpolation weights (one per trajectory)

// In host code this name is only a stand-in for the symbol, never a device
// address: the address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_lyap_scratch[2 * kNoallocQ + kNoallocAcc + kNoallocW];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_dev[kMaxDevices] = {};   // device address of g_lyap_scratch, per device ordinal

// Q = [I_h; 0] (m x h, row-major) and acc = 0
__global__ void k_lyap_init(int m, int h, double* Q, double* acc) {
    const size_t total = (size_t)m * h;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(x / h), col = (int)(x % h);
        Q[x] = (i == col) ? 1.0 : 0.0;
        if (x < (size_t)h) acc[x] = 0.0;
    }
}

}  // namespace

namespace fse {

// Device address of the static scratch on `device` (which must be current);
// looked up on the first call per device and cached.
static int noalloc_scratch(fse_ctx* c, double** out) {
    if (c->device < 0 || c->device >= kMaxDevices) {
        c->err = "static scratch: device ordinal out of range";
        return FSE_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[c->device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_lyap_scratch);
        if (e != cudaSuccess || !ptr) {
            c->err = std::string("static scratch: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return FSE_ECUDA;
        }
        g_scratch_dev[c->device] = (double*)ptr;
    }
    *out = g_scratch_dev[c->device];
    return FSE_OK;
}

int lyapunov_run_noalloc(fse_ctx* c, double w, int N_Ly, int h, double* sigma) {
    const Params& p = c->p;
    const int m = 2 * p.n;
    if (h < 1 || (size_t)h > kNoallocAcc || (size_t)m * h > kNoallocQ || (size_t)p.N > kNoallocW) {
        c->err = "static scratch: size beyond its maximum";
        return FSE_EINVAL;
    }
    double* base = nullptr;
    const int rc = noalloc_scratch(c, &base);
    if (rc) return rc;
    double* Q = base;
    double* A = base + kNoallocQ;
    double* acc = base + 2 * kNoallocQ;
    double* wts = acc + kNoallocAcc;
    k_lyap_init<<<nblocks((size_t)m * h, 256), 256, 0, c->stream>>>(m, h, Q, acc);
    const size_t warps = (size_t)m * h;
    const int g = (int)((warps * 32 + 255) / 256);
    for (int i = 1; i <= N_Ly; ++i) {
        double ph[3] = {0, 0, 0};
        for (int j = 0; j < p.d - 1; ++j) ph[j] = 2.0 * (i - 1) * M_PI * c->rho[j];
        k_lyap_weights<<<nblocks(p.N, 128), 128, 0, c->stream>>>(p.N, p.U, p.d - 1, c->d.ktab, c->d.Gi,
                                                             ph[0], ph[1], ph[2], wts);
        if (p.prec == FSE_MIXED_FP32)
            k_lyap_prop<float><<<g, 256, 0, c->stream>>>(p.N, p.n, p.ld, h, w, (const float*)c->d.X,
                                                        (const float*)c->d.V, wts, Q, A);
        else
            k_lyap_prop<double><<<g, 256, 0, c->stream>>>(p.N, p.n, p.ld, h, w, (const double*)c->d.X,
                                                         (const double*)c->d.V, wts, Q, A);
        k_lyap_qr<<<1, 512, 0, c->stream>>>(m, h, A, Q, acc);
    }
    double hacc[kNoallocAcc];
    cudaMemcpyAsync(hacc, acc, sizeof(double) * h, cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("static-scratch Lyapunov run: ") + cudaGetErrorString(e);
        return FSE_ECUDA;
    }
    const double T1 = 2.0 * M_PI / w;
    for (int j = 0; j < h; ++j) sigma[j] = hacc[j] / (N_Ly * T1);
    return FSE_OK;
}

}  // namespace fse

// ----------------------------------------------------------------------------
// small vector helpers of the outer solve and the continuation driver
// ----------------------------------------------------------------------------

namespace fse {

// y = a x + b y
__global__ void k_axpby(size_t n, double a, const double* x, double b, double* y) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        y[k] = a * x[k] + b * y[k];
}

// out[0] = sum x^2, out[1] = sum y^2 (y may be null); one block
__global__ void k_norms2(size_t n, const double* x, const double* y, double* out) {
    __shared__ double ra[1024], rb[1024];
    double a = 0.0, b = 0.0;
    for (size_t k = threadIdx.x; k < n; k += blockDim.x) {
        a += x[k] * x[k];
        if (y) b += y[k] * y[k];
    }
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ra[threadIdx.x] += ra[threadIdx.x + o];
            rb[threadIdx.x] += rb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ra[0];
        out[1] = rb[0];
    }
}

// z = mean + sum_k c_k basis[k]  (basis r x nu)
__global__ void k_pod_expand(size_t nu, int r, const double* mean, const double* basis, const double* coef,
                             double* z) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nu; x += (size_t)gridDim.x * blockDim.x) {
        double acc = mean[x];
        for (int k = 0; k < r; ++k) acc += coef[k] * basis[(size_t)k * nu + x];
        z[x] = acc;
    }
}

// coef[j][k] = basis[k] . (Z[j] - mean), one block per (j, k)
__global__ void k_pod_project(size_t nu, int r, const double* mean, const double* basis, const double* Z,
                              double* coef) {
    const int j = blockIdx.x, k = blockIdx.y;
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t x = threadIdx.x; x < nu; x += blockDim.x)
        acc += basis[(size_t)k * nu + x] * (Z[(size_t)j * nu + x] - mean[x]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) coef[(size_t)j * r + k] = red[0];
}

// out[i] = V_i . w, one block per Krylov vector
__global__ void k_mdot(size_t n, const double* __restrict__ V, const double* __restrict__ w, double* out) {
    const int i = blockIdx.x;
    __shared__ double red[512];
    double acc = 0.0;
    const double* v = V + (size_t)i * n;
    for (size_t x = threadIdx.x; x < n; x += blockDim.x) acc += v[x] * w[x];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = red[0];
}

// w += sum_{i<k} coef[i] V_i
__global__ void k_mupdate(size_t n, int k, const double* __restrict__ V, const double* __restrict__ coef,
                          double* w) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        double acc = w[x];
        for (int i = 0; i < k; ++i) acc += coef[i] * V[(size_t)i * n + x];
        w[x] = acc;
    }
}

void vec_mdot(fse_ctx* c, size_t n, int k, const double* V, const double* w, double* out_dev) {
    k_mdot<<<k, 512, 0, c->stream>>>(n, V, w, out_dev);
}

void vec_mupdate(fse_ctx* c, size_t n, int k, const double* V, const double* coef_dev, double* w) {
    k_mupdate<<<nblocks(n, 256), 256, 0, c->stream>>>(n, k, V, coef_dev, w);
}

void vec_axpby(fse_ctx* c, size_t n, double a, const double* x, double b, double* y) {
    k_axpby<<<nblocks(n, 256), 256, 0, c->stream>>>(n, a, x, b, y);
}

void vec_norms2(fse_ctx* c, size_t n, const double* x, const double* y, double* out_dev) {
    k_norms2<<<1, 1024, 0, c->stream>>>(n, x, y, out_dev);
}

void pod_expand(fse_ctx* c, size_t nu, int r, const double* mean, const double* basis, const double* coef,
                double* z) {
    k_pod_expand<<<nblocks(nu, 256), 256, 0, c->stream>>>(nu, r, mean, basis, coef, z);
}

void pod_project(fse_ctx* c, size_t nu, int r, int m, const double* mean, const double* basis, const double* Z,
                 double* coef) {
    k_pod_project<<<dim3(m, r), 256, 0, c->stream>>>(nu, r, mean, basis, Z, coef);
}

}  // namespace fse
