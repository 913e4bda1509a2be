// Learned continuation predictor: a 3-layer GELU MLP trained on the GPU with
// BF16 operand storage (weights, inputs, activations) and FP32 accumulation,
// FP32 master weights and Adam; and the POD basis of converged tori.
// (Not part of the paper: the network maps the point parameters to the torus
// coefficients in the POD basis and serves as the continuation initial guess.)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fse_internal.h"

namespace {

constexpr int NL = 3;

struct Mlp {
    int dims[NL + 1];              // n_in, n_hidden, n_hidden, n_out
    int max_batch = 0;
    int device = 0;
    cudaStream_t st = nullptr;
    size_t woff[NL], boff[NL], np = 0;   // offsets in the flat FP32 parameter vector
    float* p = nullptr;            // master parameters (FP32)
    float* g = nullptr;            // gradients
    float* m = nullptr;            // Adam moments
    float* v = nullptr;
    __nv_bfloat16* pw = nullptr;   // BF16 copy of the parameters used by the kernels
    __nv_bfloat16* act[NL + 1] = {};   // layer inputs/activations (BF16), act[0] = X
    float* z[NL] = {};             // pre-activations (FP32)
    float* dz[NL] = {};            // gradients w.r.t. pre-activations (FP32)
    float* T = nullptr;            // targets
    float* out = nullptr;          // FP32 output
    float* loss = nullptr;
    int t = 0;                     // Adam step count
    std::string err;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Z[b][o] = sum_i A[b][i] W[o][i] + bias[o];  next[b][o] = gelu(Z) (bf16) or out[b][o] = Z (last layer)
__global__ void k_linear(int B, int nin, int nout, const __nv_bfloat16* __restrict__ A,
                         const __nv_bfloat16* __restrict__ W, const __nv_bfloat16* __restrict__ bias,
                         float* Z, __nv_bfloat16* next, float* out) {
    __shared__ float sA[32][33];
    __shared__ float sW[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    const int b0 = blockIdx.y * 32, o0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < nin; i0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int b = b0 + r, i = i0 + tx, o = o0 + r;
            sA[r][tx] = (b < B && i < nin) ? __bfloat162float(A[(size_t)b * nin + i]) : 0.f;
            sW[r][tx] = (o < nout && i < nin) ? __bfloat162float(W[(size_t)o * nin + i]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const float w = sW[tx][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += sA[ty + 8 * q][k] * w;
        }
        __syncthreads();
    }
    const int o = o0 + tx;
    if (o >= nout) return;
    const float bo = __bfloat162float(bias[o]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int b = b0 + ty + 8 * q;
        if (b >= B) continue;
        const float zz = acc[q] + bo;
        Z[(size_t)b * nout + o] = zz;
        if (next) next[(size_t)b * nout + o] = __float2bfloat16(gelu_f(zz));
        if (out) out[(size_t)b * nout + o] = zz;
    }
}

// dz = (out - T) / B for the loss 1/(2B) sum (out - T)^2, and the loss itself
__global__ void k_out_grad(int B, int nout, const float* out, const float* T, float* dz, float* loss) {
    __shared__ float red[256];
    float s = 0.f;
    for (int idx = threadIdx.x; idx < B * nout; idx += blockDim.x) {
        const float r = out[idx] - T[idx];
        dz[idx] = r / (float)B;
        s += r * r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = 0.5f * red[0] / (float)B;
}

// dW[o][i] = sum_b dz[b][o] A[b][i];  db[o] = sum_b dz[b][o]
__global__ void k_wgrad(int B, int nin, int nout, const float* __restrict__ dz,
                        const __nv_bfloat16* __restrict__ A, float* dW, float* db) {
    const int o = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nin + 1; i += gridDim.x * blockDim.x) {
        float acc = 0.f;
        if (i < nin) {
            for (int b = 0; b < B; ++b) acc += dz[(size_t)b * nout + o] * __bfloat162float(A[(size_t)b * nin + i]);
            dW[(size_t)o * nin + i] = acc;
        } else {
            for (int b = 0; b < B; ++b) acc += dz[(size_t)b * nout + o];
            db[o] = acc;
        }
    }
}

// dzp[b][i] = (sum_o dz[b][o] W[o][i]) * gelu'(zp[b][i])
__global__ void k_dgrad(int B, int nin, int nout, const float* __restrict__ dz,
                        const __nv_bfloat16* __restrict__ W, const float* __restrict__ zp, float* dzp) {
    const int b = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nin; i += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int o = 0; o < nout; ++o) acc += dz[(size_t)b * nout + o] * __bfloat162float(W[(size_t)o * nin + i]);
        dzp[(size_t)b * nin + i] = acc * gelu_grad_f(zp[(size_t)b * nin + i]);
    }
}

__global__ void k_adam(size_t np, float* p, const float* g, float* m, float* v, __nv_bfloat16* pw, float lr,
                       float c1, float c2) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < np; k += (size_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = 0.9f * m[k] + 0.1f * gk;
        const float vk = 0.999f * v[k] + 0.001f * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
        p[k] = pk;
        pw[k] = __float2bfloat16(pk);
    }
}

__global__ void k_to_bf16(size_t n, const float* src, __nv_bfloat16* dst) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = __float2bfloat16(src[k]);
}

int fail(Mlp* M, int code, const char* msg) {
    if (M) M->err = msg;
    return code;
}

void forward(Mlp* M, int B) {
    for (int l = 0; l < NL; ++l) {
        const int nin = M->dims[l], nout = M->dims[l + 1];
        dim3 g((nout + 31) / 32, (B + 31) / 32);
        const bool last = l == NL - 1;
        k_linear<<<g, 256, 0, M->st>>>(B, nin, nout, M->act[l], M->pw + M->woff[l], M->pw + M->boff[l], M->z[l],
                                       last ? nullptr : M->act[l + 1], last ? M->out : nullptr);
    }
}

void backward(Mlp* M, int B) {
    k_out_grad<<<1, 256, 0, M->st>>>(B, M->dims[NL], M->out, M->T, M->dz[NL - 1], M->loss);
    for (int l = NL - 1; l >= 0; --l) {
        const int nin = M->dims[l], nout = M->dims[l + 1];
        dim3 gw((nin + 1 + 127) / 128, nout);
        k_wgrad<<<gw, 128, 0, M->st>>>(B, nin, nout, M->dz[l], M->act[l], M->g + M->woff[l], M->g + M->boff[l]);
        if (l > 0) {
            dim3 gd((nin + 127) / 128, B);
            k_dgrad<<<gd, 128, 0, M->st>>>(B, nin, nout, M->dz[l], M->pw + M->woff[l], M->z[l - 1], M->dz[l - 1]);
        }
    }
}

int upload_batch(Mlp* M, const float* X, const float* T, int B) {
    if (B < 1 || B > M->max_batch) return fail(M, FSE_EINVAL, "batch size out of range");
    const int nin = M->dims[0];
    std::vector<__nv_bfloat16> xb((size_t)B * nin);
    for (size_t k = 0; k < xb.size(); ++k) xb[k] = __float2bfloat16(X[k]);
    cudaMemcpyAsync(M->act[0], xb.data(), xb.size() * 2, cudaMemcpyHostToDevice, M->st);
    if (T) cudaMemcpyAsync(M->T, T, (size_t)B * M->dims[NL] * 4, cudaMemcpyHostToDevice, M->st);
    return FSE_OK;
}

int sync(Mlp* M, const char* what) {
    cudaError_t e = cudaStreamSynchronize(M->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(M, FSE_ECUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return FSE_OK;
}

}  // namespace

struct fse_mlp : Mlp {};

extern "C" int fse_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, int device, fse_mlp** out) {
    if (!out) return FSE_EINVAL;
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
        return FSE_EINVAL;
    fse_mlp* M = new (std::nothrow) fse_mlp();
    if (!M) return FSE_ENOMEM;
    if (device >= 0) cudaSetDevice(device);
    cudaGetDevice(&M->device);
    M->dims[0] = n_in;
    M->dims[1] = n_hidden;
    M->dims[2] = n_hidden;
    M->dims[3] = n_out;
    M->max_batch = max_batch;
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        M->woff[l] = off;
        off += (size_t)M->dims[l + 1] * M->dims[l];
        M->boff[l] = off;
        off += M->dims[l + 1];
    }
    M->np = off;
    cudaError_t e = cudaStreamCreateWithFlags(&M->st, cudaStreamNonBlocking);
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
    };
    A(&M->p, off * 4);
    A(&M->g, off * 4);
    A(&M->m, off * 4);
    A(&M->v, off * 4);
    A(&M->pw, off * 2);
    for (int l = 0; l <= NL; ++l)
        if (l < NL) A(&M->act[l], (size_t)max_batch * M->dims[l] * 2);
    for (int l = 0; l < NL; ++l) {
        A(&M->z[l], (size_t)max_batch * M->dims[l + 1] * 4);
        A(&M->dz[l], (size_t)max_batch * M->dims[l + 1] * 4);
    }
    A(&M->T, (size_t)max_batch * n_out * 4);
    A(&M->out, (size_t)max_batch * n_out * 4);
    A(&M->loss, 4);
    if (e != cudaSuccess) {
        fse_mlp_destroy(M);
        return FSE_ENOMEM;
    }
    cudaMemsetAsync(M->p, 0, off * 4, M->st);
    cudaMemsetAsync(M->m, 0, off * 4, M->st);
    cudaMemsetAsync(M->v, 0, off * 4, M->st);
    cudaMemsetAsync(M->pw, 0, off * 2, M->st);
    *out = M;
    return sync(M, "mlp create");
}

extern "C" void fse_mlp_destroy(fse_mlp* M) {
    if (!M) return;
    if (M->st) cudaStreamSynchronize(M->st);
    void* ptrs[] = {M->p, M->g, M->m, M->v, M->pw, M->act[0], M->act[1], M->act[2], M->z[0], M->z[1], M->z[2],
                    M->dz[0], M->dz[1], M->dz[2], M->T, M->out, M->loss};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (M->st) cudaStreamDestroy(M->st);
    delete M;
}

extern "C" int fse_mlp_nparams(const fse_mlp* M) { return M ? (int)M->np : 0; }

extern "C" int fse_mlp_nouts(const fse_mlp* M) { return M ? M->dims[NL] : 0; }

extern "C" const char* fse_mlp_last_error(const fse_mlp* M) { return M ? M->err.c_str() : ""; }

extern "C" int fse_mlp_set_params(fse_mlp* M, const float* flat) {
    if (!M || !flat) return FSE_EINVAL;
    cudaSetDevice(M->device);
    cudaMemcpyAsync(M->p, flat, M->np * 4, cudaMemcpyHostToDevice, M->st);
    cudaMemsetAsync(M->m, 0, M->np * 4, M->st);
    cudaMemsetAsync(M->v, 0, M->np * 4, M->st);
    M->t = 0;
    k_to_bf16<<<64, 256, 0, M->st>>>(M->np, M->p, M->pw);
    return sync(M, "mlp set params");
}

extern "C" int fse_mlp_get_params(fse_mlp* M, float* flat) {
    if (!M || !flat) return FSE_EINVAL;
    cudaSetDevice(M->device);
    cudaMemcpyAsync(flat, M->p, M->np * 4, cudaMemcpyDeviceToHost, M->st);
    return sync(M, "mlp get params");
}

extern "C" int fse_mlp_forward(fse_mlp* M, const float* X, int B, float* Y) {
    if (!M || !X || !Y) return FSE_EINVAL;
    cudaSetDevice(M->device);
    int rc = upload_batch(M, X, nullptr, B);
    if (rc) return rc;
    forward(M, B);
    cudaMemcpyAsync(Y, M->out, (size_t)B * M->dims[NL] * 4, cudaMemcpyDeviceToHost, M->st);
    return sync(M, "mlp forward");
}

extern "C" int fse_mlp_grad(fse_mlp* M, const float* X, const float* T, int B, float* loss, float* grad) {
    if (!M || !X || !T) return FSE_EINVAL;
    cudaSetDevice(M->device);
    int rc = upload_batch(M, X, T, B);
    if (rc) return rc;
    forward(M, B);
    backward(M, B);
    if (loss) cudaMemcpyAsync(loss, M->loss, 4, cudaMemcpyDeviceToHost, M->st);
    if (grad) cudaMemcpyAsync(grad, M->g, M->np * 4, cudaMemcpyDeviceToHost, M->st);
    return sync(M, "mlp grad");
}

extern "C" int fse_mlp_train(fse_mlp* M, const float* X, const float* T, int B, int steps, float lr, float* loss) {
    if (!M || !X || !T || steps < 0) return FSE_EINVAL;
    cudaSetDevice(M->device);
    int rc = upload_batch(M, X, T, B);
    if (rc) return rc;
    for (int k = 0; k < steps; ++k) {
        forward(M, B);
        backward(M, B);
        M->t += 1;
        const float c1 = 1.0f - powf(0.9f, (float)M->t), c2 = 1.0f - powf(0.999f, (float)M->t);
        k_adam<<<64, 256, 0, M->st>>>(M->np, M->p, M->g, M->m, M->v, M->pw, lr, c1, c2);
    }
    forward(M, B);
    backward(M, B);
    if (loss) cudaMemcpyAsync(loss, M->loss, 4, cudaMemcpyDeviceToHost, M->st);
    return sync(M, "mlp train");
}

// ----------------------------------------------------------------------------
// POD basis of snapshots (method of snapshots, FP64)
// ----------------------------------------------------------------------------

namespace {

__global__ void k_pod_mean(int m, int nu, const double* S, double* mean) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nu; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < m; ++a) acc += S[(size_t)a * nu + k];
        mean[k] = acc / (double)m;
    }
}

__global__ void k_pod_center(int m, int nu, double* S, const double* mean) {
    const size_t total = (size_t)m * nu;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x)
        S[idx] -= mean[idx % nu];
}

// C[a][b] = sum_k S[a][k] S[b][k], one block per (a, b)
__global__ void k_pod_gram(int m, int nu, const double* S, double* C) {
    const int a = blockIdx.x, b = blockIdx.y;
    if (b > a) return;
    __shared__ double red[256];
    double acc = 0.0;
    for (int k = threadIdx.x; k < nu; k += blockDim.x) acc += S[(size_t)a * nu + k] * S[(size_t)b * nu + k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        C[(size_t)a * m + b] = red[0];
        C[(size_t)b * m + a] = red[0];
    }
}

// cyclic Jacobi eigen-decomposition of the symmetric m x m matrix C (in place -> diag), one CTA;
// at most max_sweeps sweeps; V (m x m, columns = eigenvectors) accumulated
__global__ void k_pod_jacobi(int m, double* C, double* V, int max_sweeps) {
    __shared__ double cs[2];
    __shared__ int done;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) V[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) {
            double off = 0.0, dia = 0.0;
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) {
                    const double x = C[(size_t)i * m + j];
                    if (i == j) dia += x * x; else off += x * x;
                }
            done = off <= 1e-30 * dia;
        }
        __syncthreads();
        if (done) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                if (threadIdx.x == 0) {
                    const double apq = C[(size_t)p * m + q];
                    double c = 1.0, s = 0.0;
                    if (apq != 0.0) {
                        const double app = C[(size_t)p * m + p], aqq = C[(size_t)q * m + q];
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                    cs[0] = c;
                    cs[1] = s;
                }
                __syncthreads();
                const double c = cs[0], s = cs[1];
                if (s != 0.0) {
                    for (int k = threadIdx.x; k < m; k += blockDim.x) {   // rows p, q
                        const double xp = C[(size_t)p * m + k], xq = C[(size_t)q * m + k];
                        C[(size_t)p * m + k] = c * xp - s * xq;
                        C[(size_t)q * m + k] = s * xp + c * xq;
                    }
                    __syncthreads();
                    for (int k = threadIdx.x; k < m; k += blockDim.x) {   // columns p, q and V
                        const double xp = C[(size_t)k * m + p], xq = C[(size_t)k * m + q];
                        C[(size_t)k * m + p] = c * xp - s * xq;
                        C[(size_t)k * m + q] = s * xp + c * xq;
                        const double vp = V[(size_t)k * m + p], vq = V[(size_t)k * m + q];
                        V[(size_t)k * m + p] = c * vp - s * vq;
                        V[(size_t)k * m + q] = s * vp + c * vq;
                    }
                }
                __syncthreads();
            }
    }
}

// basis[k][:] = sum_a V[a][idx_k] S[a][:] / sqrt(lambda_k)
__global__ void k_pod_basis(int m, int nu, int r, const double* S, const double* V, const int* order,
                            const double* lam, double* basis) {
    const int kk = blockIdx.y;
    const int col = order[kk];
    const double sc = lam[col] > 0.0 ? 1.0 / sqrt(lam[col]) : 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nu; x += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < m; ++a) acc += V[(size_t)a * m + col] * S[(size_t)a * nu + x];
        basis[(size_t)kk * nu + x] = acc * sc;
    }
}

}  // namespace

namespace fse {

int pod_build_dev(double* S, int nu, int m, int r, double* mean, double* basis, double* sing_out,
                  cudaStream_t st) {
    if (!S || !mean || !basis || nu < 1 || m < 1 || r < 1 || r > m || m > 1024) return FSE_EINVAL;
    double *C = nullptr, *V = nullptr, *lam = nullptr;
    int* order = nullptr;
    cudaError_t e = cudaMalloc(&C, (size_t)m * m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&V, (size_t)m * m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&lam, (size_t)m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&order, (size_t)m * 4);
    int rc = FSE_OK;
    if (e != cudaSuccess) {
        rc = FSE_ENOMEM;
    } else {
        k_pod_mean<<<fse::num_sms(), 256, 0, st>>>(m, nu, S, mean);
        k_pod_center<<<fse::num_sms() * 4, 256, 0, st>>>(m, nu, S, mean);
        k_pod_gram<<<dim3(m, m), 256, 0, st>>>(m, nu, S, C);
        k_pod_jacobi<<<1, 256, 0, st>>>(m, C, V, 30);
        // eigenvalues (the diagonal) ordered by size on the host: index bookkeeping only
        std::vector<double> Ch((size_t)m * m);
        cudaMemcpyAsync(Ch.data(), C, Ch.size() * 8, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        std::vector<double> lh(m);
        std::vector<int> ord(m);
        for (int a = 0; a < m; ++a) {
            lh[a] = Ch[(size_t)a * m + a];
            ord[a] = a;
        }
        for (int a = 0; a < m; ++a)
            for (int b2 = a + 1; b2 < m; ++b2)
                if (lh[ord[b2]] > lh[ord[a]]) std::swap(ord[a], ord[b2]);
        cudaMemcpyAsync(lam, lh.data(), (size_t)m * 8, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(order, ord.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st);
        k_pod_basis<<<dim3(64, r), 256, 0, st>>>(m, nu, r, S, V, order, lam, basis);
        if (sing_out)
            for (int k = 0; k < r; ++k) sing_out[k] = lh[ord[k]] > 0 ? std::sqrt(lh[ord[k]]) : 0.0;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = FSE_ECUDA;
    }
    for (void* q : {(void*)C, (void*)V, (void*)lam, (void*)order})
        if (q) cudaFree(q);
    return rc;
}

}  // namespace fse

extern "C" int fse_pod_build(const double* snaps, int nu, int m, int r, double* mean_out, double* basis_out,
                             double* sing_out) {
    if (!snaps || !mean_out || !basis_out || nu < 1 || m < 1 || r < 1 || r > m || m > 1024) return FSE_EINVAL;
    double *S = nullptr, *mean = nullptr, *basis = nullptr;
    cudaError_t e = cudaMalloc(&S, (size_t)m * nu * 8);
    if (e == cudaSuccess) e = cudaMalloc(&mean, (size_t)nu * 8);
    if (e == cudaSuccess) e = cudaMalloc(&basis, (size_t)r * nu * 8);
    int rc = e == cudaSuccess ? FSE_OK : FSE_ENOMEM;
    if (rc == FSE_OK) {
        cudaMemcpy(S, snaps, (size_t)m * nu * 8, cudaMemcpyHostToDevice);
        rc = fse::pod_build_dev(S, nu, m, r, mean, basis, sing_out, 0);
        if (rc == FSE_OK) {
            cudaMemcpy(mean_out, mean, (size_t)nu * 8, cudaMemcpyDeviceToHost);
            cudaMemcpy(basis_out, basis, (size_t)r * nu * 8, cudaMemcpyDeviceToHost);
        }
    }
    for (void* q : {(void*)S, (void*)mean, (void*)basis})
        if (q) cudaFree(q);
    return rc;
}
