// Sensitivity (monodromy) propagation of FSE-Shooting: the tangents X = dq/dp,
// V = du/dp of the 2n+1 directions p = (z_0, w_1) of every trajectory through
// the Newmark step of App. E.
//
// Differentiating Eq. (E6)-(E7) and eliminating the acceleration tangent with
// the linearised equation of motion of the previous step
//     w^2 M W_k + w D V_k + (K + K_t(q_k)) X_k = [-2 w M a_k - D u_k  in the w_1 column]
// gives, for every direction (exactly the same recurrence as the one with W):
//     K_eff(q_{k+1}) X_{k+1} = (w^2 4/D^2 M + w 2/D D - K - K_t(q_k)) X_k + w^2 4/D M V_k
//                              [ - 2 w M (a_k + a_{k+1}) - D (u_k + u_{k+1})  for w_1 ]
//     V_{k+1} = 2/D (X_{k+1} - X_k) - V_k
// with X_0 = [I 0 0], V_0 = [0 I 0].  Three kernels per step: the right-hand
// side (sparse products, one pass over X, V), the forward and the backward
// blocked banded substitution (the latter also applies the V update).
// Tangent rows have stride ld (a multiple of 4); columns P..ld-1 stay zero.
#include <cuda_runtime.h>

#include "fse_common.cuh"

namespace fse {

struct SensArgs {
    int n, b, P, ld, nnz_kt, nblk, RW, RWT;
    double a2c;
    const int *cs_ptr, *cs_slot, *kt_ptr, *kt_slot;
    const void *Aop, *Bop, *kt_val, *romega;
    const void *Lc, *Lr, *Dinv;
    void *X, *V, *Y;
};

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// 4 consecutive elements, 16-byte (float) / 2 x 16-byte (double) aligned
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T v[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    } else {
        const double2 x = *reinterpret_cast<const double2*>(p);
        const double2 y = *reinterpret_cast<const double2*>(p + 2);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = y.x;
        v[3] = y.y;
    }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T v[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
    }
}

// RHS[s][i][t] = sum_j A_ij X[j][t] + B_ij V[j][t] - sum_j K_t(q_k)_ij X[j][t] (+ romega_i at t = 2n).
// One CTA = all rows of one trajectory for 64 directions; a ring of the X, V rows
// [i - b, i + b] in shared memory is filled once per row, so every tangent row is read
// from memory once per step.  8 warps process 8 consecutive rows; each lane owns 2 directions.
template <typename T>
__global__ void __launch_bounds__(256) k_sens_rhs(SensArgs A) {
    using T2 = typename Vec2<T>::type;
    const int n = A.n, b = A.b, P = A.P, ld = A.ld, RW = A.RW;
    const int s = blockIdx.y, t0 = blockIdx.x * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* rX = reinterpret_cast<T*>(smraw);        // RW x 64
    T* rV = rX + (size_t)RW * 64;
    const size_t base = (size_t)s * n * ld;
    const T* X = reinterpret_cast<const T*>(A.X) + base;
    const T* V = reinterpret_cast<const T*>(A.V) + base;
    T* Y = reinterpret_cast<T*>(A.Y) + base;
    const T* Aop = reinterpret_cast<const T*>(A.Aop);
    const T* Bop = reinterpret_cast<const T*>(A.Bop);
    const T* ktv = reinterpret_cast<const T*>(A.kt_val) + (size_t)s * A.nnz_kt;
    const T* rom = reinterpret_cast<const T*>(A.romega) + (size_t)s * n;
    int loaded = 0;   // rows [0, loaded) have been put in the ring
    for (int g0 = 0; g0 < n; g0 += 8) {
        const int need = min(n, g0 + 8 + b);
        // load rows [loaded, need) into the ring (their slots were last used by rows < g0 - b)
        const int cnt = need - loaded;
        for (int idx = threadIdx.x; idx < cnt * 16; idx += blockDim.x) {
            const int r = loaded + (idx >> 4), c = (idx & 15) * 4, t = t0 + c;
            const int slot = r % RW;
            T xv[4] = {T(0), T(0), T(0), T(0)}, vv[4] = {T(0), T(0), T(0), T(0)};
            if (t < ld) {
                ld4(X + (size_t)r * ld + t, xv);
                ld4(V + (size_t)r * ld + t, vv);
            }
            st4(rX + slot * 64 + c, xv);
            st4(rV + slot * 64 + c, vv);
        }
        loaded = need;
        __syncthreads();
        const int i = g0 + warp;
        if (i < n) {
            T acc0 = T(0), acc1 = T(0);
            const int e1 = A.cs_ptr[i + 1];
            for (int e = A.cs_ptr[i]; e < e1; ++e) {
                const int sl = A.cs_slot[e];
                const T av = Aop[e], bv = Bop[e];
                const T2 x = *reinterpret_cast<const T2*>(rX + sl * 64 + 2 * lane);
                const T2 v = *reinterpret_cast<const T2*>(rV + sl * 64 + 2 * lane);
                acc0 += av * x.x + bv * v.x;
                acc1 += av * x.y + bv * v.y;
            }
            const int k1 = A.kt_ptr[i + 1];
            for (int e = A.kt_ptr[i]; e < k1; ++e) {
                const int sl = A.kt_slot[e];
                const T kv = ktv[e];
                const T2 x = *reinterpret_cast<const T2*>(rX + sl * 64 + 2 * lane);
                acc0 -= kv * x.x;
                acc1 -= kv * x.y;
            }
            const int t = t0 + 2 * lane;
            if (t == P - 1) acc0 += rom[i];
            if (t + 1 == P - 1) acc1 += rom[i];
            if (t < ld) *reinterpret_cast<T2*>(Y + (size_t)i * ld + t) = T2{acc0, acc1};
        }
        __syncthreads();
    }
}

// Blocked forward substitution L y = rhs (in place on Y) for 128 directions of one
// trajectory: per 32-row block, y_B = Dinv_B (rhs_B - L_{B,<} y_<), both products as
// register-tiled 4 x 4 micro-kernels over a shared-memory ring of the last rows
// (RWT >= b + 32 rows, a power of two).
template <typename T>
__global__ void __launch_bounds__(256) k_trsm_fwd(SensArgs A) {
    const int n = A.n, b = A.b, ld = A.ld, nb = b + 1, RM = A.RWT - 1;
    const int s = blockIdx.y, t0 = blockIdx.x * 128;
    const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;   // rows 4tr.., cols 4tc..
    const int t = t0 + 4 * tc;
    const bool tok = t < ld;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ring = reinterpret_cast<T*>(smraw);                    // RWT x 128
    T* LbT = ring + (size_t)A.RWT * 128;                      // b x 32   (transposed)
    T* DvT = LbT + (size_t)((b + 3) & ~3) * 32;               // 32 x 32  (transposed)
    const T* Lr = reinterpret_cast<const T*>(A.Lr) + (size_t)s * n * nb;
    const T* Dv = reinterpret_cast<const T*>(A.Dinv) + (size_t)s * A.nblk * FSE_BLK * FSE_BLK;
    T* Y = reinterpret_cast<T*>(A.Y) + (size_t)s * n * ld;
    for (int B = 0; B < A.nblk; ++B) {
        const int i0 = B * FSE_BLK;
        for (int idx = threadIdx.x; idx < b * 32; idx += blockDim.x) {
            const int c = idx >> 5, r = idx & 31;
            const int i = i0 + r, j = i0 - b + c, bi = c - r;   // row-band index of L(i, j)
            LbT[idx] = (i < n && j >= 0 && bi >= 0) ? Lr[(size_t)i * nb + bi] : T(0);
        }
        for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x)
            DvT[idx] = Dv[(size_t)B * 1024 + (idx & 31) * 32 + (idx >> 5)];
        T acc[4][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + 4 * tr + rr;
            if (i < n && tok) {
                ld4(Y + (size_t)i * ld + t, acc[rr]);
            } else {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = T(0);
            }
        }
        __syncthreads();
        const int cstart = max(0, b - i0);
        for (int c = cstart; c < b; ++c) {
            const int j = i0 - b + c;
            T yv[4], lv[4];
            ld4(ring + (size_t)(j & RM) * 128 + 4 * tc, yv);
            ld4(LbT + c * 32 + 4 * tr, lv);
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc[rr][cc] -= lv[rr] * yv[cc];
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) st4(ring + (size_t)((i0 + 4 * tr + rr) & RM) * 128 + 4 * tc, acc[rr]);
        __syncthreads();
        T out[4][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) out[rr][cc] = T(0);
#pragma unroll 4
        for (int k = 0; k < FSE_BLK; ++k) {
            T tv[4], dv[4];
            ld4(ring + (size_t)((i0 + k) & RM) * 128 + 4 * tc, tv);
            ld4(DvT + k * 32 + 4 * tr, dv);
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) out[rr][cc] += dv[rr] * tv[cc];
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + 4 * tr + rr;
            st4(ring + (size_t)(i & RM) * 128 + 4 * tc, out[rr]);
            if (i < n && tok) st4(Y + (size_t)i * ld + t, out[rr]);
        }
        __syncthreads();
    }
}

// Blocked backward substitution L^T x = y, then the tangent update
// X <- x, V <- 2/D (x - X_old) - V_old (Eq. E5 differentiated).
template <typename T>
__global__ void __launch_bounds__(256) k_trsm_bwd(SensArgs A) {
    const int n = A.n, b = A.b, ld = A.ld, nb = b + 1, RM = A.RWT - 1;
    const int s = blockIdx.y, t0 = blockIdx.x * 128;
    const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;
    const int t = t0 + 4 * tc;
    const bool tok = t < ld;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ring = reinterpret_cast<T*>(smraw);
    T* Lb = ring + (size_t)A.RWT * 128;                       // b x 32:  Lb[c][r] = L(i0+32+c, i0+r)
    T* Dk = Lb + (size_t)((b + 3) & ~3) * 32;                 // 32 x 32: Dinv as stored
    const T* Lc = reinterpret_cast<const T*>(A.Lc) + (size_t)s * n * nb;
    const T* Dv = reinterpret_cast<const T*>(A.Dinv) + (size_t)s * A.nblk * FSE_BLK * FSE_BLK;
    const size_t base = (size_t)s * n * ld;
    const T* Y = reinterpret_cast<const T*>(A.Y) + base;
    T* X = reinterpret_cast<T*>(A.X) + base;
    T* V = reinterpret_cast<T*>(A.V) + base;
    const T a2 = T(A.a2c);
    for (int B = A.nblk - 1; B >= 0; --B) {
        const int i0 = B * FSE_BLK;
        for (int idx = threadIdx.x; idx < b * 32; idx += blockDim.x) {
            const int c = idx >> 5, r = idx & 31;
            const int i = i0 + r, k = i0 + FSE_BLK + c, ci = k - i;   // column-band index of L(k, i)
            Lb[idx] = (i < n && k < n && ci <= b) ? Lc[(size_t)i * nb + ci] : T(0);
        }
        for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) Dk[idx] = Dv[(size_t)B * 1024 + idx];
        T acc[4][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + 4 * tr + rr;
            if (i < n && tok) {
                ld4(Y + (size_t)i * ld + t, acc[rr]);
            } else {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = T(0);
            }
        }
        __syncthreads();
        const int cend = min(b, n - (i0 + FSE_BLK));
        for (int c = 0; c < cend; ++c) {
            const int k = i0 + FSE_BLK + c;
            T xv[4], lv[4];
            ld4(ring + (size_t)(k & RM) * 128 + 4 * tc, xv);
            ld4(Lb + c * 32 + 4 * tr, lv);
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc[rr][cc] -= lv[rr] * xv[cc];
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) st4(ring + (size_t)((i0 + 4 * tr + rr) & RM) * 128 + 4 * tc, acc[rr]);
        __syncthreads();
        T out[4][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) out[rr][cc] = T(0);
#pragma unroll 4
        for (int k = 0; k < FSE_BLK; ++k) {
            T tv[4], dv[4];
            ld4(ring + (size_t)((i0 + k) & RM) * 128 + 4 * tc, tv);
            ld4(Dk + k * 32 + 4 * tr, dv);                      // Dinv[k][4tr + rr]
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) out[rr][cc] += dv[rr] * tv[cc];
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + 4 * tr + rr;
            st4(ring + (size_t)(i & RM) * 128 + 4 * tc, out[rr]);
            if (i < n && tok) {
                const size_t o = (size_t)i * ld + t;
                T xo[4], vo[4], vn[4];
                ld4(X + o, xo);
                ld4(V + o, vo);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) vn[cc] = a2 * (out[rr][cc] - xo[cc]) - vo[cc];
                st4(X + o, out[rr]);
                st4(V + o, vn);
            }
        }
        __syncthreads();
    }
}

// X_0 = [I 0 0], V_0 = [0 I 0], zero padding columns
template <typename T>
__global__ void k_sens_init(int N, int n, int ld, T* X, T* V) {
    const size_t total = (size_t)N * n * ld;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t r = idx / ld;
        const int t = (int)(idx % ld), i = (int)(r % n);
        X[idx] = (t == i) ? T(1) : T(0);
        V[idx] = (t == i + n) ? T(1) : T(0);
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------

size_t rhs_smem(const Params& p) {
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    return (size_t)2 * p.RW * 64 * tsz;
}

size_t trsm_smem(const Params& p) {
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    return ((size_t)p.RWT * 128 + (size_t)((p.b + 3) & ~3) * 32 + 1024) * tsz;
}

template <typename T>
static void sens_launch(fse_ctx* c, const SensArgs& A, int phase, cudaStream_t st) {
    const Params& p = c->p;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sens_rhs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    if (phase == 0) {
        dim3 g((p.P + 63) / 64, p.N);
        k_sens_rhs<T><<<g, 256, p.smem_rhs, st>>>(A);
    } else {
        dim3 g((p.P + 127) / 128, p.N);
        if (phase == 1)
            k_trsm_fwd<T><<<g, 256, p.smem_trsm, st>>>(A);
        else
            k_trsm_bwd<T><<<g, 256, p.smem_trsm, st>>>(A);
    }
}

void launch_sens_init(fse_ctx* c, cudaStream_t st) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * p.n * p.ld;
    if (p.prec == FSE_MIXED_FP32)
        k_sens_init<float><<<nblocks(tot, 256, 152 * 64), 256, 0, st>>>(p.N, p.n, p.ld, (float*)c->d.X,
                                                                       (float*)c->d.V);
    else
        k_sens_init<double><<<nblocks(tot, 256, 152 * 64), 256, 0, st>>>(p.N, p.n, p.ld, (double*)c->d.X,
                                                                        (double*)c->d.V);
}

void launch_sens_phase(fse_ctx* c, int k, double w, int phase, cudaStream_t st) {
    const Params& p = c->p;
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    const double Dl = 2.0 * M_PI / p.S1;
    SensArgs A;
    A.n = p.n;
    A.b = p.b;
    A.P = p.P;
    A.ld = p.ld;
    A.nnz_kt = p.nnz_kt;
    A.nblk = p.nblk;
    A.RW = p.RW;
    A.RWT = p.RWT;
    A.a2c = 2.0 / Dl;
    A.cs_ptr = c->d.cs_ptr;
    A.cs_slot = c->d.cs_slot;
    A.kt_ptr = c->d.kt_ptr;
    A.kt_slot = c->d.kt_slot;
    A.Aop = c->d.cs_A;
    A.Bop = c->d.cs_B;
    const size_t ktsz = (size_t)p.N * p.nnz_kt * tsz;
    const size_t fsz = (size_t)p.N * p.n * (p.b + 1) * tsz;
    const size_t vsz = (size_t)p.N * p.n * tsz;
    const size_t dsz = (size_t)p.N * p.nblk * FSE_BLK * FSE_BLK * tsz;
    const int f = k % 2;
    A.kt_val = (const char*)c->d.kt_val + (k % FSE_NBUF_KT) * ktsz;   // K_t(q_k)
    A.romega = (const char*)c->d.romega + f * vsz;
    A.Lc = (const char*)c->d.Lc + f * fsz;                             // factor of K_eff(q_{k+1})
    A.Lr = (const char*)c->d.Lr + f * fsz;
    A.Dinv = (const char*)c->d.Dinv + f * dsz;
    A.X = c->d.X;
    A.V = c->d.V;
    A.Y = c->d.Y;
    (void)w;
    if (p.prec == FSE_MIXED_FP32)
        sens_launch<float>(c, A, phase, st);
    else
        sens_launch<double>(c, A, phase, st);
}

}  // namespace fse
