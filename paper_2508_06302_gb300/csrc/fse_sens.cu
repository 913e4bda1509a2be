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

// asynchronous 16-byte global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// RHS[s][i][t] = sum_j A_ij X[j][t] + B_ij V[j][t] - sum_j K_t(q_k)_ij X[j][t] (+ romega_i at t = 2n).
// One CTA = all rows of one trajectory for 64 directions.  A ring of RW = 2b + 2G rows of
// X and V in shared memory holds the rows [i - b, i + b] of the G rows being processed plus
// the G rows prefetched (cp.async) for the next step, so every tangent row is read from
// memory once per Newmark step and the loads overlap the arithmetic.
template <typename T>
__global__ void __launch_bounds__(256) k_sens_rhs(SensArgs A) {
    using T2 = typename Vec2<T>::type;
    constexpr int G = FSE_RHS_G;
    constexpr int EPC = 16 / sizeof(T);            // elements per 16-byte copy
    constexpr int CPR = 64 / EPC;                  // copies per row and array
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
    // issue the copies of rows [r0, r1) into their ring slots
    auto fill = [&](int r0, int r1) {
        const int cnt = (r1 - r0) * CPR;
        for (int idx = threadIdx.x; idx < 2 * cnt; idx += blockDim.x) {
            const int arr = idx >= cnt;
            const int q = arr ? idx - cnt : idx;
            const int r = r0 + q / CPR, c = (q % CPR) * EPC, t = t0 + c;
            const T* src = (arr ? V : X) + (size_t)r * ld + (t < ld ? t : 0);
            T* dst = (arr ? rV : rX) + (size_t)(r % RW) * 64 + c;
            cp_async16(dst, src, t < ld ? 16 : 0);
        }
    };
    int loaded = min(n, G + b);
    fill(0, loaded);
    cp_async_commit();
    for (int g0 = 0; g0 < n; g0 += G) {
        const int need = min(n, g0 + 2 * G + b);      // rows of the next step
        if (need > loaded) fill(loaded, need);
        loaded = max(loaded, need);
        cp_async_commit();
        cp_async_wait1();                                 // this step's rows have landed
        __syncthreads();
#pragma unroll
        for (int h = 0; h < G / 8; ++h) {
            const int i = g0 + warp + 8 * h;
            if (i < n) {
                T acc0 = T(0), acc1 = T(0);
                // the row's entries are fetched by the lanes in one round trip, then broadcast
                const int e0 = A.cs_ptr[i], e1 = A.cs_ptr[i + 1];
                for (int eb = e0; eb < e1; eb += 32) {
                    const int e = eb + lane, cnt = min(32, e1 - eb);
                    int sl_l = 0;
                    T a_l = T(0), b_l = T(0);
                    if (e < e1) {
                        sl_l = A.cs_slot[e];
                        a_l = Aop[e];
                        b_l = Bop[e];
                    }
                    for (int q = 0; q < cnt; ++q) {
                        const int sl = __shfl_sync(0xffffffffu, sl_l, q);
                        const T av = __shfl_sync(0xffffffffu, a_l, q);
                        const T bv = __shfl_sync(0xffffffffu, b_l, q);
                        const T2 x = *reinterpret_cast<const T2*>(rX + sl * 64 + 2 * lane);
                        const T2 v = *reinterpret_cast<const T2*>(rV + sl * 64 + 2 * lane);
                        acc0 += av * x.x + bv * v.x;
                        acc1 += av * x.y + bv * v.y;
                    }
                }
                const int k0 = A.kt_ptr[i], k1 = A.kt_ptr[i + 1];
                for (int eb = k0; eb < k1; eb += 32) {
                    const int e = eb + lane, cnt = min(32, k1 - eb);
                    int sl_l = 0;
                    T k_l = T(0);
                    if (e < k1) {
                        sl_l = A.kt_slot[e];
                        k_l = ktv[e];
                    }
                    for (int q = 0; q < cnt; ++q) {
                        const int sl = __shfl_sync(0xffffffffu, sl_l, q);
                        const T kv = __shfl_sync(0xffffffffu, k_l, q);
                        const T2 x = *reinterpret_cast<const T2*>(rX + sl * 64 + 2 * lane);
                        acc0 -= kv * x.x;
                        acc1 -= kv * x.y;
                    }
                }
                const int t = t0 + 2 * lane;
                if (t == P - 1) acc0 += rom[i];
                if (t + 1 == P - 1) acc1 += rom[i];
                if (t < ld) *reinterpret_cast<T2*>(Y + (size_t)i * ld + t) = T2{acc0, acc1};
            }
        }
        __syncthreads();
    }
    cp_async_wait0();
}

// The per-block factor tiles of the blocked solves: Lt[c][r] (b x 32) and the 32 x 32
// diagonal-block inverse, gathered into registers one block ahead and stored to the
// shared buffer of the block after the current one.
template <typename T, bool FWD, int MAXL>
struct TileLoader {   // MAXL >= b * 32 / 256
    T l[MAXL];
    T d[4];
    __device__ __forceinline__ void load(const T* Lband, const T* Dv, int B, int n, int b, int nb) {
        const int i0 = B * FSE_BLK;
#pragma unroll
        for (int q = 0; q < MAXL; ++q) {
            const int idx = threadIdx.x + q * 256;
            T v = T(0);
            if (idx < b * 32) {
                const int c = idx >> 5, r = idx & 31, i = i0 + r;
                if (FWD) {
                    const int j = i0 - b + c, bi = c - r;            // row band of L(i, j)
                    if (i < n && j >= 0 && bi >= 0) v = Lband[(size_t)i * nb + bi];
                } else {
                    const int k = i0 + FSE_BLK + c, ci = k - i;      // column band of L(k, i)
                    if (i < n && k < n && ci <= b) v = Lband[(size_t)i * nb + ci];
                }
            }
            l[q] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = threadIdx.x + q * 256;
            // forward wants Dinv transposed (DvT[k][r] = Dinv[r][k]), backward as stored
            d[q] = FWD ? Dv[(size_t)B * 1024 + (idx & 31) * 32 + (idx >> 5)] : Dv[(size_t)B * 1024 + idx];
        }
    }
    __device__ __forceinline__ void store(T* Lt, T* Dt, int b) const {
#pragma unroll
        for (int q = 0; q < MAXL; ++q) {
            const int idx = threadIdx.x + q * 256;
            if (idx < b * 32) Lt[idx] = l[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Dt[threadIdx.x + q * 256] = d[q];
    }
};

// Blocked banded substitution for 128 directions of one trajectory.
//  FWD: L y = rhs in place on Y,   y_B = Dinv_B (rhs_B - L_{B,<} y_<)
//  BWD: L^T x = y, x_B = Dinv_B^T (y_B - L_{>,B}^T x_>), then X <- x, V <- 2/D (x - X) - V.
// Both products are register-tiled 4 x 4 micro-kernels over a shared-memory ring of the
// last RWT rows (power of two >= b + 32); the next block's operands (factor tiles, Y and,
// backward, X and V) are fetched into registers while the current block computes.
template <typename T, bool FWD, int MAXL>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_trsm(SensArgs A) {
    const int n = A.n, b = A.b, ld = A.ld, nb = b + 1, RM = A.RWT - 1;
    const int s = blockIdx.y, t0 = blockIdx.x * 128;
    const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;   // rows 4tr.., cols 4tc..
    const int t = t0 + 4 * tc;
    const bool tok = t < ld;
    const int bpad = (b + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ring = reinterpret_cast<T*>(smraw);                    // RWT x 128
    T* Lt[2];
    T* Dt[2];
    Lt[0] = ring + (size_t)A.RWT * 128;
    Dt[0] = Lt[0] + (size_t)bpad * 32;
    Lt[1] = Dt[0] + 1024;
    Dt[1] = Lt[1] + (size_t)bpad * 32;
    const T* Lband = reinterpret_cast<const T*>(FWD ? A.Lr : A.Lc) + (size_t)s * n * nb;
    const T* Dv = reinterpret_cast<const T*>(A.Dinv) + (size_t)s * A.nblk * FSE_BLK * FSE_BLK;
    const size_t base = (size_t)s * n * ld;
    T* Y = reinterpret_cast<T*>(A.Y) + base;
    T* X = reinterpret_cast<T*>(A.X) + base;
    T* V = reinterpret_cast<T*>(A.V) + base;
    const T a2 = T(A.a2c);
    const int nblk = A.nblk;
    auto blk = [&](int q) { return FWD ? q : nblk - 1 - q; };
    auto load_rows = [&](const T* src, int B, T out[4][4]) {
        const int i0 = B * FSE_BLK;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + 4 * tr + rr;
            if (i < n && tok) {
                ld4(src + (size_t)i * ld + t, out[rr]);
            } else {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) out[rr][cc] = T(0);
            }
        }
    };
    TileLoader<T, FWD, MAXL> tl;
    tl.load(Lband, Dv, blk(0), n, b, nb);
    tl.store(Lt[0], Dt[0], b);
    T ynext[4][4];
    load_rows(Y, blk(0), ynext);
    for (int q = 0; q < nblk; ++q) {
        const int B = blk(q), i0 = B * FSE_BLK, buf = q & 1;
        T acc[4][4], xo[4][4], vo[4][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = ynext[rr][cc];
        if (!FWD) {
            load_rows(X, B, xo);
            load_rows(V, B, vo);
        }
        if (q + 1 < nblk) {
            load_rows(Y, blk(q + 1), ynext);
            tl.load(Lband, Dv, blk(q + 1), n, b, nb);
        }
        __syncthreads();                                  // tiles of block q are in Lt/Dt[buf]
        const T* L = Lt[buf];
        if (FWD) {
            for (int c = max(0, b - i0); c < b; ++c) {
                T yv[4], lv[4];
                ld4(ring + (size_t)((i0 - b + c) & RM) * 128 + 4 * tc, yv);
                ld4(L + c * 32 + 4 * tr, lv);
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[rr][cc] -= lv[rr] * yv[cc];
            }
        } else {
            const int cend = min(b, n - (i0 + FSE_BLK));
            for (int c = 0; c < cend; ++c) {
                T xv[4], lv[4];
                ld4(ring + (size_t)((i0 + FSE_BLK + c) & RM) * 128 + 4 * tc, xv);
                ld4(L + c * 32 + 4 * tr, lv);
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[rr][cc] -= lv[rr] * xv[cc];
            }
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) st4(ring + (size_t)((i0 + 4 * tr + rr) & RM) * 128 + 4 * tc, acc[rr]);
        __syncthreads();
        T out[4][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) out[rr][cc] = T(0);
        const T* D = Dt[buf];
#pragma unroll 4
        for (int k = 0; k < FSE_BLK; ++k) {
            T tv[4], dv[4];
            ld4(ring + (size_t)((i0 + k) & RM) * 128 + 4 * tc, tv);
            ld4(D + k * 32 + 4 * tr, dv);
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) out[rr][cc] += dv[rr] * tv[cc];
        }
        if (q + 1 < nblk) tl.store(Lt[buf ^ 1], Dt[buf ^ 1], b);
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + 4 * tr + rr;
            st4(ring + (size_t)(i & RM) * 128 + 4 * tc, out[rr]);
            if (i < n && tok) {
                const size_t o = (size_t)i * ld + t;
                if (FWD) {
                    st4(Y + o, out[rr]);
                } else {
                    T vn[4];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) vn[cc] = a2 * (out[rr][cc] - xo[rr][cc]) - vo[rr][cc];
                    st4(X + o, out[rr]);
                    st4(V + o, vn);
                }
            }
        }
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
    return ((size_t)p.RWT * 128 + 2 * ((size_t)((p.b + 3) & ~3) * 32 + 1024)) * tsz;
}

template <typename T>
static void sens_launch(fse_ctx* c, const SensArgs& A, int phase, cudaStream_t st) {
    const Params& p = c->p;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sens_rhs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm<T, true, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm<T, false, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm<T, true, 28>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm<T, false, 28>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    if (phase == 0) {
        dim3 g((p.P + 63) / 64, p.N);
        k_sens_rhs<T><<<g, 256, p.smem_rhs, st>>>(A);
    } else {
        dim3 g((p.P + 127) / 128, p.N);
        const bool small = p.b <= 96;   // factor tile of b x 32 spread over 256 threads
        if (phase == 1) {
            if (small)
                k_trsm<T, true, 12><<<g, 256, p.smem_trsm, st>>>(A);
            else
                k_trsm<T, true, 28><<<g, 256, p.smem_trsm, st>>>(A);
        } else {
            if (small)
                k_trsm<T, false, 12><<<g, 256, p.smem_trsm, st>>>(A);
            else
                k_trsm<T, false, 28><<<g, 256, p.smem_trsm, st>>>(A);
        }
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
