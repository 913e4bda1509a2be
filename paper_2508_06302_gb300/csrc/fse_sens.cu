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
    int n, b, P, ld, kt_ld, nblk, RW, RWT;
    int ng, ME, RB, MK, RECE;
    double a2c;
    const int* kt_slot;
    int* err;   // set when a pipeline wait gives up
    const void *g_rec, *g_rr, *g_info, *g_pass, *kt_val, *romega;
    const void *Lc, *Lr, *Dinv, *Rf, *Rb;
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


// explicit shared-memory loads on 32-bit shared addresses
__device__ __forceinline__ uint4 lds_u4(unsigned a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ int2 lds_i2(unsigned a) {
    int2 v;
    asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ int lds_i(unsigned a) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];\n" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_f2(unsigned a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_f(unsigned a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds_d(unsigned a) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];\n" : "=d"(v) : "r"(a));
    return v;
}
template <typename T>
__device__ __forceinline__ T lds_t(unsigned a) {
    if constexpr (sizeof(T) == 4)
        return lds_f(a);
    else
        return lds_d(a);
}

// bytes of one group record: the ring slot (int, padded to 8 bytes), then R values of A and
// R values of B
template <typename T, int R>
__host__ __device__ constexpr int rhs_record_bytes() {
    return (int)((8 + 2 * R * sizeof(T) + 15) / 16 * 16);
}

// RHS[s][i][t] = sum_j A_ij X[j][t] + B_ij V[j][t] - sum_j K_t(q_k)_ij X[j][t] (+ romega_i at t = 2n).
// One CTA = all rows of one trajectory for CW directions (64 in FP32, 32 in FP64).  Rows go
// in groups of up to R rows with one common column pattern, one group per consumer warp and
// FSE_RHS_GPS groups per pass: each X/V element read from shared memory feeds R rows.  A ring
// of RW rows of X and V in shared memory holds the rows of the passes in flight; a
// producer warp streams, for the passes ahead, the tangent rows, the group records (slot, A
// and B values), the group and row records and the pass's slice of K_t(q_k) (slots and
// values) with bulk copies that complete on a "full" mbarrier per buffer, and refills a
// buffer once all consumer warps have arrived on its "empty" mbarrier.  Every tangent row is
// read from memory once per step; the consumers read nothing else from global memory.
template <typename T, int R>
__global__ void __launch_bounds__(32 * (FSE_RHS_GPS + 1), 1)
    k_sens_rhs(SensArgs A, const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV) {
    constexpr int CW = sizeof(T) == 4 ? 64 : 32;   // columns per CTA
    constexpr int EL = CW / 32;                     // columns per lane
    constexpr int GPS = FSE_RHS_GPS;
    constexpr int NB = (sizeof(T) == 4 ? FSE_RHS_DEPTH_F32 : FSE_RHS_DEPTH_F64) + 1;   // buffers in flight
    constexpr int RB = rhs_record_bytes<T, R>();
    constexpr int RW4 = RB / 4;                     // 32-bit words per record
    const int n = A.n, P = A.P, ld = A.ld, RW = A.RW, ng = A.ng, ME = A.ME, MK = A.MK;
    const int s = blockIdx.y, t0 = blockIdx.x * CW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ __align__(8) unsigned long long bar_full[NB], bar_empty[NB];
    extern __shared__ __align__(16) unsigned char smraw[];
    // per buffer: group records ME x RB | row records GPS x R int4 | group entry ranges GPS int2 |
    // K_t slots MK int | K_t values MK T
    const size_t bufsz = (size_t)ME * RB + (size_t)GPS * R * 16 + (size_t)GPS * 8 + (size_t)MK * (4 + sizeof(T));
    unsigned char* sm128 = smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u);   // TMA boxes: 128-byte aligned
    T* rX = reinterpret_cast<T*>(sm128);            // RW x CW (RW a multiple of 32)
    T* rV = rX + (size_t)RW * CW;
    unsigned char* bufs = reinterpret_cast<unsigned char*>(rV + (size_t)RW * CW);
    const size_t base = (size_t)s * n * ld;
    T* Y = reinterpret_cast<T*>(A.Y) + base;
    const int npass = (ng + GPS - 1) / GPS;
    if (threadIdx.x == 0) {
        for (int k = 0; k < NB; ++k) {
            mbar_init(&bar_full[k], 1);
            mbar_init(&bar_empty[k], GPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == GPS) {
        // ---- producer
        const unsigned char* rec = reinterpret_cast<const unsigned char*>(A.g_rec);
        const int4* rr_g = reinterpret_cast<const int4*>(A.g_rr);
        const int2* gi_g = reinterpret_cast<const int2*>(A.g_info);
        const int4* pd = reinterpret_cast<const int4*>(A.g_pass);
        const T* ktv = reinterpret_cast<const T*>(A.kt_val) + (size_t)s * A.kt_ld;
        constexpr unsigned chunkbytes = 32u * CW * (unsigned)sizeof(T);   // one TMA box: 32 rows
        int loadedc = 0, q = 0;                                            // 32-row chunks staged
        int4 d0 = pd[0], d1 = pd[1];
        for (; q < npass; ++q) {
            const int slot = q % NB;
            int4 n0 = d0, n1 = d1;
            if (q + 1 < npass) {
                n0 = pd[2 * q + 2];
                n1 = pd[2 * q + 3];
            }
            if (q >= NB && !mbar_wait(&bar_empty[slot], ((q / NB) - 1) & 1, A.err)) break;
            const int need = d0.x, e0 = d0.y, e1 = d0.z, kb = d0.w, kn = d1.x, g0 = d1.y;
            const int g1 = min(ng, g0 + GPS);
            const int nch = max(0, ((need + 31) >> 5) - loadedc);
            const unsigned mbytes = (unsigned)((e1 - e0) * RB), rbytes = (unsigned)((g1 - g0) * R * 16);
            const unsigned ibytes = (unsigned)(((g1 - g0 + 1) / 2) * 16);
            const unsigned kbytes = (unsigned)(kn * (4 + sizeof(T)));
            unsigned char* buf = bufs + (size_t)slot * bufsz;
            if (lane == 0) mbar_arrive_tx(&bar_full[slot], 2u * nch * chunkbytes + mbytes + rbytes + ibytes + kbytes);
            __syncwarp();
            for (int k = lane; k < 2 * nch; k += 32) {
                const int arr = k & 1, r0 = 32 * (loadedc + (k >> 1));
                tma_load3((arr ? rV : rX) + (size_t)(r0 % RW) * CW, arr ? &tmV : &tmX, t0, r0, s, &bar_full[slot]);
            }
            if (lane == 0) {
                unsigned char* b2 = buf;
                bulk_g2s(b2, rec + (size_t)e0 * RB, mbytes, &bar_full[slot]);
                b2 += (size_t)ME * RB;
                bulk_g2s(b2, rr_g + (size_t)g0 * R, rbytes, &bar_full[slot]);
                b2 += (size_t)GPS * R * 16;
                bulk_g2s(b2, gi_g + g0, ibytes, &bar_full[slot]);
                b2 += (size_t)GPS * 8;
                if (kn > 0) {
                    bulk_g2s(b2, A.kt_slot + kb, (unsigned)(kn * 4), &bar_full[slot]);
                    bulk_g2s(b2 + (size_t)MK * 4, ktv + kb, (unsigned)(kn * sizeof(T)), &bar_full[slot]);
                }
            }
            loadedc += nch;
            d0 = n0;
            d1 = n1;
        }
        if (q < npass) {
            // gave up: let the copies already issued land before the CTA can exit
            for (int qq = max(0, q - NB); qq < q; ++qq)
                if (!mbar_wait(&bar_full[qq % NB], (qq / NB) & 1, A.err)) break;
        }
        return;
    }
    // ---- consumers (shared memory read through explicit 32-bit shared addresses)
    const T* rom = reinterpret_cast<const T*>(A.romega) + (size_t)s * n;
    const bool wcol = t0 + CW > P - 1;   // this CTA holds the w_1 column
    const unsigned sX = smem_addr(rX) + EL * lane * (unsigned)sizeof(T);
    const unsigned sV = smem_addr(rV) + EL * lane * (unsigned)sizeof(T);
    const unsigned sB = smem_addr(bufs);
    const unsigned oRR = (unsigned)(ME * RB), oGI = oRR + GPS * R * 16, oKS = oGI + GPS * 8, oKV = oKS + MK * 4;
    for (int pass = 0; pass < npass; ++pass) {
        const int slot = pass % NB;
        if (!mbar_wait(&bar_full[slot], (pass / NB) & 1, A.err)) break;
        const int g = pass * GPS + warp;
        if (g < ng) {
            const unsigned buf = sB + (unsigned)(slot * bufsz);
            const int2 gi = lds_i2(buf + oGI + warp * 8);
            int4 rr[R];
            T romv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint4 u = lds_u4(buf + oRR + (warp * R + r) * 16);
                rr[r] = make_int4((int)u.x, (int)u.y, (int)u.z, (int)u.w);
                romv[r] = (wcol && rr[r].x >= 0) ? rom[rr[r].x] : T(0);
            }
            const unsigned mb = buf + gi.x * RB;
            T acc[R][EL];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < EL; ++c) acc[r][c] = T(0);
#pragma unroll 2
            for (int e = 0; e < gi.y; ++e) {
                unsigned wd[RW4];
#pragma unroll
                for (int k = 0; k < RB / 16; ++k) {
                    const uint4 u = lds_u4(mb + e * RB + 16 * k);
                    wd[4 * k] = u.x;
                    wd[4 * k + 1] = u.y;
                    wd[4 * k + 2] = u.z;
                    wd[4 * k + 3] = u.w;
                }
                const unsigned off = wd[0] * (unsigned)(CW * sizeof(T));
                T x[EL], v[EL];
                if constexpr (EL == 2) {
                    const float2 xx = lds_f2(sX + off);
                    const float2 vv = lds_f2(sV + off);
                    x[0] = xx.x;
                    x[1] = xx.y;
                    v[0] = vv.x;
                    v[1] = vv.y;
                } else {
                    x[0] = lds_t<T>(sX + off);
                    v[0] = lds_t<T>(sV + off);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    T a, bb;
                    if constexpr (sizeof(T) == 4) {
                        a = __uint_as_float(wd[2 + r]);
                        bb = __uint_as_float(wd[2 + R + r]);
                    } else {
                        a = __hiloint2double((int)wd[2 + 2 * r + 1], (int)wd[2 + 2 * r]);
                        bb = __hiloint2double((int)wd[2 + 2 * (R + r) + 1], (int)wd[2 + 2 * (R + r)]);
                    }
#pragma unroll
                    for (int c = 0; c < EL; ++c) acc[r][c] += a * x[c] + bb * v[c];
                }
            }
            // - K_t(q_k) X, then the store
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = rr[r].x;
                if (i < 0) continue;
                for (int e = rr[r].y; e < rr[r].z; ++e) {
                    const unsigned off = (unsigned)lds_i(buf + oKS + 4 * e) * (unsigned)(CW * sizeof(T));
                    const T kv = lds_t<T>(buf + oKV + e * (unsigned)sizeof(T));
                    if constexpr (EL == 2) {
                        const float2 xx = lds_f2(sX + off);
                        acc[r][0] -= kv * xx.x;
                        acc[r][1] -= kv * xx.y;
                    } else {
                        acc[r][0] -= kv * lds_t<T>(sX + off);
                    }
                }
                const int t = t0 + EL * lane;
#pragma unroll
                for (int c = 0; c < EL; ++c)
                    if (t + c == P - 1) acc[r][c] += romv[r];
                if (t < ld) {
                    if constexpr (EL == 2)
                        *reinterpret_cast<float2*>(Y + (size_t)i * ld + t) = make_float2(acc[r][0], acc[r][1]);
                    else
                        Y[(size_t)i * ld + t] = acc[r][0];
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_empty[slot]);
    }
}

// group records for the current w_1: slot, then A (R values), B (R values); fill entries 0
template <typename T>
__global__ void k_build_groups(int nE, int R, int RB, const int* __restrict__ map, const int* __restrict__ slot,
                               const T* __restrict__ Aop, const T* __restrict__ Bop, unsigned char* rec) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
        unsigned char* m = rec + (size_t)e * RB;
        *reinterpret_cast<int*>(m) = slot[e];
        *reinterpret_cast<int*>(m + 4) = 0;
        T* val = reinterpret_cast<T*>(m + 8);
        for (int r = 0; r < R; ++r) {
            const int q = map[(size_t)e * R + r];
            val[r] = q >= 0 ? Aop[q] : T(0);
            val[R + r] = q >= 0 ? Bop[q] : T(0);
        }
        for (size_t o = 8 + 2 * R * sizeof(T); o < (size_t)RB; o += 4) *reinterpret_cast<int*>(m + o) = 0;
    }
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

// 16-byte load/store of 16 / sizeof(T) consecutive elements (one vector per lane)
template <typename T>
__device__ __forceinline__ void ldv(const T* p, T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    } else {
        const double2 x = *reinterpret_cast<const double2*>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
}

template <typename T>
__device__ __forceinline__ void stv(T* p, const T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// 16-byte shared-memory vector load/store at a 32-bit shared address
template <typename T>
__device__ __forceinline__ void lds_vec(unsigned a, T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                     : "r"(a));
    else
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
}
template <typename T>
__device__ __forceinline__ void sts_vec(unsigned a, const T v[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4)
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                     "f"(v[3])
                     : "memory");
    else
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};\n" ::"r"(a), "d"(v[0]), "d"(v[1]) : "memory");
}

// packed FP32 pair helpers (fma.rn.f32x2: two IEEE fused multiply-adds per instruction)
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// Blocked banded substitution with 8 x EL register tiles (b <= 96): one CTA = one trajectory
// x CW = 64 EL directions (256 in FP32, 128 in FP64), 8 warps = 4 row groups of 8 rows x 2
// column halves.  Each shared-memory read of a solved row feeds 8 rows.  The factor of the
// block (its band tile and the diagonal-block inverse, one contiguous record written by the
// state kernel) comes by one bulk copy per block, double-buffered on mbarriers; the next
// block's right-hand side rows are loaded into registers while the current block computes.
//  FWD: y_B = Dinv_B (rhs_B - L_{B,<} y_<)      record Rf = [L(i0 + r, i0 - b + c) | Dinv^T]
//  BWD: x_B = Dinv_B^T (y_B - L_{>,B}^T x_>)    record Rb = [L(i0 + 32 + c, i0 + r) | Dinv]
//       then X <- x, V <- 2/D (x - X) - V.
// FP32: the products run as packed pairs of rows (fma.rn.f32x2, two IEEE FMAs per instruction,
// the same results as scalar FMAs with half the issue slots); the ring holds -x so that the band
// update is one packed FMA per pair.
template <typename T, bool FWD>
__global__ void __launch_bounds__(256, 1) k_trsm8(SensArgs A) {
    constexpr int EL = 16 / sizeof(T);             // columns per lane
    constexpr int CW = 64 * EL;                    // columns per CTA
    constexpr int RT = 8;                          // rows per thread
    const int n = A.n, b = A.b, ld = A.ld, RM = A.RWT - 1, RECE = A.RECE, nblk = A.nblk;
    const int s = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Row group of a warp: the zeros of the band tile and of the diagonal-block inverse are
    // skipped, so the row groups do unequal work (FWD: b - 8 rg band columns and 8 + 8 rg
    // diagonal ones); the second column half takes the row groups in reverse order, so the
    // two warps that share a scheduler (warp and warp + 4) always do the same work in total.
    const int cg = warp >> 2, rg = cg ? 3 - (warp & 3) : (warp & 3);
    const int r0 = RT * rg;                        // first row of this thread in the block
    const int cl = cg * (CW / 2) + EL * lane;      // first column of this thread in the tile
    const int t = blockIdx.x * CW + cl;            // global column
    const bool tok = t < ld;
    __shared__ __align__(8) unsigned long long bar[2];
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ring = reinterpret_cast<T*>(smraw);                        // RWT x CW  solved rows
    T* stg = ring + (size_t)A.RWT * CW;                           // 32 x CW   block before Dinv
    T* rec0 = stg + (size_t)FSE_BLK * CW;                         // 2 records
    T* rec1 = rec0 + RECE;
    // shared memory is read and written through explicit 32-bit shared addresses
    constexpr unsigned TS = sizeof(T);
    const unsigned sRing = smem_addr(ring) + cl * TS, sStg = smem_addr(stg), sRec0 = smem_addr(rec0);
    const unsigned recb = (unsigned)RECE * TS;
    const T* R = reinterpret_cast<const T*>(FWD ? A.Rf : A.Rb) + (size_t)s * nblk * RECE;
    const size_t base = (size_t)s * n * ld;
    T* Y = reinterpret_cast<T*>(A.Y) + base;
    T* X = reinterpret_cast<T*>(A.X) + base;
    T* V = reinterpret_cast<T*>(A.V) + base;
    const T a2 = T(A.a2c);
    const int dofs = RECE - FSE_BLK * FSE_BLK;
    const unsigned recbytes = (unsigned)(RECE * sizeof(T));
    auto blk = [&](int q) { return FWD ? q : nblk - 1 - q; };
    auto load_rows = [&](const T* src, int B, T out[RT][EL]) {
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) {
            const int i = B * FSE_BLK + r0 + rr;
            if (i < n && tok) {
                ldv(src + (size_t)i * ld + t, out[rr]);
            } else {
#pragma unroll
                for (int e = 0; e < EL; ++e) out[rr][e] = T(0);
            }
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_tx(&bar[0], recbytes);
        bulk_g2s(rec0, R + (size_t)blk(0) * RECE, recbytes, &bar[0]);
    }
    T ynext[RT][EL];
    load_rows(Y, blk(0), ynext);
    bool ok = true;
    for (int q = 0; q < nblk; ++q) {
        const int B = blk(q), i0 = B * FSE_BLK, buf = q & 1;
        // the record buffer of block q + 1 was last read by block q - 1 (finished at its last barrier)
        if (threadIdx.x == 0 && q + 1 < nblk) {
            mbar_arrive_tx(&bar[buf ^ 1], recbytes);
            bulk_g2s(buf ? rec0 : rec1, R + (size_t)blk(q + 1) * RECE, recbytes, &bar[buf ^ 1]);
        }
        T acc[RT][EL], xo[RT][EL], vo[RT][EL];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr)
#pragma unroll
            for (int e = 0; e < EL; ++e) acc[rr][e] = ynext[rr][e];
        if (q + 1 < nblk) load_rows(Y, blk(q + 1), ynext);
        // BWD: X_k and V_k rows of the next block go to L2 now, so that their loads after the
        // next band part hit L2
        if (!FWD && q + 1 < nblk && tok) {
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) {
                const int i = blk(q + 1) * FSE_BLK + r0 + rr;
                if (i < n) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(X + (size_t)i * ld + t));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(V + (size_t)i * ld + t));
                }
            }
        }
        const bool wok = mbar_wait(&bar[buf], (q >> 1) & 1, A.err);
        const unsigned sL = sRec0 + (buf ? recb : 0u) + r0 * TS;     // this thread's 8 rows of the record
        // band part: rows of earlier (FWD) or later (BWD) blocks from the ring.  Record column c
        // is zero for row r when c < r (FWD: L(i0 + r, i0 - b + c) lies outside the band) or when
        // c > b - 32 + r (BWD: L(i0 + 32 + c, i0 + r)), so this thread's rows r0 .. r0 + 7 need
        // c >= r0 (FWD) or c < b - 24 + r0 (BWD) only.
        const int c0 = FWD ? max(max(0, b - i0), r0) : 0;
        const int c1 = FWD ? b : min(min(b, n - (i0 + FSE_BLK)), b - FSE_BLK + RT + r0);
        // the operands of column c + 1 are read from shared memory before the products of column c
        auto ldc = [&](int c, T xv[EL], T lv[RT]) {
            const int rowg = FWD ? (i0 - b + c) : (i0 + FSE_BLK + c);
            lds_vec<T>(sRing + (unsigned)(rowg & RM) * (CW * TS), xv);
#pragma unroll
            for (int k = 0; k < RT / EL; ++k) lds_vec<T>(sL + (c * FSE_BLK + EL * k) * TS, lv + EL * k);
        };
        // FP32: accumulators in row pairs, the ring holds -y, so one packed FMA gives acc - l y
        unsigned long long A2[RT / 2][EL];
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int p2 = 0; p2 < RT / 2; ++p2)
#pragma unroll
                for (int e = 0; e < EL; ++e) A2[p2][e] = pk2(acc[2 * p2][e], acc[2 * p2 + 1][e]);
        }
        auto fmc = [&](const T xv[EL], const T lv[RT]) {
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int e = 0; e < EL; ++e) {
                    const unsigned long long xd = pk2(xv[e], xv[e]);
#pragma unroll
                    for (int p2 = 0; p2 < RT / 2; ++p2) fma2(A2[p2][e], pk2(lv[2 * p2], lv[2 * p2 + 1]), xd);
                }
            } else {
#pragma unroll
                for (int rr = 0; rr < RT; ++rr)
#pragma unroll
                    for (int e = 0; e < EL; ++e) acc[rr][e] -= lv[rr] * xv[e];
            }
        };
        {
            T xa[EL], la[RT], xb[EL], lb[RT];
            int c = c0;
            if (c < c1) ldc(c, xa, la);
            for (; c + 1 < c1; c += 2) {
                ldc(c + 1, xb, lb);
                fmc(xa, la);
                if (c + 2 < c1) ldc(c + 2, xa, la);
                fmc(xb, lb);
            }
            if (c < c1) fmc(xa, la);
        }
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int p2 = 0; p2 < RT / 2; ++p2)
#pragma unroll
                for (int e = 0; e < EL; ++e) upk2(A2[p2][e], acc[2 * p2][e], acc[2 * p2 + 1][e]);
        }
        // X_k and V_k of the block (for the V update) are read after the band part: fewer live
        // registers during it, and still a whole diagonal step ahead of their use
        if (!FWD) {
            load_rows(X, B, xo);
            load_rows(V, B, vo);
        }
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) sts_vec<T>(sStg + ((r0 + rr) * CW + cl) * TS, acc[rr]);
        ok = __syncthreads_and(wok) != 0;   // the whole CTA leaves together if a wait gave up
        if (!ok) {
            if (threadIdx.x == 0 && q + 1 < nblk) mbar_wait(&bar[buf ^ 1], ((q + 1) >> 1) & 1, A.err);
            break;
        }
        // diagonal block: out_r = sum_k D'[k][r] stg_k with D' = Dinv^T (FWD) or Dinv (BWD)
        T out[RT][EL];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr)
#pragma unroll
            for (int e = 0; e < EL; ++e) out[rr][e] = T(0);
        // Dinv is lower triangular: row r takes k <= r (FWD, D'[k][r] = Dinv[r][k]) or k >= r
        // (BWD, D'[k][r] = Dinv[k][r]), so this thread needs k < r0 + 8 (FWD) or k >= r0 (BWD)
        const unsigned sD = sL + dofs * TS;
        const int k0 = FWD ? 0 : r0, k1 = FWD ? r0 + RT : FSE_BLK;
        unsigned long long O2[RT / 2][EL];
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int p2 = 0; p2 < RT / 2; ++p2)
#pragma unroll
                for (int e = 0; e < EL; ++e) O2[p2][e] = 0ull;
        }
        for (int kb = k0; kb < k1; kb += RT) {
#pragma unroll
            for (int kk = 0; kk < RT; ++kk) {
                const int k = kb + kk;
                T tv[EL], dv[RT];
                lds_vec<T>(sStg + (k * CW + cl) * TS, tv);
#pragma unroll
                for (int j = 0; j < RT / EL; ++j) lds_vec<T>(sD + (k * FSE_BLK + EL * j) * TS, dv + EL * j);
                if constexpr (sizeof(T) == 4) {
#pragma unroll
                    for (int e = 0; e < EL; ++e) {
                        const unsigned long long td = pk2(tv[e], tv[e]);
#pragma unroll
                        for (int p2 = 0; p2 < RT / 2; ++p2) fma2(O2[p2][e], pk2(dv[2 * p2], dv[2 * p2 + 1]), td);
                    }
                } else {
#pragma unroll
                    for (int rr = 0; rr < RT; ++rr)
#pragma unroll
                        for (int e = 0; e < EL; ++e) out[rr][e] += dv[rr] * tv[e];
                }
            }
        }
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int p2 = 0; p2 < RT / 2; ++p2)
#pragma unroll
                for (int e = 0; e < EL; ++e) upk2(O2[p2][e], out[2 * p2][e], out[2 * p2 + 1][e]);
        }
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) {
            const int i = i0 + r0 + rr;
            if constexpr (sizeof(T) == 4) {
                T ng[EL];
#pragma unroll
                for (int e = 0; e < EL; ++e) ng[e] = -out[rr][e];
                sts_vec<T>(sRing + (unsigned)(i & RM) * (CW * TS), ng);
            } else {
                sts_vec<T>(sRing + (unsigned)(i & RM) * (CW * TS), out[rr]);
            }
            if (i < n && tok) {
                const size_t o = (size_t)i * ld + t;
                if (FWD) {
                    stv(Y + o, out[rr]);
                } else {
                    T vn[EL];
#pragma unroll
                    for (int e = 0; e < EL; ++e) vn[e] = a2 * (out[rr][e] - xo[rr][e]) - vo[rr][e];
                    stv(X + o, out[rr]);
                    stv(V + o, vn);
                }
            }
        }
        __syncthreads();
    }
}

// Velocity-dependent elements (C_t = d f_nl / d qdot != 0): the right-hand side of the tangent
// step gains (w 2/D C_t(k+1)) X_k + w (C_t(k+1) - C_t(k)) V_k (the linearised equation of motion of
// step k eliminates the acceleration tangent as in the C_t = 0 case, and the velocity tangent of
// the new step enters through u' = 2/D (q' - q_k') - u_k').  C_t lives on the K_t pattern; one
// thread per tangent column, rows without velocity-tangent entries are skipped.
template <typename T>
__global__ void k_ct_rhs(int n, int ld, int kt_ld, double wa2, double w, const int* __restrict__ kt_ptr,
                         const int* __restrict__ kt_col, const T* __restrict__ c1, const T* __restrict__ c0,
                         const T* __restrict__ X, const T* __restrict__ V, T* Y) {
    const int s = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ld) return;
    const size_t base = (size_t)s * n * ld;
    const T* C1 = c1 + (size_t)s * kt_ld;
    const T* C0 = c0 + (size_t)s * kt_ld;
    for (int i = 0; i < n; ++i) {
        const int e0 = kt_ptr[i], e1 = kt_ptr[i + 1];
        if (e0 == e1) continue;
        double acc = 0.0;
        for (int e = e0; e < e1; ++e) {
            const size_t o = base + (size_t)kt_col[e] * ld + t;
            acc += wa2 * (double)C1[e] * (double)X[o] + w * ((double)C1[e] - (double)C0[e]) * (double)V[o];
        }
        Y[base + (size_t)i * ld + t] = T((double)Y[base + (size_t)i * ld + t] + acc);
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
    const size_t cw = tsz == 4 ? 64 : 32;
    const size_t buf = (size_t)p.ME * p.RB + (size_t)FSE_RHS_GPS * p.R * 16 + (size_t)FSE_RHS_GPS * 8 +
                       (size_t)p.MK * (4 + tsz);
    const int dep = tsz == 4 ? FSE_RHS_DEPTH_F32 : FSE_RHS_DEPTH_F64;
    return 128 + (size_t)2 * p.RW * cw * tsz + (size_t)(dep + 1) * buf;
}

int make_tangent_maps(fse_ctx* c) {
    using encode_fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    // cuTensorMapEncodeTiled from the CUDA driver API, looked up once per process (thread-safe static
    // initialisation)
    static const encode_fn encode = []() -> encode_fn {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<encode_fn>(fn);
    }();
    if (!encode) return FSE_ECUDA;
    const Params& p = c->p;
    const bool f32 = p.prec == FSE_MIXED_FP32;
    const size_t tsz = f32 ? 4 : 8;
    const cuuint32_t cw = f32 ? 64 : 32;
    const cuuint64_t dims[3] = {(cuuint64_t)p.ld, (cuuint64_t)p.n, (cuuint64_t)p.N};
    const cuuint64_t strides[2] = {(cuuint64_t)p.ld * tsz, (cuuint64_t)p.n * p.ld * tsz};
    const cuuint32_t box[3] = {cw, 32, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    for (int k = 0; k < 2; ++k) {
        CUtensorMap* m = k ? &c->tmV : &c->tmX;
        void* ptr = k ? c->d.V : c->d.X;
        if (encode(m, dt, 3, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return FSE_ECUDA;
    }
    return FSE_OK;
}

void launch_build_groups(fse_ctx* c) {
    const Params& p = c->p;
    const int g = nblocks(p.nE, 256);
    if (p.prec == FSE_MIXED_FP32)
        k_build_groups<float><<<g, 256, 0, c->stream>>>(p.nE, p.R, p.RB, c->d.g_map, c->d.g_slot,
                                                        (const float*)c->d.cs_A, (const float*)c->d.cs_B,
                                                        (unsigned char*)c->d.g_rec);
    else
        k_build_groups<double><<<g, 256, 0, c->stream>>>(p.nE, p.R, p.RB, c->d.g_map, c->d.g_slot,
                                                         (const double*)c->d.cs_A, (const double*)c->d.cs_B,
                                                         (unsigned char*)c->d.g_rec);
}

template <typename T, int R>
static void rhs_launch(fse_ctx* c, const SensArgs& A, cudaStream_t st) {
    static std::atomic<unsigned long long> attr{0};
    if (needs_device_setup(attr)) {
        cudaFuncSetAttribute(k_sens_rhs<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        mark_device(attr);
    }
    const Params& p = c->p;
    constexpr int CW = sizeof(T) == 4 ? 64 : 32;
    dim3 g((p.P + CW - 1) / CW, p.N);
    k_sens_rhs<T, R><<<g, 32 * (FSE_RHS_GPS + 1), p.smem_rhs, st>>>(A, c->tmX, c->tmV);
}

size_t trsm_smem(const Params& p) {
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    if (p.b <= 96) {   // k_trsm8: ring + staging block of CW = 64 x 16 / tsz columns + 2 records
        const size_t cw = 64 * (16 / tsz);
        return ((size_t)p.RWT * cw + (size_t)FSE_BLK * cw + 2 * (size_t)p.RECE) * tsz;
    }
    return ((size_t)p.RWT * 128 + 2 * ((size_t)((p.b + 3) & ~3) * 32 + 1024)) * tsz;
}

template <typename T>
static void sens_launch(fse_ctx* c, const SensArgs& A, int phase, cudaStream_t st) {
    const Params& p = c->p;
    static std::atomic<unsigned long long> attr{0};
    if (needs_device_setup(attr)) {
        cudaFuncSetAttribute(k_trsm<T, true, 28>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        cudaFuncSetAttribute(k_trsm<T, false, 28>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        mark_device(attr);
    }
    if (phase == 0) {
        switch (p.R) {
            case 1: rhs_launch<T, 1>(c, A, st); break;
            case 2: rhs_launch<T, 2>(c, A, st); break;
            case 3: rhs_launch<T, 3>(c, A, st); break;
            default: rhs_launch<T, 4>(c, A, st); break;
        }
    } else if (p.b <= 96) {
        static std::atomic<unsigned long long> attr8{0};
        if (needs_device_setup(attr8)) {
            cudaFuncSetAttribute(k_trsm8<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
            cudaFuncSetAttribute(k_trsm8<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
            mark_device(attr8);
        }
        constexpr int CW = 64 * (16 / (int)sizeof(T));
        dim3 g((p.P + CW - 1) / CW, p.N);
        if (phase == 1)
            k_trsm8<T, true><<<g, 256, p.smem_trsm, st>>>(A);
        else
            k_trsm8<T, false><<<g, 256, p.smem_trsm, st>>>(A);
    } else {
        // 96 < b <= FSE_MAX_BAND (224): the factor tile of b x 32 values over 256 threads needs
        // MAXL = 28 registers per thread
        dim3 g((p.P + 127) / 128, p.N);
        if (phase == 1)
            k_trsm<T, true, 28><<<g, 256, p.smem_trsm, st>>>(A);
        else
            k_trsm<T, false, 28><<<g, 256, p.smem_trsm, st>>>(A);
    }
}

void launch_sens_init(fse_ctx* c, cudaStream_t st) {
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * p.n * p.ld;
    if (p.prec == FSE_MIXED_FP32)
        k_sens_init<float><<<nblocks(tot, 256, 64), 256, 0, st>>>(p.N, p.n, p.ld, (float*)c->d.X,
                                                                       (float*)c->d.V);
    else
        k_sens_init<double><<<nblocks(tot, 256, 64), 256, 0, st>>>(p.N, p.n, p.ld, (double*)c->d.X,
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
    A.kt_ld = p.kt_ld;
    A.MK = p.MK;
    A.nblk = p.nblk;
    A.RW = p.RW;
    A.RWT = p.RWT;
    A.RECE = p.RECE;
    A.a2c = 2.0 / Dl;
    A.ng = p.ng;
    A.ME = p.ME;
    A.RB = p.RB;
    A.g_rr = c->d.g_rr;
    A.g_info = c->d.g_info;
    A.g_pass = c->d.g_pass;
    A.g_rec = c->d.g_rec;
    A.kt_slot = c->d.kt_slot;
    A.err = c->d.flag;
    const size_t ktsz = (size_t)p.N * p.kt_ld * tsz;
    const size_t fsz = (size_t)p.N * p.n * (p.b + 1) * tsz;
    const size_t vsz = (size_t)p.N * p.n * tsz;
    const size_t dsz = (size_t)p.N * p.nblk * FSE_BLK * FSE_BLK * tsz;
    const int f = k % 2;
    A.kt_val = (const char*)c->d.kt_val + (k % FSE_NBUF_KT) * ktsz;   // K_t(q_k)
    A.romega = (const char*)c->d.romega + f * vsz;
    A.Lc = (const char*)c->d.Lc + f * fsz;                             // factor of K_eff(q_{k+1})
    A.Lr = (const char*)c->d.Lr + f * fsz;
    A.Dinv = (const char*)c->d.Dinv + f * dsz;
    const size_t rsz = (size_t)p.N * p.nblk * p.RECE * tsz;
    A.Rf = (const char*)c->d.Rf + f * rsz;
    A.Rb = (const char*)c->d.Rb + f * rsz;
    A.X = c->d.X;
    A.V = c->d.V;
    A.Y = c->d.Y;
    if (phase == 0 && p.has_vel) {
        // the plain right-hand side first, then the velocity-tangent terms on top of it
        if (p.prec == FSE_MIXED_FP32)
            sens_launch<float>(c, A, 0, st);
        else
            sens_launch<double>(c, A, 0, st);
        const size_t csz = (size_t)p.N * p.kt_ld * tsz;
        const void* c1 = (const char*)c->d.ct_val + ((k + 1) % FSE_NBUF_KT) * csz;
        const void* c0 = (const char*)c->d.ct_val + (k % FSE_NBUF_KT) * csz;
        const dim3 g((p.ld + 127) / 128, p.N);
        const double wa2 = w * 2.0 / Dl;
        if (p.prec == FSE_MIXED_FP32)
            k_ct_rhs<float><<<g, 128, 0, st>>>(p.n, p.ld, p.kt_ld, wa2, w, c->d.kt_ptr, c->d.kt_col,
                                               (const float*)c1, (const float*)c0, (const float*)c->d.X,
                                               (const float*)c->d.V, (float*)c->d.Y);
        else
            k_ct_rhs<double><<<g, 128, 0, st>>>(p.n, p.ld, p.kt_ld, wa2, w, c->d.kt_ptr, c->d.kt_col,
                                                (const double*)c1, (const double*)c0, (const double*)c->d.X,
                                                (const double*)c->d.V, (double*)c->d.Y);
        return;
    }
    if (phase > 0 && use_tc(c)) {
        launch_tc_solve(c, k, phase, st);
        return;
    }
    if (p.prec == FSE_MIXED_FP32)
        sens_launch<float>(c, A, phase, st);
    else
        sens_launch<double>(c, A, phase, st);
}

}  // namespace fse
