// Tensor-core form of the blocked banded tangent solves (App. E: the sensitivities X = dq/dp of
// all 2n+1 directions go through the factor of the same effective stiffness K_eff = L L^T).
//
// Forward   L Y' = Y:      Y'_t = Dinv_t Y_t - sum_{u=1..ND} G(t, t-u) Y'_{t-u}
// Backward  L^T X = Y':    X_t  = Dinv_t^T Y'_t - sum_{u=1..ND} H(t, t+u) X_{t+u},
//                          then V_{k+1} = 2/D (X_{k+1} - X_k) - V_k
// over 32-row blocks t (ND = ceil(b / 32) coupled blocks for half-bandwidth b <= 96), with the
// couplings premultiplied by the inverse of the target's diagonal block:
//     G(t, s) = Dinv_t L_{t,s},   H(t, s) = Dinv_t^T L_{s,t}^T,
// so that each block costs one accumulation in tensor memory and one read-out.
//
// Precision: FP32-level products from TF32 tensor cores by splitting both operands,
// a = a_hi + a_lo with a_hi = a with its 13 low mantissa bits cleared (exact in TF32) and
// a_lo = a - a_hi (exact in FP32), and summing a_lo b_hi + a_hi b_lo + a_hi b_hi with FP32
// accumulation (the dropped a_lo b_lo is 2^-22 relative).
//
// One CTA solves 128 tangent columns of one trajectory.  The MMA is D[m][r] += sum_k
// A[m][k] B[r][k] with M = 128 (tangent columns, TMEM lanes), N = 32 (rows of the target
// block, TMEM columns) and K = 32 (rows of the source block), kind::tf32, both operands
// K-major in shared memory without swizzle.  Four accumulators of 32 TMEM columns rotate over
// the blocks.  Roles: warps 0-3 (epilogue, thread m = column m) read a finished block out of
// TMEM, store it, stage it as the A operand of later blocks and stage the right-hand side of
// the block two ahead; warp 4 (one thread) issues the MMAs; warp 5 (one thread) streams the
// factor records with bulk copies.  After block q is read out ("round q") the MMA thread issues
//   1. the critical term of block q+1: G(q+1, q) Y'_q, then commits block q+1;
//   2. the right-hand-side term Dinv_{q+2} Y_{q+2} and the terms G(q+2, q) Y'_q, G(q+3, q) Y'_q.
// The accumulators are zeroed by the epilogue after each read-out, so every MMA accumulates.
// Every wait is bounded (about 2 s of SM clock); a wait that gives up raises the context's
// error flag, the CTA drains its MMAs and copies in flight, frees its tensor memory and exits.
#include <cuda_runtime.h>

#include "fse_common.cuh"

namespace fse {

constexpr int TC_M = 128;                       // tangent columns per CTA (MMA M, TMEM lanes)
constexpr int TC_MAT = FSE_BLK * FSE_BLK;       // floats of one 32 x 32 operand
constexpr int TC_REC = 8 * TC_MAT;              // floats of one record: 4 operands x (hi, lo)
constexpr int TC_AOP = TC_M * FSE_BLK;          // floats of one 128 x 32 A operand (hi or lo)
constexpr int TC_NREC = 3;                      // record slots in shared memory
constexpr unsigned TC_SMEM = (unsigned)((2 * 2 + 2 * 2) * TC_AOP + TC_NREC * TC_REC) * 4u;
constexpr unsigned TC_TMEM_COLS = 128;          // 4 accumulators x 32 columns
constexpr int TC_THREADS = 192;

// Byte offset of element (row, k), k < 32, of a K-major operand in the no-swizzle canonical
// layout: 8 rows x 16 bytes per core matrix, K-adjacent core matrices 128 bytes apart (the
// descriptor's leading byte offset), 8-row groups 1024 bytes apart (its stride byte offset).
__host__ __device__ constexpr unsigned kmaj_off(int row, int k) {
    return (unsigned)((row & 7) * 16 + (k & 3) * 4 + (k >> 2) * 128 + (row >> 3) * 1024);
}

// shared-memory matrix descriptor: start address, leading byte offset 128 (K direction),
// stride byte offset 1024 (8-row groups), descriptor version 1, no swizzle
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr) {
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(128u >> 4) << 16) |
           ((unsigned long long)(1024u >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N = 32, M = 128
constexpr unsigned TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned dtm, unsigned long long ad, unsigned long long bd) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %4, p;\n}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(1), "r"(TC_IDESC)
        : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane (warp w reads lanes 32 (w % 4) ..)
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float v[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// zero 32 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_zero32(unsigned taddr) {
    const unsigned z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(taddr),
        "r"(z)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// TF32 split: hi exact in TF32 (13 low mantissa bits cleared), lo = x - hi exact in FP32
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// rows 32 B .. 32 B + 31 of column t of a tangent-sized array (zero outside)
__device__ __forceinline__ void load_col32(const float* base, int B, int n, int ld, int t, float v[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = B * FSE_BLK + r;
        v[r] = (i < n && t < ld) ? __ldcs(base + (size_t)i * ld + t) : 0.0f;
    }
}

// L2 prefetch of rows 32 B .. 32 B + 31 of the warp's 32 columns t0w .. t0w + 31 (lane r: row r;
// the 128-byte segment may straddle two lines)
__device__ __forceinline__ void prefetch_rows32(const float* base, int B, int n, int ld, int t0w) {
    const int r = threadIdx.x & 31, i = B * FSE_BLK + r;
    if (B < 0 || i >= n || t0w >= ld) return;
    const float* a = base + (size_t)i * ld + t0w;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a + min(31, ld - 1 - t0w)));
}

// this thread's row m of a 128 x 32 A operand (hi at sA, lo at sA + TC_AOP floats)
__device__ __forceinline__ void stage_row(unsigned sA, int m, const float v[32]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = tf32_hi(v[4 * c + j]);
            l[j] = v[4 * c + j] - h[j];
        }
        const unsigned o = kmaj_off(m, 4 * c);
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(sA + o), "f"(h[0]), "f"(h[1]), "f"(h[2]),
                     "f"(h[3])
                     : "memory");
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(sA + TC_AOP * 4u + o), "f"(l[0]), "f"(l[1]),
                     "f"(l[2]), "f"(l[3])
                     : "memory");
    }
}

// D (32 TMEM columns at dtm) += A (128 x 32, hi at sA, lo at sA + 16 KB) B^T (B 32 x 32, hi at sB,
// lo at sB + 4 KB): per K step of 8, the three split products, small ones first
__device__ __forceinline__ void mma_k32(unsigned dtm, unsigned sA, unsigned sB) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const unsigned long long ah = tc_desc(sA + kk * 256u), al = tc_desc(sA + TC_AOP * 4u + kk * 256u);
        const unsigned long long bh = tc_desc(sB + kk * 256u), bl = tc_desc(sB + TC_MAT * 4u + kk * 256u);
        tc_mma(dtm, al, bh);
        tc_mma(dtm, ah, bl);
        tc_mma(dtm, ah, bh);
    }
}

struct TcArgs {
    int n, ld, nblk, ND;
    float a2c;
    int* err;
    const float* rec;   // N x (nblk + 1) records of this direction
    float *X, *V, *Y;
};

template <bool FWD>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_solve(TcArgs A) {
    const int n = A.n, ld = A.ld, nblk = A.nblk, ND = A.ND;
    const int s = blockIdx.y, t0 = blockIdx.x * TC_M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ __align__(128) unsigned char smraw[];
    // A operands of the last two solved blocks [2][hi | lo], staged right-hand sides [2][hi | lo],
    // factor records [3]
    const unsigned sAop = smem_addr(smraw);
    const unsigned sRhs = sAop + 2u * 2u * TC_AOP * 4u;
    const unsigned sRec = sRhs + 2u * 2u * TC_AOP * 4u;
    float* recs = reinterpret_cast<float*>(smraw + (size_t)8 * TC_AOP * 4);
    // rhs_ready[a & 1] completes arrival a of the staged right-hand sides (a = 0: blocks 0 and 1 in the
    // prologue, a = q + 1: block q + 2 in round q); two barriers so that the MMA thread, which waits
    // for arrival a after committing block q + 1, can never see arrival a + 2 on the same barrier first
    __shared__ __align__(8) unsigned long long acc_full[4], rec_full[TC_NREC], epi_done, rhs_ready[2], drain;
    __shared__ unsigned s_taddr;
    __shared__ volatile int s_abort;
    const size_t base = (size_t)s * n * ld;
    float* Y = A.Y + base;
    float* X = A.X + base;
    float* V = A.V + base;
    const float* R = A.rec + (size_t)s * (nblk + 1) * TC_REC;
    auto blk = [&](int q) { return FWD ? q : nblk - 1 - q; };
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) mbar_init(&acc_full[k], 1);
        for (int k = 0; k < TC_NREC; ++k) mbar_init(&rec_full[k], 1);
        mbar_init(&epi_done, 128);
        mbar_init(&rhs_ready[0], 128);
        mbar_init(&rhs_ready[1], 128);
        mbar_init(&drain, 1);
        s_abort = 0;
        mbar_fence_init();
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&s_taddr)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tbase = s_taddr;
    const unsigned recb = (unsigned)TC_REC * 4u;

    if (warp < 4) {
        // ---------------- epilogue: thread m = column t0 + m, TMEM lane m
        const int m = threadIdx.x, t = t0 + m;
        const unsigned tl = tbase + ((unsigned)(warp * 32) << 16);
        for (int a = 0; a < 4; ++a) tmem_zero32(tl + a * 32);
        float rhs[32];
        load_col32(Y, blk(0), n, ld, t, rhs);
        stage_row(sRhs, m, rhs);
        if (nblk > 1) {
            load_col32(Y, blk(1), n, ld, t, rhs);
            stage_row(sRhs + 2u * TC_AOP * 4u, m, rhs);
        }
        fence_async_smem();
        tc_fence_before();
        mbar_arrive(&rhs_ready[0]);
        const int t0w = t0 + warp * 32;
        for (int q = 2; q < 5 && q < nblk; ++q) prefetch_rows32(Y, blk(q), n, ld, t0w);
        if (!FWD)
            for (int q = 0; q < 3 && q < nblk; ++q) {
                prefetch_rows32(X, blk(q), n, ld, t0w);
                prefetch_rows32(V, blk(q), n, ld, t0w);
            }
        for (int q = 0; q < nblk; ++q) {
            const int B = blk(q);
            const bool more = q + 2 < nblk;
            // L2 prefetch three blocks ahead of the loads below: right-hand side rows of block q + 5,
            // backward X_k and V_k rows of block q + 3
            if (q + 5 < nblk) prefetch_rows32(Y, blk(q + 5), n, ld, t0w);
            if (!FWD && q + 3 < nblk) {
                prefetch_rows32(X, blk(q + 3), n, ld, t0w);
                prefetch_rows32(V, blk(q + 3), n, ld, t0w);
            }
            if (more) load_col32(Y, blk(q + 2), n, ld, t, rhs);
            float xo[32], vo[32];
            if (!FWD) {
                load_col32(X, B, n, ld, t, xo);
                load_col32(V, B, n, ld, t, vo);
            }
            if (s_abort || !mbar_wait(&acc_full[q & 3], (q >> 2) & 1, A.err)) {
                s_abort = 1;
                break;
            }
            tc_fence_after();
            float y[32];
            tmem_ld32(tl + (q & 3) * 32, y);
            tmem_zero32(tl + (q & 3) * 32);   // ready for block q + 4
            stage_row(sAop + (unsigned)(q & 1) * 2u * TC_AOP * 4u, m, y);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(&epi_done);
            if (t < ld) {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const int i = B * FSE_BLK + r;
                    if (i < n) {
                        const size_t o = (size_t)i * ld + t;
                        if (FWD) {
                            __stcs(Y + o, y[r]);
                        } else {
                            __stcs(X + o, y[r]);
                            __stcs(V + o, A.a2c * (y[r] - xo[r]) - vo[r]);
                        }
                    }
                }
            }
            if (more) stage_row(sRhs + (unsigned)(q & 1) * 2u * TC_AOP * 4u, m, rhs);
            fence_async_smem();
            mbar_arrive(&rhs_ready[(q + 1) & 1]);
        }
    } else if (warp == 4) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            bool ok = mbar_wait(&rec_full[0], 0, A.err) && mbar_wait(&rhs_ready[0], 0, A.err);
            if (ok) {
                tc_fence_after();
                // round -1: the right-hand-side terms of blocks 0 and 1 (record 0: Dinv'_0, Dinv'_1)
                mma_k32(tbase + 0, sRhs, sRec);
                tc_commit(&acc_full[0]);
                if (nblk > 1) mma_k32(tbase + 32, sRhs + 2u * TC_AOP * 4u, sRec + 2u * TC_MAT * 4u);
            }
            for (int q = 0; ok && q < nblk; ++q) {
                if (s_abort || !mbar_wait(&epi_done, q & 1, A.err)) {
                    ok = false;
                    break;
                }
                if (q + 1 >= nblk) break;
                const int rs = (q + 1) % TC_NREC;
                if (!mbar_wait(&rec_full[rs], ((q + 1) / TC_NREC) & 1, A.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned sA = sAop + (unsigned)(q & 1) * 2u * TC_AOP * 4u;
                const unsigned sB = sRec + (unsigned)rs * recb;
                // record q + 1: [-G(q+1, q), -G(q+2, q), -G(q+3, q), Dinv'_{q+2}], each hi | lo
                if (ND >= 1) mma_k32(tbase + ((q + 1) & 3) * 32, sA, sB);
                tc_commit(&acc_full[(q + 1) & 3]);
                // arrival q + 1 (right-hand side of block q + 2 staged by the epilogue of block q)
                if (!mbar_wait(&rhs_ready[(q + 1) & 1], ((q + 1) >> 1) & 1, A.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (q + 2 < nblk) {
                    mma_k32(tbase + ((q + 2) & 3) * 32, sRhs + (unsigned)(q & 1) * 2u * TC_AOP * 4u,
                            sB + 6u * TC_MAT * 4u);
                    if (ND >= 2) mma_k32(tbase + ((q + 2) & 3) * 32, sA, sB + 2u * TC_MAT * 4u);
                }
                if (ND >= 3 && q + 3 < nblk) mma_k32(tbase + ((q + 3) & 3) * 32, sA, sB + 4u * TC_MAT * 4u);
            }
            if (!ok) s_abort = 1;
            // every MMA issued has finished before the tensor memory is released
            tc_commit(&drain);
            mbar_wait(&drain, 0, A.err);
        }
    } else {
        // ---------------- factor records (one thread): record r into slot r % 3
        if (lane == 0) {
            int issued = 0;
            for (int r = 0; r < TC_NREC && r < nblk; ++r) {
                mbar_arrive_tx(&rec_full[r], recb);
                bulk_g2s(recs + (size_t)r * TC_REC, R + (size_t)r * TC_REC, recb, &rec_full[r]);
                issued = r + 1;
            }
            // record q + 3 (round q + 2) replaces record q once block q + 1 is committed, which
            // implies that every MMA of round q - 1 (the last reader of record q) has finished
            for (int q = 0; q + 3 < nblk; ++q) {
                if (s_abort || !mbar_wait(&acc_full[(q + 1) & 3], ((q + 1) >> 2) & 1, A.err)) {
                    s_abort = 1;
                    break;
                }
                const int r = q + 3, sl = r % TC_NREC;
                mbar_arrive_tx(&rec_full[sl], recb);
                bulk_g2s(recs + (size_t)sl * TC_REC, R + (size_t)r * TC_REC, recb, &rec_full[sl]);
                issued = r + 1;
            }
            // the copies in flight land before the CTA can exit
            for (int r = max(0, issued - TC_NREC); r < issued; ++r)
                if (!mbar_wait(&rec_full[r % TC_NREC], (r / TC_NREC) & 1, A.err)) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TC_TMEM_COLS)
                     : "memory");
}

// Factor records of both directions for the tensor-core solves, one CTA per (target block in
// processing order tau, trajectory, direction).  Processing order: forward blocks 0, 1, ..;
// backward blocks nblk-1, nblk-2, ...  Record sigma + 1 holds the B operands of round sigma:
//   [-C(sigma+1, sigma), -C(sigma+2, sigma), -C(sigma+3, sigma), D'(sigma+2)],
// record 0 holds [D'(0), D'(1), -, -], each as hi | lo in the K-major layout (element (r, k) =
// B[r][k], r the row of the target block, k the row of the source block).
//   forward:  C(t, s)[r][k] = sum_j Dinv_t[r][j] L(32 t + j, 32 s + k),     D'(t) = Dinv_t
//   backward: C(t, s)[r][k] = sum_j Dinv_t[j][r] L(32 s + k, 32 t + j),     D'(t) = Dinv_t^T
// (t, s block indices of the processing positions; the rows and columns past n are zero, the
// diagonal-block inverse is the identity there).
__global__ void __launch_bounds__(256) k_tc_records(int n, int b, int nblk, int ND, const float* __restrict__ Lr,
                                                    const float* __restrict__ Dinv, float* __restrict__ recF,
                                                    float* __restrict__ recB) {
    const int tau = blockIdx.x, s = blockIdx.y;
    const bool fwd = blockIdx.z == 0;
    const int nb = b + 1;
    const int Bt = fwd ? tau : nblk - 1 - tau;
    __shared__ float Dv[32][33];
    __shared__ float Lt[32][33];
    const float* Lband = Lr + (size_t)s * n * nb;
    const float* Dt = Dinv + ((size_t)s * nblk + Bt) * TC_MAT;
    float* rec = (fwd ? recF : recB) + (size_t)s * (nblk + 1) * TC_REC;
    for (int x = threadIdx.x; x < TC_MAT; x += blockDim.x) Dv[x >> 5][x & 31] = Dt[x];
    __syncthreads();
    auto L = [&](int i, int j) -> float {
        return (i < n && j >= 0 && j <= i && i - j <= b) ? Lband[(size_t)i * nb + (j - i + b)] : 0.0f;
    };
    auto put = [&](int rho, int slot, int r, int k, float v) {
        float* m = rec + (size_t)rho * TC_REC + (size_t)slot * 2 * TC_MAT;
        const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        const unsigned o = kmaj_off(r, k) / 4u;
        m[o] = h;
        m[TC_MAT + o] = v - h;
    };
    {   // D'(tau)
        const int rho = tau >= 2 ? tau - 1 : 0, slot = tau >= 2 ? 3 : tau;
        for (int x = threadIdx.x; x < TC_MAT; x += blockDim.x) {
            const int r = x >> 5, k = x & 31;
            put(rho, slot, r, k, fwd ? Dv[r][k] : Dv[k][r]);
        }
    }
    for (int u = 1; u <= ND; ++u) {
        const int sig = tau - u;
        if (sig < 0) break;
        const int Bs = fwd ? Bt - u : Bt + u;
        __syncthreads();
        // forward: Lt[j][k] = L(32 Bt + j, 32 Bs + k); backward: Lt[j][k] = L(32 Bs + k, 32 Bt + j)
        for (int x = threadIdx.x; x < TC_MAT; x += blockDim.x) {
            const int j = x >> 5, k = x & 31;
            Lt[j][k] = fwd ? L(Bt * 32 + j, Bs * 32 + k) : L(Bs * 32 + k, Bt * 32 + j);
        }
        __syncthreads();
        for (int x = threadIdx.x; x < TC_MAT; x += blockDim.x) {
            const int r = x >> 5, k = x & 31;
            float acc = 0.0f;
#pragma unroll 8
            for (int j = 0; j < 32; ++j) acc = fmaf(fwd ? Dv[r][j] : Dv[j][r], Lt[j][k], acc);
            put(sig + 1, u - 1, r, k, -acc);
        }
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------

size_t tc_smem() { return TC_SMEM; }

void launch_tc_records(fse_ctx* c, int k, cudaStream_t st) {
    const Params& p = c->p;
    const int f = k % 2;
    const size_t fsz = (size_t)p.N * p.n * (p.b + 1) * 4;
    const size_t dsz = (size_t)p.N * p.nblk * FSE_BLK * FSE_BLK * 4;
    const float* Lr = reinterpret_cast<const float*>((const char*)c->d.Lr + f * fsz);
    const float* Dv = reinterpret_cast<const float*>((const char*)c->d.Dinv + f * dsz);
    k_tc_records<<<dim3(p.nblk, p.N, 2), 256, 0, st>>>(p.n, p.b, p.nblk, p.ND, Lr, Dv, (float*)c->d.Tf,
                                                        (float*)c->d.Tb);
}

void launch_tc_solve(fse_ctx* c, int phase, cudaStream_t st) {
    const Params& p = c->p;
    static std::atomic<unsigned long long> attr{0};
    if (needs_device_setup(attr)) {
        cudaFuncSetAttribute(k_tc_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        cudaFuncSetAttribute(k_tc_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        mark_device(attr);
    }
    TcArgs A;
    A.n = p.n;
    A.ld = p.ld;
    A.nblk = p.nblk;
    A.ND = p.ND;
    A.a2c = (float)(2.0 / (2.0 * M_PI / p.S1));
    A.err = c->d.flag;
    A.X = (float*)c->d.X;
    A.V = (float*)c->d.V;
    A.Y = (float*)c->d.Y;
    dim3 g((p.ld + TC_M - 1) / TC_M, p.N);
    if (phase == 1) {
        A.rec = (const float*)c->d.Tf;
        k_tc_solve<true><<<g, TC_THREADS, TC_SMEM, st>>>(A);
    } else {
        A.rec = (const float*)c->d.Tb;
        k_tc_solve<false><<<g, TC_THREADS, TC_SMEM, st>>>(A);
    }
}

}  // namespace fse
