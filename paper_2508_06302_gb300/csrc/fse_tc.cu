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
// A[m][k] B[r][k] with M = 128 (tangent columns, TMEM lanes), K = 32 (rows of the source block)
// and N = 32 rows per target block, kind::tf32.  A (the solved block or a right-hand side, split
// hi/lo) lives in tensor memory, written by the epilogue with tcgen05.st; B (the factor couplings)
// is K-major in shared memory without swizzle.  With A in shared memory the small-N MMAs were
// bound by shared-memory bandwidth (an M = 128, K = 8 A tile is 4 KB per MMA); from tensor memory
// the tensor core reads only B there.  Eight accumulators of 32 TMEM columns rotate over the blocks (block t in columns
// 32 (t mod 8)), so the three blocks a solved block feeds are adjacent: one MMA of N = 96 pushes
// a source block into all of them (N = 32 MMAs run at a third of the tensor rate, N >= 96 at
// two thirds or more; the push splits in two where the ring wraps).  Roles: the epilogue warps
// read a finished block out of TMEM, stage it as the A operand (in TMEM), stage the
// right-hand side three blocks ahead (loaded into registers one block earlier) and store the
// block; warps 0-15 share this (thread = one column, 8 of the 32 rows of each block, so four
// warps per TMEM lane quarter), with the next block's loads in flight in register double
// buffers; warp 16 (one thread) issues the MMAs; warp 17 (one thread) streams the factor records
// with bulk copies.  After block q is read out ("round q") the MMA thread issues
//   1. the push of Y'_q into blocks q+1 .. q+ND, then commits block q+1;
//   2. the right-hand-side term Dinv'_{q+3} Y_{q+3} of block q+3.
// The accumulators are zeroed by the epilogue after each read-out, so every MMA accumulates.
// Every wait is bounded (about 2 s of SM clock); a wait that gives up raises the context's
// error flag, the CTA drains its MMAs and copies in flight, frees its tensor memory and exits.
#include <cuda_runtime.h>

#include "fse_common.cuh"

namespace fse {

constexpr int TC_M = 128;                       // tangent columns per CTA (MMA M, TMEM lanes)
constexpr int TC_MAT = FSE_BLK * FSE_BLK;       // floats of one 32 x 32 operand
constexpr int TC_CPL = 3 * TC_MAT;              // floats of the 96-row coupling operand (hi or lo)
constexpr int TC_REC = 2 * TC_CPL + 2 * TC_MAT; // floats of one record: couplings (hi, lo), D' (hi, lo)
constexpr int TC_AOP = TC_M * FSE_BLK;          // floats of one 128 x 32 A operand (hi or lo)
constexpr int TC_NREC = 3;                      // record slots in shared memory
constexpr int TC_NACC = 8;                      // accumulators of 32 TMEM columns
// shared memory holds only the record slots (both A operands live in tensor memory); the launch
// asks for more than half of an SM's shared memory so that no second CTA, which would block in
// tcgen05.alloc until this one frees its 512 TMEM columns, is placed on the same SM
constexpr unsigned TC_SMEM_USED = (unsigned)(TC_NREC * TC_REC) * 4u;
constexpr unsigned TC_SMEM = 116u * 1024u;
static_assert(TC_SMEM >= TC_SMEM_USED, "record slots exceed the launch's shared memory");
// tensor memory columns: 8 accumulators (0..255), the solved block's A operand hi | lo (256..319),
// two right-hand-side A operands hi | lo (320..447)
constexpr unsigned TC_COL_A = 32 * TC_NACC;
constexpr unsigned TC_COL_RHS = TC_COL_A + 64;
constexpr unsigned TC_TMEM_COLS = 512;
constexpr int TC_EPI = 512;                     // epilogue threads: 16 warps, four per TMEM lane quarter
constexpr int TC_THREADS = TC_EPI + 64;         // + the MMA warp and the record warp

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

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N = nrows
__host__ __device__ constexpr unsigned tc_idesc(int nrows) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(nrows >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned dtm, unsigned long long ad, unsigned long long bd, unsigned idesc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %4, p;\n}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(1), "r"(idesc)
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

// TC_HR consecutive TMEM columns of this thread's lane (warp w reads lanes 32 (w % 4) ..)
constexpr int TC_HR = 8;    // rows of a block per epilogue thread (four warps per TMEM lane quarter)
__device__ __forceinline__ void tmem_ld8(unsigned taddr, float v[TC_HR]) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// zero 8 consecutive TMEM columns of this thread's lane (completion waited for by the caller's
// tcgen05.wait::st before its next thread synchronisation)
__device__ __forceinline__ void tmem_zero8(unsigned taddr) {
    const unsigned z = 0u;
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(taddr),
                 "r"(z)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// TF32 split: hi exact in TF32 (13 low mantissa bits cleared), lo = x - hi exact in FP32
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// rows 32 B + r0 .. 32 B + r0 + 7 of column t of a tangent-sized array (zero outside)
__device__ __forceinline__ void load_rows8(const float* base, int B, int r0, int n, int ld, int t, float v[TC_HR]) {
#pragma unroll
    for (int r = 0; r < TC_HR; ++r) {
        const int i = B * FSE_BLK + r0 + r;
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

// D (nrows TMEM columns at dtm) += A B^T with A (128 x 32) in tensor memory (hi in the 32 columns
// at ahi, lo in the 32 at ahi + 32: lane m = row m, column k = K index k) and B (nrows x 32) in
// shared memory (hi at sB, lo at sB + lo_off bytes): per K step of 8, the three split products,
// small ones first
__device__ __forceinline__ void tc_mma_ts(unsigned dtm, unsigned atm, unsigned long long bd, unsigned idesc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %4, p;\n}\n" ::"r"(dtm),
        "r"(atm), "l"(bd), "r"(1), "r"(idesc)
        : "memory");
}
__device__ __forceinline__ void mma_k32(unsigned dtm, unsigned ahi, unsigned sB, unsigned lo_off, int nrows) {
    const unsigned idesc = tc_idesc(nrows);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const unsigned long long bh = tc_desc(sB + kk * 256u), bl = tc_desc(sB + lo_off + kk * 256u);
        tc_mma_ts(dtm, ahi + 32 + 8 * kk, bh, idesc);
        tc_mma_ts(dtm, ahi + 8 * kk, bl, idesc);
        tc_mma_ts(dtm, ahi + 8 * kk, bh, idesc);
    }
}

// this thread's 8 K values (rows r0 .. r0 + 7 of the block, A row m = its TMEM lane) split into hi
// and lo and written to TMEM columns col .. col + 7 (hi) and col + 32 .. (lo) of its lane (taddr =
// lane quarter + col + r0); completion is waited for by the caller's tcgen05.wait::st
__device__ __forceinline__ void tmem_stage8(unsigned taddr, const float v[TC_HR]) {
    float h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        h[j] = tf32_hi(v[j]);
        l[j] = v[j] - h[j];
    }
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
                 "f"(h[0]), "f"(h[1]), "f"(h[2]), "f"(h[3]), "f"(h[4]), "f"(h[5]), "f"(h[6]), "f"(h[7])
                 : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr + 32u),
                 "f"(l[0]), "f"(l[1]), "f"(l[2]), "f"(l[3]), "f"(l[4]), "f"(l[5]), "f"(l[6]), "f"(l[7])
                 : "memory");
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
    // A operand of the last solved block [hi | lo], staged right-hand sides [2][hi | lo], records [3]
    const unsigned sRec = smem_addr(smraw);
    float* recs = reinterpret_cast<float*>(smraw);
    const unsigned recb = (unsigned)TC_REC * 4u;
    const unsigned cpl_lo = (unsigned)TC_CPL * 4u;           // lo part of the coupling operand
    const unsigned dsl = 2u * TC_CPL * 4u, dsl_lo = (unsigned)TC_MAT * 4u;   // D' operand, its lo part
    // rhs_ready[a & 1] completes arrival a of the staged right-hand sides: a = 0 blocks 0 and 1
    // (prologue), a = 1 block 2 (prologue), a = q + 2 block q + 3 (round q).  The MMA thread waits
    // for arrival a before the epilogue can start arrival a + 2 on the same barrier.
    __shared__ __align__(8) unsigned long long acc_full[TC_NACC], rec_full[TC_NREC], epi_done, rhs_ready[2],
        rhs_free, drain;
    __shared__ unsigned s_taddr;
    __shared__ volatile int s_abort;
    const size_t base = (size_t)s * n * ld;
    float* Y = A.Y + base;
    float* X = A.X + base;
    float* V = A.V + base;
    const float* R = A.rec + (size_t)s * (nblk + 1) * TC_REC;
    auto blk = [&](int q) { return FWD ? q : nblk - 1 - q; };
    // TMEM column of the right-hand-side A operand of block t (hi; lo 32 columns further)
    auto rhs_slot = [&](int t) { return TC_COL_RHS + (unsigned)(t & 1) * 64u; };
    if (threadIdx.x == 0) {
        for (int k = 0; k < TC_NACC; ++k) mbar_init(&acc_full[k], 1);
        for (int k = 0; k < TC_NREC; ++k) mbar_init(&rec_full[k], 1);
        mbar_init(&epi_done, TC_EPI);
        mbar_init(&rhs_ready[0], TC_EPI);
        mbar_init(&rhs_ready[1], TC_EPI);
        mbar_init(&rhs_free, 1);
        mbar_init(&drain, 1);
        s_abort = 0;
        mbar_fence_init();
    }
    if (warp == 16) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&s_taddr)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tbase = s_taddr;

    if (warp < 16) {
        // ---------------- epilogue: thread (warp w, lane l) = column t0 + m, m = 32 (w % 4) + l (TMEM
        // lane m), rows r0 .. r0 + 7 of each block, r0 = 8 (w / 4)
        const int m = (warp & 3) * 32 + lane, r0 = (warp >> 2) * TC_HR, t = t0 + m;
        const int t0w = t0 + (warp & 3) * 32;
        const bool pf = warp < 4;                  // one warp of each lane quarter issues the L2 prefetches
        const unsigned tl = tbase + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)r0;
        for (int a = 0; a < TC_NACC; ++a) tmem_zero8(tl + a * 32);
        tmem_wait_st();
        // register double buffers: right-hand side three blocks ahead, backward X_k and V_k of the block
        float rA[TC_HR], rB[TC_HR], xA[TC_HR], xB[TC_HR], vA[TC_HR], vB[TC_HR];
        load_rows8(Y, blk(0), r0, n, ld, t, rA);
        tmem_stage8(tl + rhs_slot(0), rA);
        if (nblk > 1) {
            load_rows8(Y, blk(1), r0, n, ld, t, rA);
            tmem_stage8(tl + rhs_slot(1), rA);
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&rhs_ready[0]);                       // arrival 0
        if (nblk > 2) load_rows8(Y, blk(2), r0, n, ld, t, rA);
        if (pf) {
            for (int q = 3; q < 6 && q < nblk; ++q) prefetch_rows32(Y, blk(q), n, ld, t0w);
            if (!FWD)
                for (int q = 0; q < 3 && q < nblk; ++q) {
                    prefetch_rows32(X, blk(q), n, ld, t0w);
                    prefetch_rows32(V, blk(q), n, ld, t0w);
                }
        }
        // block 2's right-hand side goes into slot 0 once the MMAs of blocks 0 and 1 have read it
        if (!mbar_wait(&rhs_free, 0, A.err)) s_abort = 1;
        tc_fence_after();
        if (nblk > 2) tmem_stage8(tl + rhs_slot(2), rA);
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&rhs_ready[1]);                       // arrival 1
        if (nblk > 3) load_rows8(Y, blk(3), r0, n, ld, t, rA);
        if (!FWD) {
            load_rows8(X, blk(0), r0, n, ld, t, xA);
            load_rows8(V, blk(0), r0, n, ld, t, vA);
        }
        // one block: rc holds the right-hand side of block q + 3 and xc, vc the backward X_k, V_k of
        // block q; the next block's are loaded into rn, xn, vn here and used one block later
        auto round = [&](int q, float (&rc)[TC_HR], float (&rn)[TC_HR], float (&xc)[TC_HR], float (&vc)[TC_HR],
                         float (&xn)[TC_HR], float (&vn)[TC_HR]) -> bool {
            const int B = blk(q);
            if (q + 4 < nblk) load_rows8(Y, blk(q + 4), r0, n, ld, t, rn);
            if (pf && q + 6 < nblk) prefetch_rows32(Y, blk(q + 6), n, ld, t0w);
            if (!FWD && q + 1 < nblk) {
                if (pf && q + 3 < nblk) {
                    prefetch_rows32(X, blk(q + 3), n, ld, t0w);
                    prefetch_rows32(V, blk(q + 3), n, ld, t0w);
                }
                load_rows8(X, blk(q + 1), r0, n, ld, t, xn);
                load_rows8(V, blk(q + 1), r0, n, ld, t, vn);
            }
            if (s_abort || !mbar_wait(&acc_full[q & 7], (q >> 3) & 1, A.err)) {
                s_abort = 1;
                return false;
            }
            tc_fence_after();
            float y[TC_HR];
            tmem_ld8(tl + (q & 7) * 32, y);
            tmem_stage8(tl + TC_COL_A, y);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&epi_done);
            // off the critical path: zero the accumulator for block q + 8, stage the right-hand side of
            // block q + 3 (its slot's previous block, q + 1, was read by round q - 2, finished before
            // block q was committed)
            tmem_zero8(tl + (q & 7) * 32);
            if (q + 3 < nblk) tmem_stage8(tl + rhs_slot(q + 3), rc);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&rhs_ready[q & 1]);               // arrival q + 2
            if (t < ld) {
#pragma unroll
                for (int r = 0; r < TC_HR; ++r) {
                    const int i = B * FSE_BLK + r0 + r;
                    if (i < n) {
                        const size_t o = (size_t)i * ld + t;
                        if (FWD) {
                            __stcs(Y + o, y[r]);
                        } else {
                            __stcs(X + o, y[r]);
                            __stcs(V + o, A.a2c * (y[r] - xc[r]) - vc[r]);
                        }
                    }
                }
            }
            return true;
        };
        for (int q = 0; q < nblk; q += 2) {
            if (!round(q, rA, rB, xA, vA, xB, vB)) break;
            if (q + 1 < nblk && !round(q + 1, rB, rA, xB, vB, xA, vA)) break;
        }
    } else if (warp == 16) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            bool ok = mbar_wait(&rec_full[0], 0, A.err) && mbar_wait(&rhs_ready[0], 0, A.err);
            if (ok) {
                // prologue: right-hand-side terms of blocks 0, 1 (slots 0, 1), then 2 (slot 0 again);
                // record 0 holds D'_0, D'_1, D'_2 as rows 0-31, 32-63, 64-95 of its coupling operand
                tc_fence_after();
                mma_k32(tbase + 0, tbase + rhs_slot(0), sRec, cpl_lo, 32);
                if (nblk > 1) mma_k32(tbase + 32, tbase + rhs_slot(1), sRec + 4096u, cpl_lo, 32);
                tc_commit(&rhs_free);
                ok = mbar_wait(&rhs_ready[1], 0, A.err);
                if (ok) {
                    tc_fence_after();
                    if (nblk > 2) mma_k32(tbase + 64, tbase + rhs_slot(2), sRec + 8192u, cpl_lo, 32);
                    tc_commit(&acc_full[0]);
                }
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
                const unsigned sB = sRec + (unsigned)rs * recb;
                // record q + 1: couplings C(q+1, q), C(q+2, q), C(q+3, q) as rows 0-95, then D'(q+3)
                const int nt = min(ND, nblk - 1 - q);          // blocks this one feeds
                if (nt > 0) {
                    const int a0 = (q + 1) & 7, n1 = min(nt, TC_NACC - a0);
                    mma_k32(tbase + a0 * 32, tbase + TC_COL_A, sB, cpl_lo, 32 * n1);
                    if (n1 < nt) mma_k32(tbase, tbase + TC_COL_A, sB + (unsigned)n1 * 4096u, cpl_lo, 32 * (nt - n1));
                }
                tc_commit(&acc_full[(q + 1) & 7]);
                // arrival q + 2: the right-hand side of block q + 3 is staged
                if (!mbar_wait(&rhs_ready[q & 1], ((q + 2) >> 1) & 1, A.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (q + 3 < nblk) mma_k32(tbase + ((q + 3) & 7) * 32, tbase + rhs_slot(q + 3), sB + dsl, dsl_lo, 32);
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
            // record q + 3 (round q + 2) replaces record q (round q - 1) once block q + 1 is committed:
            // that commit follows every MMA of round q - 1
            for (int q = 0; q + 3 < nblk; ++q) {
                if (s_abort || !mbar_wait(&acc_full[(q + 1) & 7], ((q + 1) >> 3) & 1, A.err)) {
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
    if (warp == 16)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TC_TMEM_COLS)
                     : "memory");
}

// Factor records of both directions for the tensor-core solves, one CTA per (target block in
// processing order tau, trajectory, direction).  Processing order: forward blocks 0, 1, ..;
// backward blocks nblk-1, nblk-2, ...  Record sigma + 1 holds the B operands of round sigma: the
// 96-row coupling operand [-C(sigma+1, sigma); -C(sigma+2, sigma); -C(sigma+3, sigma)] and
// D'(sigma+3); record 0 holds [D'(0); D'(1); D'(2)] in its coupling operand.  Each operand as
// hi | lo in the K-major layout (element (r, k) = B[r][k], r the row of the target block, k the
// row of the source block).
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
    // element (r, k) of an operand whose hi part starts at float offset o0 (lo at o0 + lo)
    auto put = [&](size_t o0, size_t lo, int r, int k, float v) {
        const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        const size_t o = o0 + kmaj_off(r, k) / 4u;
        rec[o] = h;
        rec[o + lo] = v - h;
    };
    {   // D'(tau): record 0 rows 32 tau.. of the coupling operand (tau <= 2), else record tau - 2's D'
        for (int x = threadIdx.x; x < TC_MAT; x += blockDim.x) {
            const int r = x >> 5, k = x & 31;
            const float v = fwd ? Dv[r][k] : Dv[k][r];
            if (tau <= 2)
                put(0, TC_CPL, 32 * tau + r, k, v);
            else
                put((size_t)(tau - 2) * TC_REC + 2 * TC_CPL, TC_MAT, r, k, v);
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
            put((size_t)(sig + 1) * TC_REC, TC_CPL, 32 * (u - 1) + r, k, -acc);
        }
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------

// floats of one record buffer (one direction, one step parity)
static size_t tc_records_floats(const Params& p) { return (size_t)p.N * (p.nblk + 1) * TC_REC; }

void launch_tc_records(fse_ctx* c, int k, cudaStream_t st) {
    const Params& p = c->p;
    const int f = k % 2;
    const size_t fsz = (size_t)p.N * p.n * (p.b + 1) * 4;
    const size_t dsz = (size_t)p.N * p.nblk * FSE_BLK * FSE_BLK * 4;
    const float* Lr = reinterpret_cast<const float*>((const char*)c->d.Lr + f * fsz);
    const float* Dv = reinterpret_cast<const float*>((const char*)c->d.Dinv + f * dsz);
    const size_t ro = (size_t)f * tc_records_floats(p);
    k_tc_records<<<dim3(p.nblk, p.N, 2), 256, 0, st>>>(p.n, p.b, p.nblk, p.ND, Lr, Dv, (float*)c->d.Tf + ro,
                                                        (float*)c->d.Tb + ro);
}

void launch_tc_solve(fse_ctx* c, int k, int phase, cudaStream_t st) {
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
    const size_t ro = (size_t)(k % 2) * tc_records_floats(p);
    if (phase == 1) {
        A.rec = (const float*)c->d.Tf + ro;
        k_tc_solve<true><<<g, TC_THREADS, TC_SMEM, st>>>(A);
    } else {
        A.rec = (const float*)c->d.Tb + ro;
        k_tc_solve<false><<<g, TC_THREADS, TC_SMEM, st>>>(A);
    }
}

}  // namespace fse
