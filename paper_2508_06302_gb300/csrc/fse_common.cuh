// Device helpers shared by the FSE-Shooting kernels.
#pragma once

#include <cuda_runtime.h>

#include "fse_internal.h"

namespace fse {

// 5-point Gauss-Legendre nodes on [-1, 1] and weights (exact for the von Karman element
// integrands); filled by ensure_constants() of the translation unit that evaluates elements
static __constant__ double c_glx[5];
static __constant__ double c_glw[5];

__device__ __forceinline__ double qval(const double* q, int g) { return g >= 0 ? q[g] : 0.0; }

// slope of the Hermite cubic (w1, th1, w2, th2) at xi in [-1, 1] of an element of length L
__device__ __forceinline__ void vk_slope(double xi, double L, double Nd[4]) {
    const double s = 0.5 * (xi + 1.0);
    Nd[0] = (-6.0 * s + 6.0 * s * s) / L;
    Nd[1] = 1.0 - 4.0 * s + 3.0 * s * s;
    Nd[2] = (6.0 * s - 6.0 * s * s) / L;
    Nd[3] = -2.0 * s + 3.0 * s * s;
}

__device__ __forceinline__ int elem_ndof(int type) {
    return (type == FSE_NL_CUBIC_GROUND || type == FSE_NL_VDP) ? 1 : (type == FSE_NL_CUBIC_DIFF ? 2 : 6);
}

// Element force fe[6] (local dof order) and, if ke != nullptr, its tangent ke[36] = d fe / d q
// and, if ce != nullptr, its velocity tangent ce[36] = d fe / d qdot of the nonlinear elements of
// Eq. (1): cubic springs, the von Karman beam (gradient of EA/2 int (u' w'^2 + w'^4/4) dx,
// 5-point Gauss-Legendre) and the self-excited damper f = p0 (q^2 - 1) qdot.  qd holds the
// physical velocities qdot = w_1 u of the dofs (nullptr: zero).
__device__ inline void elem_eval(int type, const int* dof, const double* p, const double* q, const double* qd,
                                 double fe[6], double* ke, double* ce = nullptr) {
    for (int a = 0; a < 6; ++a) fe[a] = 0.0;
    if (ke)
        for (int a = 0; a < 36; ++a) ke[a] = 0.0;
    if (ce)
        for (int a = 0; a < 36; ++a) ce[a] = 0.0;
    if (type == FSE_NL_VDP) {
        const double x = qval(q, dof[0]), v = qd ? qval(qd, dof[0]) : 0.0;
        fe[0] = p[0] * (x * x - 1.0) * v;
        if (ke) ke[0] = 2.0 * p[0] * x * v;
        if (ce) ce[0] = p[0] * (x * x - 1.0);
    } else if (type == FSE_NL_CUBIC_GROUND) {
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

// y_i = sum_e val[e] x[col[e]] over CSR row i (FP64)
__device__ __forceinline__ double csr_row(const int* __restrict__ ptr, const int* __restrict__ col,
                                          const double* __restrict__ val, int i, const double* x) {
    double acc = 0.0;
    const int e1 = ptr[i + 1];
    for (int e = ptr[i]; e < e1; ++e) acc += val[e] * x[col[e]];
    return acc;
}

// max that propagates NaN from either argument (fmax drops it), so that a non-finite
// value anywhere reaches the convergence test
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

// Block-wide max reduction of two values (blockDim.x multiple of 32, <= 1024), NaN-propagating.
__device__ __forceinline__ void block_max2(double& a, double& b) {
    __shared__ double ra[32], rb[32];
    for (int o = 16; o > 0; o >>= 1) {
        a = nanmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = nanmax(b, __shfl_xor_sync(0xffffffffu, b, o));
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
        a = nanmax(a, ra[k]);
        b = nanmax(b, rb[k]);
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
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
// asynchronous global -> shared copy of one element (4 or 8 bytes)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"((int)sizeof(T)));
}

// ---- mbarrier / bulk-copy helpers (every wait is bounded: after about 2 s of SM clock the
// waiting thread raises the error flag and gives up)
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned tx) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_addr(bar)),
                 "r"(tx)
                 : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
    const unsigned a = smem_addr(bar);
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1ll << 32)) {
            atomicExch(err, 1);
            return false;
        }
    }
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// 3-D tiled TMA load (box of the tensor map at {x, y, z}) completing on bar; the shared
// destination is 128-byte aligned and x * element size a multiple of 16 bytes
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}


// grid of a grid-stride loop: enough blocks for `total` items, at most per_sm blocks per SM
static inline int nblocks(size_t total, int bs, int per_sm = 16) {
    size_t g = (total + bs - 1) / bs;
    const size_t cap = (size_t)num_sms() * per_sm;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace fse
