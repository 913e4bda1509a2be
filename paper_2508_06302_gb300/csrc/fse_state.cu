// Trajectory state path of FSE-Shooting (App. E): one CTA per trajectory per
// Newmark step; FP64 state, residual and Newton test; factor of the effective
// stiffness in the sensitivity precision T.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "fse_common.cuh"

namespace fse {

static std::atomic<unsigned long long> g_const_ready{0};   // per device (bit = device id)

void ensure_constants() {
    if (!needs_device_setup(g_const_ready)) return;
    // closed forms of the 5-point Gauss-Legendre rule
    const double r = 2.0 * sqrt(10.0 / 7.0);
    double x[5] = {-sqrt(5.0 + r) / 3.0, -sqrt(5.0 - r) / 3.0, 0.0, sqrt(5.0 - r) / 3.0,
                   sqrt(5.0 + r) / 3.0};
    const double s70 = 13.0 * sqrt(70.0);
    double w[5] = {(322.0 - s70) / 900.0, (322.0 + s70) / 900.0, 128.0 / 225.0,
                   (322.0 + s70) / 900.0, (322.0 - s70) / 900.0};
    cudaMemcpyToSymbol(c_glx, x, sizeof(x));
    cudaMemcpyToSymbol(c_glw, w, sizeof(w));
    mark_device(g_const_ready);
}

// ----------------------------------------------------------------------------
// AFT tables (App. D, Eq. 14) and per-w_1 operators
// ----------------------------------------------------------------------------

// (the sums over samples of Eq. D3 are normalised by the whole grid's Nglob; a trajectory shard
// holds its own N columns of Gamma^-1)
__global__ void k_tables(int N, int Nglob, int U, int dm1, const int* __restrict__ ktab,
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
        Gi[(size_t)c * N + s] = (c == 0 ? 1.0 : 2.0) * g / (double)Nglob;
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

// S = w^2 4/D^2 M + w 2/D D + K (Eq. E7) in FP64, and the two operators of the
// sensitivity right-hand side A = w^2 4/D^2 M + w 2/D D - K and B = w^2 4/D M.
template <typename T>
__global__ void k_build_ops(int nnz, double cm, double cd, double cb, const double* m,
                            const double* d, const double* k, double* S, T* Aop, T* Bop) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
        S[e] = cm * m[e] + cd * d[e] + k[e];
        Aop[e] = T(cm * m[e] + cd * d[e] - k[e]);
        Bop[e] = T(cb * m[e]);
    }
}

// lower column band of S in FP32 for the panel factor: Sband[j (b + 1) + i - j] = S_ij, i >= j (zero
// elsewhere: the caller clears it first); one thread per row
__global__ void k_sband(int n, int nb, const int* __restrict__ ptr, const int* __restrict__ col,
                        const double* __restrict__ S, float* Sband) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
            const int j = col[e];
            if (j <= i) Sband[(size_t)j * nb + (i - j)] = float(S[e]);
        }
}

// ----------------------------------------------------------------------------
// banded Cholesky inside one CTA: column band Ac (global, in place) -> Lc, Lr, Linv
// ----------------------------------------------------------------------------

// columns of the band staged ahead of the Cholesky window (cp.async ring)
#define FSE_CHOL_PF 8

// Banded Cholesky with a warp-cooperative trailing update.  The window holds the nb columns
// j..j+b in nb + 1 shared slots (column c in slot c mod (nb + 1)).  Step j, between two barriers:
//  (a) threads r < nb write column j - 1 of L out of its slot, refill that slot with column
//      j + nb from the cp.async staging ring (entry r was staged by thread r) and stage
//      column j + nb + PF - 1;
//  (b) warp w updates columns j + cc, cc = w + 1, w + 1 + 8, ..., with lanes over the rows:
//      A_(j+cc+rr, j+cc) -= A_(j+cc+rr, j) A_(j+cc, j) / A_(j, j), rr <= b - cc.
// (a) and (b) touch different slots, so one barrier per column suffices.
template <typename T>
__device__ int cta_band_cholesky_w(T* Ac, T* Lr, T* Linv, int n, int b, T* wnd, T* stg, T* Rf, T* Rb, int RECE) {
    constexpr int PF = FSE_CHOL_PF;
    const int nb = b + 1, ns = nb + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
        const int c = idx / nb;   // column c starts in slot c
        wnd[idx] = (c < n) ? Ac[(size_t)c * nb + (idx - c * nb)] : T(0);
    }
    auto issue = [&](int col) {   // thread tid < nb stages entry tid of column col
        if (col < n) cp_async_elem(stg + (col % PF) * nb + tid, Ac + (size_t)col * nb + tid);
        cp_async_commit();
    };
    if (tid < nb)
        for (int c = 0; c < PF - 1; ++c) issue(nb + c);
    // write column jp of L (its pivot 1/L_jj = inv, L_jj = ljj) from slot colp; thread r < nb
    auto write_col = [&](int jp, const T* colp, T ljj, T inv) {
        const int r = tid;
        const T v = (jp + r < n) ? (r == 0 ? ljj : colp[r] * inv) : T(0);
        Ac[(size_t)jp * nb + r] = v;
        if (jp + r < n) {
            const int i = jp + r;
            Lr[(size_t)i * nb + (b - r)] = v;
            if (Rf) {
                const int i0 = i & ~(FSE_BLK - 1);
                if (jp < i0) Rf[(size_t)(i >> 5) * RECE + (jp - i0 + b) * FSE_BLK + (i - i0)] = v;
                const int j0 = jp & ~(FSE_BLK - 1), cbk = i - j0 - FSE_BLK;
                if (cbk >= 0) Rb[(size_t)(jp >> 5) * RECE + cbk * FSE_BLK + (jp - j0)] = v;
            }
        }
        if (r == 0) {
            Linv[jp] = inv;
            for (int c = 0; c < b - jp; ++c) Lr[(size_t)jp * nb + c] = T(0);
        }
    };
    __syncthreads();
    T ljj_prev = T(0), inv_prev = T(0);
    int slot = 0;   // slot of column j
    int j = 0;
    for (; j < n; ++j) {
        const T* colj = wnd + slot * nb;
        const T piv = colj[0];
        if (!(piv > T(0)) || !isfinite((double)piv)) {
            if (tid == 0) bad = 1;
            break;
        }
        const T ljj = sqrt(piv);
        const T inv = T(1) / ljj;
        const T inv2 = inv * inv;
        const int sp = (slot == 0) ? ns - 1 : slot - 1;   // slot of column j - 1 = slot of column j + nb
        if (tid < nb) {
            T* colp = wnd + sp * nb;
            if (j > 0) write_col(j - 1, colp, ljj_prev, inv_prev);
            cp_async_wait<PF - 2>();   // entry tid of column j + nb has landed
            const int jn = j + nb;
            colp[tid] = (jn < n) ? stg[(jn % PF) * nb + tid] : T(0);
            issue(jn + PF - 1);        // into the staging slot just read
        }
        for (int cc = warp + 1; cc <= b; cc += nw) {
            if (j + cc >= n) break;
            int sc = slot + cc;
            sc = (sc >= ns) ? sc - ns : sc;
            T* colc = wnd + sc * nb;
            const T g = colj[cc] * inv2;
            for (int rr = lane; rr <= b - cc; rr += 32) colc[rr] -= colj[cc + rr] * g;
        }
        __syncthreads();
        ljj_prev = ljj;
        inv_prev = inv;
        slot = (slot + 1 == ns) ? 0 : slot + 1;
    }
    if (j == n && tid < nb) write_col(n - 1, wnd + ((slot == 0) ? ns - 1 : slot - 1) * nb, ljj_prev, inv_prev);
    cp_async_wait<0>();
    __syncthreads();
    return bad;
}

// Banded Cholesky with the window in registers (b + 1 <= 32 MAXK, nb <= 8 MAXS): warp w owns
// window slots s = w, w + 8, ... (column c in slot c mod nb) and lane l the rows l + 32k of
// them.  Step j: the owner warp of column j publishes it to a shared buffer (two, alternating),
// one barrier, then every warp applies A_(c+rr, c) -= A_(c+rr, j) A_(c, j) / A_(j, j) to its
// slots c = j + cc from that read-only buffer, threads < nb write column j of L out, and the
// owner warp of slot j takes column j + nb from the cp.async staging ring.  Every warp has the
// same work per step and the window never aliases the buffer it reads.
template <typename T, int MAXS, int MAXK>
__device__ int cta_band_cholesky_r(T* Ac, T* Lr, T* Linv, int n, int b, T* colbuf, T* stg, T* Rf, T* Rb,
                                   int RECE) {
    constexpr int PF = FSE_CHOL_PF;
    const int nb = b + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    T val[MAXS][MAXK];
    int cc[MAXS];   // slot q holds column j + cc[q] (cc = 0: column j itself)
#pragma unroll
    for (int q = 0; q < MAXS; ++q) {
        const int sl = warp + 8 * q;   // column sl at the start
        cc[q] = sl < nb ? sl : -(1 << 28);   // slots past the window never become active
#pragma unroll
        for (int k = 0; k < MAXK; ++k) {
            const int rr = lane + 32 * k;
            val[q][k] = (sl < nb && sl < n && rr < nb) ? Ac[(size_t)sl * nb + rr] : T(0);
        }
    }
    auto issue = [&](int col) {   // thread tid < nb stages entry tid of column col
        if (col < n) cp_async_elem(stg + (col % PF) * nb + tid, Ac + (size_t)col * nb + tid);
        cp_async_commit();
    };
    if (tid < nb)
        for (int c = 0; c < PF - 1; ++c) issue(nb + c);
    const unsigned sbuf = (unsigned)__cvta_generic_to_shared(colbuf);
    int slot = 0;   // window slot of column j (= j mod nb)
    for (int j = 0; j < n; ++j, slot = (slot + 1 == nb) ? 0 : slot + 1) {
        T* cb = colbuf + (j & 1) * nb;
        const int ow = slot & 7, oq = slot >> 3;   // owner warp and its slot index
        if (warp == ow) {
#pragma unroll
            for (int q = 0; q < MAXS; ++q)
                if (q == oq) {
#pragma unroll
                    for (int k = 0; k < MAXK; ++k)
                        if (lane + 32 * k < nb) cb[lane + 32 * k] = val[q][k];
                }
        }
        if (tid < nb) cp_async_wait<PF - 2>();   // entry tid of column j + nb has landed
        __syncthreads();
        if (tid < nb) issue(j + nb + PF - 1);     // into the staging slot read at step j - 1
        const T piv = cb[0];
        if (!(piv > T(0)) || !(piv < T(INFINITY))) {
            if (tid == 0) bad = 1;
            break;
        }
        const T inv = rsqrtf(piv);   // 1 / L_jj (FP32 factor: refined by the FP64 residual)
        const T ljj = piv * inv;
        const T inv2 = inv * inv;
        const unsigned cbs = sbuf + (unsigned)((j & 1) * nb) * 4u;
#pragma unroll
        for (int q = 0; q < MAXS; ++q) {
            const int c = cc[q];
            if (c >= 1 && c <= b && j + c < n) {
                const unsigned a = cbs + (unsigned)(c + lane) * 4u;   // cb[c + lane]
                T g;
                asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(g) : "r"(cbs + (unsigned)c * 4u));
                g *= inv2;
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    if (lane + 32 * k <= b - c) {
                        T x;
                        asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(x) : "r"(a + 128u * k));
                        val[q][k] -= x * g;
                    }
                }
            }
            cc[q] = (c == 0) ? b : c - 1;   // next step: column j + 1 + cc
        }
        if (tid < nb) {   // column j of L
            const int r = tid;
            const T v = (j + r < n) ? (r == 0 ? ljj : cb[r] * inv) : T(0);
            Ac[(size_t)j * nb + r] = v;
            if (j + r < n) {
                const int i = j + r;
                Lr[(size_t)i * nb + (b - r)] = v;
                if (Rf) {
                    const int i0 = i & ~(FSE_BLK - 1);
                    if (j < i0) Rf[(size_t)(i >> 5) * RECE + (j - i0 + b) * FSE_BLK + (i - i0)] = v;
                    const int j0 = j & ~(FSE_BLK - 1), cbk = i - j0 - FSE_BLK;
                    if (cbk >= 0) Rb[(size_t)(j >> 5) * RECE + cbk * FSE_BLK + (j - j0)] = v;
                }
            }
            if (r == 0) {
                Linv[j] = inv;
                for (int c = 0; c < b - j; ++c) Lr[(size_t)j * nb + c] = T(0);
            }
        }
        if (warp == ow) {   // slot j takes column j + nb
            const int jn = j + nb;
#pragma unroll
            for (int q = 0; q < MAXS; ++q)
                if (q == oq) {
#pragma unroll
                    for (int k = 0; k < MAXK; ++k) {
                        const int rr = lane + 32 * k;
                        if (rr < nb) val[q][k] = (jn < n) ? stg[(jn % PF) * nb + rr] : T(0);
                    }
                }
        }
    }
    if (tid < nb) cp_async_wait<0>();
    __syncthreads();
    return bad;
}

// Panel (blocked, right-looking) banded Cholesky for FP32 factors, b <= 96, 256 threads.
// K_eff = L L^T is factored by panels of 32 columns j0 .. j0 + 31:
//   [L11; L21] = the panel's columns, factored column by column: L11 = chol(A11) for the
//                32 x 32 diagonal block and L21 = A21 L11^-T for the rows j0 + 32 .. j0 + 31 + b
//   A22 -= L21 L21^T   the trailing band
// The panel is factored by warps 0-4 without a barrier: each factors its own copy of the
// diagonal block through shuffles and sweeps one row of its own with the same column operations
// (the rows below the block; for warp 4, rows that start as the identity and end as the columns
// of L11^-1, the diagonal-block inverse the tangent solves use: x L11^T = e_c gives x = column c
// of L11^-1).  The trailing update (4 x 4 register tiles, all warps) and two CTA barriers come
// once per panel, against one barrier per column in the unblocked form.  Warps 5-7 write the
// previous panel's columns of L out (column band, row band, Linv, block inverse and the tangent-
// solve records) while the panel is factored; warps 4-7 then stage the columns that the next panel
// updates first, as the band of S (one FP32 copy for all trajectories) plus the trajectory's K_t
// and C_t entries of those columns: K_eff is never assembled in global memory.
// Shared workspace (floats): a ring of CHB_R columns of the band (column c in slot c mod CHB_R,
// entry c + r at r), L21 transposed [32][CHB_RP], L11^-1 of two panels [2][32][33], 1/L_jj of
// two panels, per panel warp two buffers of the current column of L11.
constexpr int CHB_R = 160;    // >= b + 64 columns are live at once
constexpr int CHB_RP = 100;   // row pitch of the transposed L21 (>= b, a multiple of 4)
__host__ __device__ constexpr size_t chol_blk_floats(int nb) {
    return (size_t)CHB_R * nb + 32 * CHB_RP + 2 * 32 * 33 + 64 + 5 * 64;
}

// where the panel factor takes K_eff = S + K_t + w (2/Delta) C_t from: the lower band of S (FP32,
// all trajectories), the lower K_t entries by column, this trajectory's K_t and C_t values
// (ct null without velocity-dependent elements) and w (2/Delta)
struct ChbSource {
    const float* Sband;
    const int *ktc_ptr, *ktc_e, *ktc_c, *ktc_r;
    const float *kt, *ct;
    float wa;
};

// column c of the ring: W + (c mod CHB_R) nb
__device__ __forceinline__ float* chb_col(float* W, int c, int nb) { return W + (size_t)(c % CHB_R) * nb; }

// The panel factor and the trailing update are separate (not inlined) functions: inlined into the
// panel loop, their 32-entry register arrays were kept in local memory.
//
// Panel at column j0 (threads 0-159, five warps, no barrier): every warp factors its own copy of
// the diagonal block (lane i: row j0 + i, the identity past n) with shuffles, and applies the
// same column operations to one row of its own: warps 1-3 the rows j0 + 32 .. j0 + 127 below the
// block (rows past j0 + 31 + nr are zero), warp 4 the identity rows that become the columns of
// L11^-1.  li[k] gets 1 / L_kk; L goes back into the ring, L21 transposed into P, L11^-1 into
// Zo[i * 33 + c].  Returns false (warp 0) on a non-positive or non-finite pivot.  (Forming the
// pivots once and sharing each column through shared memory and a barrier per column measured
// 3-4x slower: the barrier chain set the pace.)
__device__ __noinline__ bool chb_panel(int W_o, int li_o, int P_o, int Zo_o, int cb_o, int j0, int jb, int nr, int b,
                                       int nb) {
    extern __shared__ float chb_dyn[];   // the kernel's dynamic shared memory: plain shared loads and stores
    float *W = chb_dyn + W_o, *li = chb_dyn + li_o, *P = chb_dyn + P_o, *Zo = chb_dyn + Zo_o;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    float* cbw = chb_dyn + cb_o + w * 64;   // this warp's two buffers for the current column of L11
    const int ib = 32 * (w - 1) + lane;   // warps 1-3: row j0 + 32 + ib
    const bool below = w >= 1 && w <= 3 && ib < nr, ident = w == 4;
    float d[32], a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        d[k] = (k <= lane && lane < jb && lane - k <= b) ? chb_col(W, j0 + k, nb)[lane - k] : (k == lane ? 1.f : 0.f);
        a[k] = below ? ((32 + ib - k <= b) ? chb_col(W, j0 + k, nb)[32 + ib - k] : 0.f) : ((ident && k == lane) ? 1.f : 0.f);
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float piv = __shfl_sync(0xffffffffu, d[k], k);
        ok = ok && (piv > 0.f) && (piv < INFINITY);
        const float inv = rsqrtf(piv);   // 1 / L_kk (FP32 factor: refined by the FP64 residual)
        const float lk = (lane == k) ? piv * inv : (lane > k ? d[k] * inv : 0.f);
        d[k] = lk;
        a[k] *= inv;
        if (w == 0 && lane == k) li[k] = inv;
        // column k goes through the warp's buffer (k & 1) and comes back as broadcast 16-byte
        // loads: a quarter of the shared-memory operations of one shuffle per entry.  The
        // buffer written at step k + 1 was last read at step k - 1, before this __syncwarp.
        float* cbk = cbw + (k & 1) * 32;
        cbk[lane] = lk;
        __syncwarp();
        const float4* c4 = reinterpret_cast<const float4*>(cbk);
#pragma unroll
        for (int g = (k + 1) / 4; g < 8; ++g) {
            const float4 v = c4[g];   // L(j0 + 4g .. j0 + 4g + 3, j0 + k)
            const float lv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int m = 4 * g + u;
                if (m > k) {
                    d[m] = fmaf(-lk, lv[u], d[m]);
                    a[m] = fmaf(-a[k], lv[u], a[m]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (w == 0) {
            if (k <= lane && lane < jb && lane - k <= b) chb_col(W, j0 + k, nb)[lane - k] = d[k];
        } else if (below) {
            if (32 + ib - k <= b) chb_col(W, j0 + k, nb)[32 + ib - k] = a[k];
            P[k * CHB_RP + ib] = a[k];
        } else if (ident) {
            Zo[k * 33 + lane] = a[k];
        }
    }
    return ok;
}

// A22 -= L21 L21^T over the nr x nr lower triangle of the trailing band: 4 x 4 tiles (ti, tc),
// tc <= ti, tiles t = tid, tid + 256, ...
__device__ __noinline__ void chb_update(int W_o, int P_o, int j0, int nr, int nb) {
    extern __shared__ float chb_dyn[];
    float* W = chb_dyn + W_o;
    const float* P = chb_dyn + P_o;
    const int nt4 = (nr + 3) >> 2, ntile = nt4 * (nt4 + 1) / 2;
    for (int t = threadIdx.x; t < ntile; t += 256) {
        int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
        while (ti * (ti + 1) / 2 > t) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        const int tc = t - ti * (ti + 1) / 2;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const float4 x = *reinterpret_cast<const float4*>(P + k * CHB_RP + 4 * ti);
            const float4 y = *reinterpret_cast<const float4*>(P + k * CHB_RP + 4 * tc);
            const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u], yv[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int ii = 4 * ti + u, cc = 4 * tc + v;
                if (ii < nr && cc <= ii) chb_col(W, j0 + 32 + cc, nb)[ii - cc] -= acc[u][v];
            }
    }
}

__device__ int cta_band_cholesky_blk(float* Ac, float* Lr, float* Linv, float* Dinv, int n, int b, float* ws,
                                     float* Rf, float* Rb, int RECE, bool full, const ChbSource& src) {
    const int nb = b + 1;
    const int tid = threadIdx.x, warp = tid >> 5;
    float* W = ws;
    float* P = W + (size_t)CHB_R * nb;   // P[k * CHB_RP + i'] = L(j0 + 32 + i', j0 + k)
    float* Z = P + 32 * CHB_RP;          // panel q: Z[(q & 1) * 1056 + i * 33 + c] = (L11^-1)(i, c)
    float* Li = Z + 2 * 32 * 33;         // 1/L_jj of panels of even / odd index
    float* cb = Li + 64;                 // per panel warp, two buffers of the current column of L11
    // offsets (floats) of the workspace parts in the dynamic shared memory, for the panel bodies
    extern __shared__ float chb_dyn[];
    const int o_W = (int)(W - chb_dyn), o_P = (int)(P - chb_dyn), o_Z = (int)(Z - chb_dyn), o_Li = (int)(Li - chb_dyn),
              o_cb = (int)(cb - chb_dyn);
    __shared__ int bad;
    if (tid == 0) bad = 0;
    // rows i < b of the row band have no columns j < 0
    for (int idx = tid; full && idx < min(b, n) * b; idx += 256) {
        const int i = idx / b, c = idx - i * b;
        if (c < b - i) Lr[(size_t)i * nb + c] = 0.f;
    }
    // columns [c0, c1) of K_eff into the ring (zero past n): the band of S, then this trajectory's
    // K_t (and C_t) entries of those columns; threads t0 .. t0 + nthr - 1, either the whole CTA or
    // warps 4-7, which synchronise on named barrier 1 between the two
    auto stage = [&](int c0, int c1, int t0, int nthr) {
        const int cnt = max(0, c1 - c0) * nb;
        const float* g = src.Sband + (size_t)c0 * nb;
        for (int base = tid - t0; base < cnt; base += 4 * nthr) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * nthr;
                v[u] = idx < cnt ? g[idx] : 0.f;   // entries past row n are zero in the band of S
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * nthr;
                if (idx < cnt) {
                    const int q = idx / nb;
                    chb_col(W, c0 + q, nb)[idx - q * nb] = v[u];
                }
            }
        }
        if (nthr == 256)
            __syncthreads();
        else
            asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (c1 > c0) {
            const int k1 = src.ktc_ptr[c1];
            for (int k = src.ktc_ptr[c0] + tid - t0; k < k1; k += nthr) {
                const int e = src.ktc_e[k];
                float v = src.kt[e];
                if (src.ct) v += src.wa * src.ct[e];
                chb_col(W, src.ktc_c[k], nb)[src.ktc_r[k]] += v;
            }
        }
    };
    // write panel q's columns of L out of the ring; threads t0 .. t0 + nthr - 1
    auto write_panel = [&](int q, int t0, int nthr) {
        const int j0 = 32 * q, jb = min(32, n - j0), t = tid - t0;
        const float* li = Li + (q & 1) * 32;
        const float* Zq = Z + (q & 1) * 32 * 33;
        for (int k = 0; full && k < jb; ++k) {   // column band, contiguous
            const float* src = chb_col(W, j0 + k, nb);
            float* dst = Ac + (size_t)(j0 + k) * nb;
            for (int r = t; r < nb; r += nthr) dst[r] = (j0 + k + r < n) ? src[r] : 0.f;
        }
        const int rows = min(n, j0 + 32 + b) - j0;
        // row band and backward records, j fastest (records only: the rows below the block)
        for (int idx = t + (full ? 0 : 32 * FSE_BLK); idx < rows * 32; idx += nthr) {
            const int ip = idx >> 5, k = idx & 31, i = j0 + ip, j = j0 + k, r = ip - k;
            if (k >= jb || r < 0 || r > b) continue;
            const float v = chb_col(W, j, nb)[r];
            if (full) Lr[(size_t)i * nb + (b - r)] = v;
            if (Rb && ip >= 32) Rb[(size_t)q * RECE + (ip - 32) * FSE_BLK + k] = v;
        }
        if (Rf) {
            const int rb = rows - 32;   // rows below the diagonal block
            for (int k = 0; k < jb; ++k) {   // forward records, i fastest
                const int j = j0 + k;
                const float* src = chb_col(W, j, nb);
                for (int ii = t; ii < rb; ii += nthr) {
                    const int i = j0 + 32 + ii, r = i - j, i0 = i & ~(FSE_BLK - 1);
                    if (r <= b) Rf[(size_t)(i >> 5) * RECE + (j - i0 + b) * FSE_BLK + (i - i0)] = src[r];
                }
            }
        }
        for (int k = t; full && k < jb; k += nthr) Linv[j0 + k] = li[k];
        float* D = Dinv + (size_t)q * FSE_BLK * FSE_BLK;
        const int dofs = RECE - FSE_BLK * FSE_BLK;
        for (int idx = t; idx < FSE_BLK * FSE_BLK; idx += nthr) {
            const int i = idx >> 5, c = idx & 31;
            const float z = Zq[i * 33 + c];
            if (full) D[idx] = z;
            if (Rf && Rb) {
                Rb[(size_t)q * RECE + dofs + idx] = z;                 // backward record: Dinv
                Rf[(size_t)q * RECE + dofs + c * FSE_BLK + i] = z;     // forward record: Dinv^T
            }
        }
    };
    stage(0, min(n, 32 + b), 0, 256);
    __syncthreads();
    const int npan = (n + FSE_BLK - 1) / FSE_BLK;
    int p = 0;
    for (; p < npan; ++p) {
        const int j0 = 32 * p, jb = min(32, n - j0);
        const int nr = max(0, min(n, j0 + 32 + b) - (j0 + 32));   // rows of L21 (<= b)
        if (tid < 160) {
            const bool ok = chb_panel(o_W, o_Li + (p & 1) * 32, o_P, o_Z + (p & 1) * 32 * 33, o_cb, j0, jb, nr, b, nb);
            if (tid == 0 && !ok) bad = 1;
        } else if (p > 0) {
            write_panel(p - 1, 160, 96);
        }
        __syncthreads();
        if (bad) break;
        // columns first updated by panel p + 1; their ring slots held panels < p, written out above
        if (warp >= 4) {
            const int c0 = 32 * (p + 1) + b;
            stage(min(n, c0), min(n, c0 + 32), 128, 128);
        }
        chb_update(o_W, o_P, j0, nr, nb);
        __syncthreads();
    }
    if (p == npan) write_panel(npan - 1, 0, 256);
    __syncthreads();
    return bad;
}

// FP32 factors with b + 1 <= 96 keep the window in registers; others use the shared window
template <typename T>
__device__ int band_cholesky(T* Ac, T* Lr, T* Linv, int n, int b, T* wnd, T* stg, T* Rf, T* Rb, int RECE) {
    if constexpr (sizeof(T) == 4) {
        const int nb = b + 1;
        if (nb >= 2 && blockDim.x == 256) {
            if (nb <= 32) return cta_band_cholesky_r<T, 4, 1>(Ac, Lr, Linv, n, b, wnd, stg, Rf, Rb, RECE);
            if (nb <= 64) return cta_band_cholesky_r<T, 8, 2>(Ac, Lr, Linv, n, b, wnd, stg, Rf, Rb, RECE);
            if (nb <= 96) return cta_band_cholesky_r<T, 12, 3>(Ac, Lr, Linv, n, b, wnd, stg, Rf, Rb, RECE);
        }
    }
    return cta_band_cholesky_w<T>(Ac, Lr, Linv, n, b, wnd, stg, Rf, Rb, RECE);
}

// inverses of the 32 x 32 diagonal blocks of L (one warp per block, one lane per column);
// the block's lower triangle is first copied to the warp's shared tile
template <typename T>
__device__ void cta_diag_inverses(const T* Lr, const T* Linv, int n, int b, int nblk, T* Dinv, T* tiles,
                                  T* Rf = nullptr, T* Rb = nullptr, int RECE = 0) {
    const int nb = b + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T* Lt = tiles + (size_t)warp * (FSE_BLK * FSE_BLK + FSE_BLK);   // [i][j] j < i, then 1/L_ii
    for (int B = warp; B < nblk; B += nw) {
        const int i0 = B * FSE_BLK;
        __syncwarp();
        for (int idx = lane; idx < FSE_BLK * FSE_BLK; idx += 32) {
            const int i = idx >> 5, j = idx & 31, gi = i0 + i, c = j - i + b;   // row band of L(gi, i0 + j)
            Lt[idx] = (gi < n && j < i && c >= 0) ? Lr[(size_t)gi * nb + c] : T(0);
        }
        Lt[FSE_BLK * FSE_BLK + lane] = (i0 + lane < n) ? Linv[i0 + lane] : T(1);   // identity past n
        __syncwarp();
        T z[FSE_BLK];
#pragma unroll
        for (int i = 0; i < FSE_BLK; ++i) {
            T acc = (i == lane) ? T(1) : T(0);
#pragma unroll
            for (int j = 0; j < i; ++j) acc -= Lt[i * FSE_BLK + j] * z[j];
            z[i] = acc * Lt[FSE_BLK * FSE_BLK + i];
        }
        T* D = Dinv + (size_t)B * FSE_BLK * FSE_BLK;
#pragma unroll
        for (int i = 0; i < FSE_BLK; ++i) D[i * FSE_BLK + lane] = z[i];
        if (Rf) {
            const int dofs = RECE - FSE_BLK * FSE_BLK;
            T* DT = Rf + (size_t)B * RECE + dofs;   // forward record: Dinv^T
            T* Db = Rb + (size_t)B * RECE + dofs;   // backward record: Dinv
#pragma unroll
            for (int i = 0; i < FSE_BLK; ++i) {
                DT[lane * FSE_BLK + i] = z[i];
                Db[i * FSE_BLK + lane] = z[i];
            }
        }
    }
    __syncwarp();
}


// span (elements of the factor precision) of the state kernel's factorisation workspace
__host__ __device__ inline size_t state_wspan(int nb, int blk) {
    const size_t a = (size_t)(nb + 1 + FSE_CHOL_PF) * nb, d = (size_t)8 * (FSE_BLK * FSE_BLK + FSE_BLK);
    size_t w = a > d ? a : d;
    if (blk && chol_blk_floats(nb) > w) w = chol_blk_floats(nb);
    return w;
}

// ----------------------------------------------------------------------------
// the state kernel
// ----------------------------------------------------------------------------

struct StateArgs {
    int n, b, e, dm1, maxit, ncolors, n_el, nnz_kt, kt_ld, nblk, init;
    int refactor;       // 0: keep the previous factors (residual-only steps, see launch_state_step)
    double tol, Dl, a0c, a1c, a2c, w, phi;
    double rho[FSE_MAX_D - 1];
    const double *F, *phis;
    const int *cs_ptr, *cs_col;
    const double *cs_m, *cs_d, *cs_k, *cs_s;
    const int *el_type, *el_dof, *col_off;
    const double* el_p;
    const int *kt_ptr, *kt_col, *kt_soff, *kt_src;
    double* ke;
    void* kt_out;       // N x kt_ld, K_t at the new state
    int has_vel;        // velocity-dependent elements present: C_t values and the velocity vector
    double* ce;         // N x n_el x 36 element velocity tangents (scratch), when has_vel
    void* ct_out;       // N x kt_ld, C_t at the new state (same pattern and ring as K_t)
    const void* ct_prev;   // N x kt_ld, C_t at the previous state
    void* romega;       // N x n, w_1-column term of this step (regular steps)
    const double *LMc, *LMr, *LMinv;
    double *q, *u, *a;
    const void *cLc, *cLr, *cLinv, *cDinv;   // chord factor (regular steps)
    void *oLc, *oLr, *oLinv, *oDinv;         // factor of K_eff at the new state
    void *oRf, *oRb;                         // its block records for the tangent solves
    const void *cRf, *cRb;                   // records of the chord factor (panel factor: the chord
                                             // solves read them instead of the bands)
    int full_factor;                         // panel factor: also write the bands, 1/L_jj and the block
                                             // inverses (read by the tensor-core records)
    const float* Sband;                      // panel factor: lower band of S (all trajectories)
    const int *ktc_ptr, *ktc_e, *ktc_c, *ktc_r;   // ... and the lower K_t entries by column
    int RECE;
    int chol_blk;       // factor K_eff by 32-column panels (FP32, b <= 96)
    int *status, *iters, *nref;
};

// factor of K_eff (column band Ac in place, row band, 1/L_jj, diagonal-block inverses and the
// tangent-solve records); nonzero on a non-positive or non-finite pivot
template <typename T, bool BLK>
__device__ int band_factor(const StateArgs& A, T* Ac, T* Lr, T* Linv, T* Dinv, T* wnd, T* stg, T* Rf, T* Rb,
                           const T* kt = nullptr, const T* ct = nullptr) {
    if constexpr (BLK) {
        const ChbSource src{A.Sband, A.ktc_ptr, A.ktc_e, A.ktc_c, A.ktc_r, kt, ct, float(A.w * A.a2c)};
        return cta_band_cholesky_blk(Ac, Lr, Linv, Dinv, A.n, A.b, wnd, Rf, Rb, A.RECE, A.full_factor != 0, src);
    }
    const int bad = band_cholesky<T>(Ac, Lr, Linv, A.n, A.b, wnd, stg, Rf, Rb, A.RECE);
    if (!bad) cta_diag_inverses<T>(Lr, Linv, A.n, A.b, A.nblk, Dinv, wnd, Rf, Rb, A.RECE);
    return bad;
}

__device__ __forceinline__ double forcing_i(const StateArgs& A, int s, int i, double phi) {
    double e = A.F[i] * cos(phi);
    for (int j = 1; j < A.e; ++j)
        e += A.F[(size_t)j * A.n + i] * cos(A.phis[s * A.dm1 + (j - 1)] + A.rho[j - 1] * phi);
    return e;
}

// r += f_nl(q, qdot), elements processed colour by colour (no two elements of a colour share a
// dof); qd: physical velocities (nullptr when no element depends on them)
__device__ void add_fnl(const StateArgs& A, const double* q, const double* qd, double* r) {
    for (int c = 0; c < A.ncolors; ++c) {
        const int e0 = A.col_off[c], e1 = A.col_off[c + 1];
        for (int el = e0 + threadIdx.x; el < e1; el += blockDim.x) {
            const int type = A.el_type[el];
            const int* dof = A.el_dof + 6 * el;
            double fe[6];
            elem_eval(type, dof, A.el_p + 6 * el, q, qd, fe, nullptr);
            const int nd = elem_ndof(type);
            for (int a = 0; a < nd; ++a)
                if (dof[a] >= 0) r[dof[a]] += fe[a];
        }
        __syncthreads();
    }
}

// Ac = lower column band of K_eff = S + K_t(q, qdot) + w (2/Delta) C_t(q, qdot) (type T), kt_out =
// K_t values on its CSR pattern and, with velocity-dependent elements, ct_out = C_t values on it.
// BAND = false (panel factor): kt_out and ct_out only; the factor stages K_eff itself from the
// band of S and these values.
template <typename T, bool BAND = true>
__device__ void assemble_keff(const StateArgs& A, int s, const double* q, const double* qd, T* Ac, T* kt_out,
                              T* ct_out) {
    const int n = A.n, b = A.b, nb = b + 1;
    double* ke = A.ke + (size_t)s * A.n_el * 36;
    double* ce = A.has_vel ? A.ce + (size_t)s * A.n_el * 36 : nullptr;
    for (int el = threadIdx.x; el < A.n_el; el += blockDim.x) {
        double fe[6];
        elem_eval(A.el_type[el], A.el_dof + 6 * el, A.el_p + 6 * el, q, qd, fe, ke + (size_t)el * 36,
                  ce ? ce + (size_t)el * 36 : nullptr);
    }
    if constexpr (BAND) {
        for (int idx = threadIdx.x; idx < n * nb; idx += blockDim.x) Ac[idx] = T(0);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int e1 = A.cs_ptr[i + 1];
            for (int e = A.cs_ptr[i]; e < e1; ++e) {
                const int j = A.cs_col[e];
                if (j <= i) Ac[(size_t)j * nb + (i - j)] = T(A.cs_s[e]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int e1 = A.kt_ptr[i + 1];
        for (int e = A.kt_ptr[i]; e < e1; ++e) {
            double v = 0.0, vc = 0.0;
            const int s1 = A.kt_soff[e + 1];
            for (int k = A.kt_soff[e]; k < s1; ++k) v += ke[A.kt_src[k]];
            kt_out[e] = T(v);
            if (ce) {
                for (int k = A.kt_soff[e]; k < s1; ++k) vc += ce[A.kt_src[k]];
                ct_out[e] = T(vc);
                v += A.w * A.a2c * vc;   // d u / d q = 2 / Delta, d qdot / d u = w
            }
            const int j = A.kt_col[e];
            if (BAND && j <= i) {
                const size_t o = (size_t)j * nb + (i - j);
                Ac[o] = T((double)Ac[o] + v);
            }
        }
    }
    __syncthreads();
}

// Blocked banded solve L L^T x = r in place (r in shared memory, FP64 in and out) with the
// arithmetic in the factor precision T: r is rounded to T once, both substitutions run in T
// and x is widened back.  With the FP64 residual of the Newton iteration around it this is
// iterative refinement, so the converged state keeps FP64 accuracy.  32-row blocks; the
// off-diagonal band part as dot products (32 rows x 8 lanes); diagonal blocks through their
// stored inverses.  For b <= 96 the next block's band entries and inverse are loaded into
// registers while the current block computes.
template <typename T>
__device__ void cta_blocked_solve(const T* __restrict__ Lc, const T* __restrict__ Lr,
                                  const T* __restrict__ Dinv, int n, int b, int nblk, double* r, T* y,
                                  T* tmp) {
    constexpr int MC = 12;                                     // band entries per lane (b <= 96)
    const int nb = b + 1;
    const int row = threadIdx.x >> 3, l8 = threadIdx.x & 7;   // 32 rows x 8 lanes
    const bool pf = b <= 8 * MC;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = T(r[i]);
    __syncthreads();
    T lcur[MC], lnxt[MC], dcur[4], dnxt[4];
    // forward: y_B = Dinv_B (r_B - L_{B,<} y_<); lane l8 holds L(i, i0 - b + l8 + 8q)
    auto fwd_load = [&](int B, T* lv, T* dv) {
        const int i0 = B * FSE_BLK, i = i0 + row;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int c = l8 + 8 * q, j = i0 - b + c, bi = c - row;
            lv[q] = (i < n && c < b && j >= 0 && bi >= 0) ? Lr[(size_t)i * nb + bi] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = l8 + 8 * q;
            dv[q] = (k <= row) ? Dinv[(size_t)B * FSE_BLK * FSE_BLK + row * FSE_BLK + k] : T(0);
        }
    };
    if (pf) fwd_load(0, lnxt, dnxt);
    for (int B = 0; B < nblk; ++B) {
        const int i0 = B * FSE_BLK, i = i0 + row;
        T part = T(0);
        if (pf) {
#pragma unroll
            for (int q = 0; q < MC; ++q) lcur[q] = lnxt[q];
#pragma unroll
            for (int q = 0; q < 4; ++q) dcur[q] = dnxt[q];
            if (B + 1 < nblk) fwd_load(B + 1, lnxt, dnxt);
#pragma unroll
            for (int q = 0; q < MC; ++q) {
                const int c = l8 + 8 * q, j = i0 - b + c;   // j < i0 <= n - 1 for c < b
                if (c < b && j >= 0) part += lcur[q] * y[j];
            }
        } else if (i < n) {
            for (int c = l8; c < b; c += 8) {
                const int j = i0 - b + c, bi = c - row;
                if (j >= 0 && bi >= 0) part += Lr[(size_t)i * nb + bi] * y[j];
            }
        }
        part += __shfl_xor_sync(0xffffffffu, part, 4);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        if (l8 == 0) tmp[row] = (i < n) ? y[i] - part : T(0);
        __syncthreads();
        T yv = T(0);
        if (pf) {
#pragma unroll
            for (int q = 0; q < 4; ++q) yv += dcur[q] * tmp[l8 + 8 * q];
        } else {
            const T* D = Dinv + (size_t)B * FSE_BLK * FSE_BLK + row * FSE_BLK;
            for (int k = l8; k <= row; k += 8) yv += D[k] * tmp[k];
        }
        yv += __shfl_xor_sync(0xffffffffu, yv, 4);
        yv += __shfl_xor_sync(0xffffffffu, yv, 2);
        yv += __shfl_xor_sync(0xffffffffu, yv, 1);
        if (l8 == 0 && i < n) y[i] = yv;
        __syncthreads();
    }
    // backward: x_B = Dinv_B^T (y_B - L_{>,B}^T x_>); lane l8 holds L(i0 + 32 + l8 + 8q, i)
    auto bwd_load = [&](int B, T* lv, T* dv) {
        const int i0 = B * FSE_BLK, i = i0 + row;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int c = l8 + 8 * q, k = i0 + FSE_BLK + c, ci = k - i;
            lv[q] = (i < n && c < b && k < n && ci <= b) ? Lc[(size_t)i * nb + ci] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = row + l8 + 8 * q;
            dv[q] = (k < FSE_BLK) ? Dinv[(size_t)B * FSE_BLK * FSE_BLK + k * FSE_BLK + row] : T(0);
        }
    };
    if (pf) bwd_load(nblk - 1, lnxt, dnxt);
    for (int B = nblk - 1; B >= 0; --B) {
        const int i0 = B * FSE_BLK, i = i0 + row;
        T part = T(0);
        if (pf) {
#pragma unroll
            for (int q = 0; q < MC; ++q) lcur[q] = lnxt[q];
#pragma unroll
            for (int q = 0; q < 4; ++q) dcur[q] = dnxt[q];
            if (B > 0) bwd_load(B - 1, lnxt, dnxt);
#pragma unroll
            for (int q = 0; q < MC; ++q) {
                const int c = l8 + 8 * q, k = i0 + FSE_BLK + c;
                if (c < b && k < n) part += lcur[q] * y[k];
            }
        } else if (i < n) {
            for (int c = l8; c < b; c += 8) {
                const int k = i0 + FSE_BLK + c, ci = k - i;
                if (k < n && ci <= b) part += Lc[(size_t)i * nb + ci] * y[k];
            }
        }
        part += __shfl_xor_sync(0xffffffffu, part, 4);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        if (l8 == 0) tmp[row] = (i < n) ? y[i] - part : T(0);
        __syncthreads();
        T xv = T(0);
        if (pf) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = row + l8 + 8 * q;
                if (k < FSE_BLK) xv += dcur[q] * tmp[k];
            }
        } else {
            const T* D = Dinv + (size_t)B * FSE_BLK * FSE_BLK;
            for (int k = row + l8; k < FSE_BLK; k += 8) xv += D[k * FSE_BLK + row] * tmp[k];
        }
        xv += __shfl_xor_sync(0xffffffffu, xv, 4);
        xv += __shfl_xor_sync(0xffffffffu, xv, 2);
        xv += __shfl_xor_sync(0xffffffffu, xv, 1);
        if (l8 == 0 && i < n) y[i] = xv;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = (double)y[i];
    __syncthreads();
}

// The same solve for the panel factor (FP32, b <= 96), from the tangent-solve records of the
// factor: forward record of block B [L(i0 + r, i0 - b + c) at c * 32 + r | Dinv^T at
// (bpad + k) * 32 + r], backward record [L(i0 + 32 + c, i0 + r) at c * 32 + r | Dinv]; entries
// outside the band are zero there.  Each block's record (RECE floats) is copied to shared memory
// by 16-byte cp.async while the previous block computes, into rows padded to 36 floats (ws: two
// such buffers): the 32 lanes of a warp (4 rows r x 8 record rows c) then read 32 different
// banks, 4 c + r.
__device__ void cta_record_solve(const float* __restrict__ Rf, const float* __restrict__ Rb, int RECE, int n, int b,
                                 int nblk, double* r, float* y, float* tmp, float* ws) {
    constexpr int MC = 12;     // band entries per lane (b <= 96)
    constexpr int MAXU = 4;    // 16-byte chunks per thread (RECE <= (96 + 32) * 32 = 4 * 4 * 256)
    constexpr int RP = 36;
    const int tid = threadIdx.x, row = tid >> 3, l8 = tid & 7;   // 32 rows x 8 lanes
    const int nrr = RECE / FSE_BLK, dr = nrr - FSE_BLK;          // record rows; first row of the block inverse
    float* rs[2] = {ws, ws + nrr * RP};
    auto fetch = [&](const float* R, float* d) {   // record R into the padded buffer d
#pragma unroll
        for (int u = 0; u < MAXU; ++u) {
            const int ch = tid + 256 * u;   // floats 4 ch .. 4 ch + 3: record row ch / 8
            if (4 * ch < RECE) cp_async16(d + (ch >> 3) * RP + 4 * (ch & 7), R + 4 * ch, 16);
        }
        cp_async_commit();
    };
    for (int i = tid; i < n; i += blockDim.x) y[i] = float(r[i]);
    // forward: y_B = Dinv_B (r_B - L_{B,<} y_<)
    fetch(Rf, rs[0]);
    cp_async_wait0();
    __syncthreads();
    for (int B = 0; B < nblk; ++B) {
        const int i0 = B * FSE_BLK, i = i0 + row;
        const float* R = rs[B & 1];
        if (B + 1 < nblk) fetch(Rf + (size_t)(B + 1) * RECE, rs[(B + 1) & 1]);   // last read at block B - 1
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int c = l8 + 8 * q, j = i0 - b + c;
            if (c < b && j >= 0) part += R[c * RP + row] * y[j];
        }
        part += __shfl_xor_sync(0xffffffffu, part, 4);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        if (l8 == 0) tmp[row] = (i < n) ? y[i] - part : 0.f;
        __syncthreads();
        float yv = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = l8 + 8 * q;
            yv += R[(dr + k) * RP + row] * tmp[k];
        }
        yv += __shfl_xor_sync(0xffffffffu, yv, 4);
        yv += __shfl_xor_sync(0xffffffffu, yv, 2);
        yv += __shfl_xor_sync(0xffffffffu, yv, 1);
        if (l8 == 0 && i < n) y[i] = yv;
        cp_async_wait0();
        __syncthreads();
    }
    // backward: x_B = Dinv_B^T (y_B - L_{>,B}^T x_>)
    fetch(Rb + (size_t)(nblk - 1) * RECE, rs[0]);
    cp_async_wait0();
    __syncthreads();
    for (int q2 = 0; q2 < nblk; ++q2) {
        const int B = nblk - 1 - q2, i0 = B * FSE_BLK, i = i0 + row;
        const float* R = rs[q2 & 1];
        if (B > 0) fetch(Rb + (size_t)(B - 1) * RECE, rs[(q2 + 1) & 1]);
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int c = l8 + 8 * q, k = i0 + FSE_BLK + c;
            if (c < b && k < n) part += R[c * RP + row] * y[k];
        }
        part += __shfl_xor_sync(0xffffffffu, part, 4);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        if (l8 == 0) tmp[row] = (i < n) ? y[i] - part : 0.f;
        __syncthreads();
        float xv = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = row + l8 + 8 * q;
            if (k < FSE_BLK) xv += R[(dr + k) * RP + row] * tmp[k];
        }
        xv += __shfl_xor_sync(0xffffffffu, xv, 4);
        xv += __shfl_xor_sync(0xffffffffu, xv, 2);
        xv += __shfl_xor_sync(0xffffffffu, xv, 1);
        if (l8 == 0 && i < n) y[i] = xv;
        cp_async_wait0();
        __syncthreads();
    }
    for (int i = tid; i < n; i += blockDim.x) r[i] = (double)y[i];
    __syncthreads();
}

// Single-warp banded solve of the FP64 mass factor (setup-time layouts), used once per
// evaluation for the consistent initial acceleration.
__device__ void warp_band_solve_fp64(const double* __restrict__ Lc, const double* __restrict__ Lr,
                                     const double* __restrict__ Linv, int n, int b, double* r) {
    const int lane = threadIdx.x & 31;
    const int nb = b + 1;
    for (int j = 0; j < n; ++j) {
        const double x = r[j] * Linv[j];
        __syncwarp();
        if (lane == 0) r[j] = x;
        for (int rr = 1 + lane; rr <= b; rr += 32) {
            const int i = j + rr;
            if (i < n) r[i] -= Lc[(size_t)j * nb + rr] * x;
        }
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {
        const double x = r[j] * Linv[j];
        __syncwarp();
        if (lane == 0) r[j] = x;
        for (int rr = 1 + lane; rr <= b; rr += 32) {
            const int i = j - rr;
            if (i >= 0) r[i] -= Lr[(size_t)j * nb + b - rr] * x;
        }
        __syncwarp();
    }
}

// BLK: FP32 factor by 32-column panels (the launcher picks it when chol_blk is set)
template <typename T, bool BLK>
__global__ void __launch_bounds__(256) k_state(StateArgs A) {
    static_assert(!BLK || sizeof(T) == 4, "panel Cholesky is FP32 only");
    const int s = blockIdx.x, n = A.n, b = A.b, nb = b + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ double sm[];
    double *sq = sm, *su = sq + n, *sa = su + n, *sqn = sa + n, *sb = sqn + n, *sr = sb + n;
    T* tmp = reinterpret_cast<T*>(sr + n);                // 32
    // Cholesky window ((nb + 1) x nb) and staging ring (FSE_CHOL_PF x nb); the diagonal-block
    // tiles of cta_diag_inverses reuse the same space once the factorisation is done
    T* wnd = reinterpret_cast<T*>(sr + n + FSE_BLK);
    T* stg = wnd + (size_t)(nb + 1) * nb;
    const size_t wspan = state_wspan(nb, BLK ? 1 : 0);
    T* ysol = wnd + wspan;                                // n: solve vector in the factor precision
    // physical velocities qdot = w u of the current iterate (velocity-dependent elements only)
    double* sv = A.has_vel
                     ? reinterpret_cast<double*>((reinterpret_cast<size_t>(ysol + n) + 7) & ~static_cast<size_t>(7))
                     : nullptr;
    __shared__ int s_conv, s_stat;
    const size_t off = (size_t)s * n;
    const size_t foff = (size_t)s * n * nb;
    const size_t doff = (size_t)s * A.nblk * FSE_BLK * FSE_BLK;
    T* oLc = reinterpret_cast<T*>(A.oLc) + foff;
    T* oLr = reinterpret_cast<T*>(A.oLr) + foff;
    T* oLi = reinterpret_cast<T*>(A.oLinv) + off;
    T* oDi = reinterpret_cast<T*>(A.oDinv) + doff;
    T* oRf = reinterpret_cast<T*>(A.oRf) + (size_t)s * A.nblk * A.RECE;
    T* oRb = reinterpret_cast<T*>(A.oRb) + (size_t)s * A.nblk * A.RECE;
    T* kt_out = reinterpret_cast<T*>(A.kt_out) + (size_t)s * A.kt_ld;
    T* ct_out = A.has_vel ? reinterpret_cast<T*>(A.ct_out) + (size_t)s * A.kt_ld : nullptr;
    // sv = w u at the state (sq, su), or, in the step, at u(q) = 2/Delta (q - q_k) - u_k
    auto vel_state = [&]() {
        if (!sv) return;
        for (int i = tid; i < n; i += nt) sv[i] = A.w * su[i];
        __syncthreads();
    };
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
    int it = 0, nref = 0;
    if (A.init) {
        // consistent start: w^2 M a0 = e(0) - w D u0 - K q0 - f_nl(q0)  (Eq. E2 at phi_1 = 0)
        for (int i = tid; i < n; i += nt) sr[i] = 0.0;
        __syncthreads();
        vel_state();
        add_fnl(A, sq, sv, sr);
        for (int i = tid; i < n; i += nt)
            sb[i] = forcing_i(A, s, i, 0.0) - A.w * csr_row(A.cs_ptr, A.cs_col, A.cs_d, i, su) -
                    csr_row(A.cs_ptr, A.cs_col, A.cs_k, i, sq) - sr[i];
        __syncthreads();
        if (tid < 32) warp_band_solve_fp64(A.LMc, A.LMr, A.LMinv, n, b, sb);
        __syncthreads();
        const double iw2 = 1.0 / (A.w * A.w);
        double zmax = 0.0, amax = 0.0;
        for (int i = tid; i < n; i += nt) {
            sa[i] = sb[i] * iw2;
            A.a[off + i] = sa[i];
            zmax = nanmax(zmax, nanmax(fabs(sq[i]), fabs(su[i])));
            amax = nanmax(amax, fabs(sa[i]));
        }
        block_max2(zmax, amax);
        // a non-finite start point (from Z(0)) is reported as such, not as a failed factorisation
        if (tid == 0 && (!isfinite(zmax) || !isfinite(amax))) s_stat = FSE_ENAN;
        __syncthreads();
    } else {
        const T* cLc = reinterpret_cast<const T*>(A.cLc) + foff;
        const T* cLr = reinterpret_cast<const T*>(A.cLr) + foff;
        const T* cDi = reinterpret_cast<const T*>(A.cDinv) + doff;
        const size_t roff = (size_t)s * A.nblk * A.RECE;
        const T* cRf = BLK ? reinterpret_cast<const T*>(A.cRf) + roff : nullptr;
        const T* cRb = BLK ? reinterpret_cast<const T*>(A.cRb) + roff : nullptr;
        // b = e_{k+1} + w^2 M (a0 q + a1 u + a) + w D (a2 q + u)   (Eq. E7)
        for (int i = tid; i < n; i += nt) {
            sr[i] = A.a0c * sq[i] + A.a1c * su[i] + sa[i];
            sqn[i] = A.a2c * sq[i] + su[i];
        }
        __syncthreads();
        const double w2 = A.w * A.w;
        for (int i = tid; i < n; i += nt)
            sb[i] = forcing_i(A, s, i, A.phi) + w2 * csr_row(A.cs_ptr, A.cs_col, A.cs_m, i, sr) +
                    A.w * csr_row(A.cs_ptr, A.cs_col, A.cs_d, i, sqn);
        __syncthreads();
        for (int i = tid; i < n; i += nt) sqn[i] = sq[i];   // predictor: the previous displacement
        __syncthreads();
        // Newton on Eq. (E6): starts as a chord iteration with the factor of K_eff(q_k) and
        // refactors at the current iterate whenever the contraction ratio exceeds 0.1
        double prev = -1.0;
        auto vel_iterate = [&]() {
            if (!sv) return;
            for (int i = tid; i < n; i += nt) sv[i] = A.w * (A.a2c * (sqn[i] - sq[i]) - su[i]);
            __syncthreads();
        };
        for (it = 0; it < A.maxit; ++it) {
            for (int i = tid; i < n; i += nt) sr[i] = csr_row(A.cs_ptr, A.cs_col, A.cs_s, i, sqn) - sb[i];
            __syncthreads();
            vel_iterate();
            add_fnl(A, sqn, sv, sr);
            if constexpr (BLK)
                cta_record_solve(cRf, cRb, A.RECE, n, b, A.nblk, sr, ysol, tmp, wnd);
            else
                cta_blocked_solve<T>(cLc, cLr, cDi, n, b, A.nblk, sr, ysol, tmp);
            double dmax = 0.0, qmax = 0.0;
            for (int i = tid; i < n; i += nt) {
                const double v = sqn[i] - sr[i];
                sqn[i] = v;
                dmax = nanmax(dmax, fabs(sr[i]));
                qmax = nanmax(qmax, fabs(v));
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
            // an FP32 factor limits the chord contraction by itself: one refactorisation per
            // step is enough to tell nonlinearity from rounding, more would only repeat it
            const bool allow = sizeof(T) == 8 || nref == 0;
            if (prev > 0.0 && dmax > 0.1 * prev && it + 1 < A.maxit && allow) {
                ++nref;
                vel_iterate();
                assemble_keff<T, !BLK>(A, s, sqn, sv, oLc, kt_out, ct_out);
                if (band_factor<T, BLK>(A, oLc, oLr, oLi, oDi, wnd, stg, oRf, oRb, kt_out, ct_out)) {
                    if (tid == 0) s_stat = FSE_ENONPOS_PIVOT;
                    ++it;
                    break;
                }
                __syncthreads();
                cLc = oLc;
                cLr = oLr;
                cDi = oDi;
                cRf = oRf;
                cRb = oRb;
            }
            prev = dmax;
        }
        __syncthreads();
        if (tid == 0 && A.tol > 0.0 && !s_conv && s_stat == 0) s_stat = FSE_ENOCONV;
        // corrector (Eq. E5); sums of old and new u, a for the w_1 column of the tangents
        for (int i = tid; i < n; i += nt) {
            const double dq = sqn[i] - sq[i];
            const double un = A.a2c * dq - su[i];
            const double an = A.a0c * dq - A.a1c * su[i] - sa[i];
            sb[i] = su[i] + un;
            sr[i] = sa[i] + an;
            sq[i] = sqn[i];
            su[i] = un;
            sa[i] = an;
            A.q[off + i] = sqn[i];
            A.u[off + i] = un;
            A.a[off + i] = an;
        }
        __syncthreads();
        // w_1 column: -2 w M (a_k + a_{k+1}) - D (u_k + u_{k+1})
        T* rom = reinterpret_cast<T*>(A.romega) + off;
        for (int i = tid; i < n; i += nt)
            rom[i] = T(-2.0 * A.w * csr_row(A.cs_ptr, A.cs_col, A.cs_m, i, sr) -
                       csr_row(A.cs_ptr, A.cs_col, A.cs_d, i, sb));
        __syncthreads();
    }
    // effective stiffness at the new state, its banded Cholesky factor and block inverses
    int bad = 0;
    if (A.refactor) {
        vel_state();
        assemble_keff<T, !BLK>(A, s, sq, sv, oLc, kt_out, ct_out);
        if (A.has_vel && !A.init) {
            // velocity-dependent elements add - C_t(k+1) u_{k+1} - C_t(k) u_k to the w_1 column
            // (d f / d w_1 = C_t u at both ends of the step); sb holds u_k + u_{k+1}, su u_{k+1}
            __syncthreads();
            T* rom = reinterpret_cast<T*>(A.romega) + off;
            const T* cp = reinterpret_cast<const T*>(A.ct_prev) + (size_t)s * A.kt_ld;
            for (int i = tid; i < n; i += nt) {
                double acc = 0.0;
                const int e1 = A.kt_ptr[i + 1];
                for (int e = A.kt_ptr[i]; e < e1; ++e) {
                    const int j = A.kt_col[e];
                    acc += (double)ct_out[e] * su[j] + (double)cp[e] * (sb[j] - su[j]);
                }
                rom[i] = T((double)rom[i] - acc);
            }
        }
        bad = band_factor<T, BLK>(A, oLc, oLr, oLi, oDi, wnd, stg, oRf, oRb, kt_out, ct_out);
    }
    if (tid == 0) {
        if (bad && s_stat == 0) s_stat = FSE_ENONPOS_PIVOT;
        A.status[s] = s_stat;
        A.iters[s] = (A.init ? 0 : A.iters[s]) + it;
        A.nref[s] = (A.init ? 0 : A.nref[s]) + nref;
    }
}

// ----------------------------------------------------------------------------
// mass factor at setup
// ----------------------------------------------------------------------------

__global__ void k_factor_M(int n, int b, const double* Mb, double* LMc, double* LMr, double* LMinv,
                           int* flag) {
    extern __shared__ double wndM[];
    const int nb = b + 1;
    double* stgM = wndM + (nb + 1) * nb;
    for (int idx = threadIdx.x; idx < n * nb; idx += blockDim.x) {
        const int j = idx / nb, r = idx - j * nb, i = j + r;
        LMc[idx] = (i < n) ? Mb[(size_t)(b - r) * n + i] : 0.0;
    }
    __syncthreads();
    const int bad = cta_band_cholesky_w<double>(LMc, LMr, LMinv, n, b, wndM, stgM, nullptr, nullptr, 0);
    if (threadIdx.x == 0) *flag = bad;
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------

void launch_fill_tables(fse_ctx* c) {
    ensure_constants();
    const Params& p = c->p;
    k_tables<<<p.N, 128, 0, c->stream>>>(p.N, p.N_glob, p.U, p.d - 1, c->d.ktab, c->d.phis, c->d.rc, c->d.rs,
                                         c->d.G, c->d.Gi, c->d.RG);
}

void launch_build_ops(fse_ctx* c, double w) {
    const Params& p = c->p;
    const double Dl = 2.0 * M_PI / p.S1;
    const double cm = w * w * 4.0 / (Dl * Dl), cd = w * 2.0 / Dl, cb = w * w * 4.0 / Dl;
    const int g = nblocks(p.nnz, 256);
    if (p.prec == FSE_MIXED_FP32)
        k_build_ops<float><<<g, 256, 0, c->stream>>>(p.nnz, cm, cd, cb, c->d.cs_m, c->d.cs_d, c->d.cs_k,
                                                     c->d.cs_s, (float*)c->d.cs_A, (float*)c->d.cs_B);
    else
        k_build_ops<double><<<g, 256, 0, c->stream>>>(p.nnz, cm, cd, cb, c->d.cs_m, c->d.cs_d, c->d.cs_k,
                                                      c->d.cs_s, (double*)c->d.cs_A, (double*)c->d.cs_B);
    if (p.chol_blk) {
        const int nb = p.b + 1;
        cudaMemsetAsync(c->d.Sband, 0, (size_t)p.n * nb * 4, c->stream);
        k_sband<<<nblocks(p.n, 128), 128, 0, c->stream>>>(p.n, nb, c->d.cs_ptr, c->d.cs_col, c->d.cs_s,
                                                          (float*)c->d.Sband);
    }
}

int launch_factor_M(fse_ctx* c) {
    ensure_constants();
    const Params& p = c->p;
    const int nb = p.b + 1;
    int* flag = c->d.flag + 2;   // non-positive pivot of M: the context's third status word
    cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    const size_t smem = (size_t)(nb + 1 + FSE_CHOL_PF) * nb * sizeof(double);
    cudaFuncSetAttribute(k_factor_M, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_factor_M<<<1, 256, smem, c->stream>>>(p.n, p.b, c->d.Mb, c->d.LMc, c->d.LMr, c->d.LMinv, flag);
    int h = 0;
    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    return h;
}

size_t state_smem(const Params& p) {
    const int nb = p.b + 1;
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    const size_t wspan = state_wspan(nb, tsz == 4 ? p.chol_blk : 0);
    return (size_t)(6 * p.n + FSE_BLK) * 8 + (wspan + (size_t)p.n) * tsz + (p.has_vel ? (size_t)p.n * 8 + 8 : 0);
}

static StateArgs make_state_args(fse_ctx* c, double w, int init, int k) {
    const Params& p = c->p;
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    StateArgs A;
    A.n = p.n;
    A.b = p.b;
    A.e = p.e;
    A.dm1 = p.d - 1;
    A.maxit = p.maxit;
    A.ncolors = p.ncolors;
    A.n_el = p.n_el;
    A.nnz_kt = p.nnz_kt;
    A.kt_ld = p.kt_ld;
    A.nblk = p.nblk;
    A.init = init;
    A.tol = p.tol;
    A.Dl = 2.0 * M_PI / p.S1;
    A.a0c = 4.0 / (A.Dl * A.Dl);
    A.a1c = 4.0 / A.Dl;
    A.a2c = 2.0 / A.Dl;
    A.w = w;
    A.phi = (k + 1) * A.Dl;
    for (int j = 0; j < FSE_MAX_D - 1; ++j) A.rho[j] = j < (int)c->rho.size() ? c->rho[j] : 0.0;
    A.F = c->d.F;
    A.phis = c->d.phis;
    A.cs_ptr = c->d.cs_ptr;
    A.cs_col = c->d.cs_col;
    A.cs_m = c->d.cs_m;
    A.cs_d = c->d.cs_d;
    A.cs_k = c->d.cs_k;
    A.cs_s = c->d.cs_s;
    A.el_type = c->d.el_type;
    A.el_dof = c->d.el_dof;
    A.col_off = c->d.col_off;
    A.el_p = c->d.el_p;
    A.kt_ptr = c->d.kt_ptr;
    A.kt_col = c->d.kt_col;
    A.kt_soff = c->d.kt_soff;
    A.kt_src = c->d.kt_src;
    A.ke = c->d.ke;
    A.has_vel = p.has_vel ? 1 : 0;
    A.ce = c->d.ce;
    const size_t ktsz = (size_t)p.N * p.kt_ld * tsz;
    const size_t fsz = (size_t)p.N * p.n * (p.b + 1) * tsz;
    const size_t vsz = (size_t)p.N * p.n * tsz;
    const size_t dsz = (size_t)p.N * p.nblk * FSE_BLK * FSE_BLK * tsz;
    // state k (new state q_{k+1}) writes K_t(q_{k+1}) to buffer (k+1) % 3 and the factor to k % 2;
    // the init call (k = -1) writes buffer 0 and factor 1
    const int kt_idx = (k + 1) % FSE_NBUF_KT;
    const int fo = ((k % 2) + 2) % 2, fi = 1 - fo;
    A.kt_out = (char*)c->d.kt_val + kt_idx * ktsz;
    A.ct_out = p.has_vel ? (char*)c->d.ct_val + kt_idx * ktsz : nullptr;
    A.ct_prev = p.has_vel ? (const char*)c->d.ct_val + (size_t)(((k % FSE_NBUF_KT) + FSE_NBUF_KT) % FSE_NBUF_KT) * ktsz
                          : nullptr;
    A.romega = (char*)c->d.romega + (size_t)fo * vsz;
    A.LMc = c->d.LMc;
    A.LMr = c->d.LMr;
    A.LMinv = c->d.LMinv;
    A.q = c->d.q;
    A.u = c->d.u;
    A.a = c->d.a;
    A.cLc = (char*)c->d.Lc + fi * fsz;
    A.cLr = (char*)c->d.Lr + fi * fsz;
    A.cLinv = (char*)c->d.Linv + fi * vsz;
    A.cDinv = (char*)c->d.Dinv + fi * dsz;
    A.oLc = (char*)c->d.Lc + fo * fsz;
    A.oLr = (char*)c->d.Lr + fo * fsz;
    A.oLinv = (char*)c->d.Linv + fo * vsz;
    A.oDinv = (char*)c->d.Dinv + fo * dsz;
    const size_t rsz = (size_t)p.N * p.nblk * p.RECE * tsz;
    A.oRf = (char*)c->d.Rf + fo * rsz;
    A.oRb = (char*)c->d.Rb + fo * rsz;
    A.cRf = (char*)c->d.Rf + fi * rsz;
    A.cRb = (char*)c->d.Rb + fi * rsz;
    A.full_factor = use_tc(c) ? 1 : 0;
    A.Sband = (const float*)c->d.Sband;
    A.ktc_ptr = c->d.ktc_ptr;
    A.ktc_e = c->d.ktc_e;
    A.ktc_c = c->d.ktc_c;
    A.ktc_r = c->d.ktc_r;
    A.RECE = p.RECE;
    A.chol_blk = p.chol_blk;
    A.status = c->d.status;
    A.iters = c->d.iters;
    A.nref = c->d.nref;
    return A;
}

template <typename T, bool BLK>
static void state_launch_k(fse_ctx* c, const StateArgs& A, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_set{0};
    if (needs_device_setup(attr_set)) {
        cudaFuncSetAttribute(k_state<T, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        mark_device(attr_set);
    }
    k_state<T, BLK><<<c->p.N, 256, c->p.smem_state, st>>>(A);
}
template <typename T>
static void state_launch(fse_ctx* c, const StateArgs& A, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (A.chol_blk) {
            state_launch_k<float, true>(c, A, st);
            return;
        }
    }
    state_launch_k<T, false>(c, A, st);
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

void launch_init_state(fse_ctx* c, double w) {
    ensure_constants();
    const Params& p = c->p;
    const size_t tot = (size_t)p.N * p.n;
    k_split<<<nblocks(tot, 256), 256, 0, c->stream>>>(p.N, p.n, c->d.zb, c->d.q, c->d.u);
    StateArgs A = make_state_args(c, w, 1, -1);
    A.refactor = 1;
    if (p.prec == FSE_MIXED_FP32)
        state_launch<float>(c, A, c->stream);
    else
        state_launch<double>(c, A, c->stream);
}

// Without tangents (residual-only evaluations) the factor at the end of a step only serves as
// the chord matrix of the next step's Newton, whose FP64 residual makes any recent factor
// good enough; those evaluations refactor on two consecutive steps out of four (both parity
// buffers stay at most four steps old) and always on steps 0 and 1, and the in-loop refactor
// of k_state still reacts to a slow contraction.
void launch_state_step(fse_ctx* c, int k, double w, cudaStream_t st, bool sens) {
    StateArgs A = make_state_args(c, w, 0, k);
    A.refactor = (sens || k < 2 || (k & 3) < 2) ? 1 : 0;
    if (c->p.prec == FSE_MIXED_FP32)
        state_launch<float>(c, A, st);
    else
        state_launch<double>(c, A, st);
    // the tensor-core solves of step k read records built from this step's factor: built here, on the
    // state stream, so that they overlap the tangent kernels of step k - 1 (record buffer k % 2)
    if (sens && use_tc(c)) launch_tc_records(c, k, st);
}

}  // namespace fse
