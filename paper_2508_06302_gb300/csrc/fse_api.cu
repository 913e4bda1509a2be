// C-ABI entry points of the FSE-Shooting library (include/fse.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <map>
#include <string>
#include <vector>

#include "fse_internal.h"

using fse::Params;

static std::string g_setup_err;

static int set_err(fse_ctx* c, int code, const std::string& msg) {
    if (c)
        c->err = msg;
    else
        g_setup_err = msg;
    return code;
}

static int cuda_check(fse_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FSE_OK;
    return set_err(c, e == cudaErrorMemoryAllocation ? FSE_ENOMEM : FSE_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// App. B, Eq. (B1)-(B2): rows k~_1 .. k~_L, then the zero row.
static std::vector<std::vector<int>> harmonic_rows(const std::vector<int>& H) {
    std::vector<std::vector<int>> tab;
    for (int k = 1; k <= H[0]; ++k) tab.push_back({k});
    tab.push_back({0});
    for (size_t dd = 1; dd < H.size(); ++dd) {
        const int Hd = H[dd];
        std::vector<std::vector<int>> next;
        // K^{d,g}: k_d slowest, the rows of K~^{d-1} without its zero row fastest, last entry -k_d
        for (int kd = 1; kd <= Hd; ++kd)
            for (size_t r = 0; r + 1 < tab.size(); ++r) {
                std::vector<int> row = tab[r];
                row.push_back(-kd);
                next.push_back(row);
            }
        // K~^{d,b}: [k_d; 0] slowest, all rows of K~^{d-1} fastest, last entry +k_d (or 0)
        for (int kk = 1; kk <= Hd + 1; ++kk) {
            const int kd = (kk <= Hd) ? kk : 0;
            for (size_t r = 0; r < tab.size(); ++r) {
                std::vector<int> row = tab[r];
                row.push_back(kd);
                next.push_back(row);
            }
        }
        tab.swap(next);
    }
    return tab;
}

template <typename P>
static cudaError_t dalloc(P** p, size_t bytes) {
    return cudaMalloc((void**)p, bytes > 0 ? bytes : 16);
}

// Row groups of the right-hand-side kernel: rows whose column patterns are identical and
// at most 7 rows apart (the dofs of one FE node that couple to the same neighbours), at most
// R rows per group.  Entries of a group are the common pattern; map holds the CSR index of
// every (entry, row) pair.
struct RowGroups {
    int R = 1;
    std::vector<int> rows;   // ng x R, -1 = padding
    std::vector<int> ptr;    // ng + 1
    std::vector<int> col;    // E
    std::vector<int> map;    // E x R
};

static RowGroups group_rows(int n, const std::vector<int>& cptr, const std::vector<int>& ccol, int R) {
    RowGroups G;
    G.R = R;
    std::map<std::vector<int>, int> open;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < n; ++i) {
        std::vector<int> pat(ccol.begin() + cptr[i], ccol.begin() + cptr[i + 1]);
        auto it = open.find(pat);
        if (it != open.end()) {
            std::vector<int>& mem = members[it->second];
            if ((int)mem.size() < R && i - mem[0] < 8) {
                mem.push_back(i);
                continue;
            }
        }
        open[pat] = (int)members.size();
        members.push_back({i});
    }
    G.ptr.push_back(0);
    for (const auto& mem : members) {
        const int i0 = mem[0], len = cptr[i0 + 1] - cptr[i0];
        for (int r = 0; r < R; ++r) G.rows.push_back(r < (int)mem.size() ? mem[r] : -1);
        for (int k = 0; k < len; ++k) {
            G.col.push_back(ccol[cptr[i0] + k]);
            for (int r = 0; r < R; ++r) G.map.push_back(r < (int)mem.size() ? cptr[mem[r]] + k : -1);
        }
        G.ptr.push_back((int)G.col.size());
    }
    return G;
}

// bytes of one group record: the ring slot (int, padded to 8 bytes), then 2R values
static int group_record_bytes(int R, size_t tsz) { return (int)((8 + 2 * R * tsz + 15) / 16 * 16); }

// cos and sin of the rotation angles 2 pi k~_l . rho of Eq. (14), l < L, for the context's rho
static void rotation_tables(const fse_ctx* c, std::vector<double>& rc, std::vector<double>& rs) {
    const int L = c->p.L, dm1 = c->p.d - 1;
    rc.assign(std::max(L, 1), 0.0);
    rs.assign(std::max(L, 1), 0.0);
    for (int l = 0; l < L; ++l) {
        double th = 0.0;
        for (int j = 0; j < dm1; ++j) th += (double)c->ktab_host[(size_t)l * dm1 + j] * c->rho[j];
        th *= 2.0 * M_PI;
        rc[l] = cos(th);
        rs[l] = sin(th);
    }
}

// dofs of a nonlinear element type (FSE_NL_*)
static int host_elem_ndof(int type) {
    return (type == FSE_NL_CUBIC_GROUND || type == FSE_NL_VDP) ? 1 : (type == FSE_NL_CUBIC_DIFF ? 2 : 6);
}

static void free_ctx(fse_ctx* c) {
    if (!c) return;
    void* ptrs[] = {c->d.Mb, c->d.F, c->d.el_type, c->d.el_dof, c->d.el_p, c->d.col_off,
                    c->d.cs_ptr, c->d.cs_col, c->d.kt_slot, c->d.g_pass, c->d.g_info, c->d.g_rr, c->d.g_map, c->d.g_slot,
                    c->d.g_rec, c->d.cs_m, c->d.cs_d, c->d.cs_k, c->d.cs_s, c->d.cs_A,
                    c->d.cs_B, c->d.kt_ptr, c->d.kt_col, c->d.kt_soff, c->d.kt_src, c->d.ke,
                    c->d.kt_val, c->d.ce, c->d.ct_val, c->d.romega, c->d.phis, c->d.G, c->d.Gi, c->d.RG, c->d.rc, c->d.rs,
                    c->d.ktab, c->d.LMc, c->d.LMr, c->d.LMinv, c->d.q, c->d.u, c->d.a, c->d.zb,
                    c->d.Lc, c->d.Lr, c->d.Linv, c->d.Dinv, c->d.Rf, c->d.Rb, c->d.Tf, c->d.Tb, c->d.X, c->d.V, c->d.Y, c->d.Z0, c->d.R,
                    c->d.vec, c->d.vec2, c->d.yb, c->d.status, c->d.iters, c->d.nref, c->d.flag, c->Jd, c->piv, c->kry, c->kdot,
                    c->ht, c->unk, c->d.Sband, c->d.ktc_ptr, c->d.ktc_e, c->d.ktc_c, c->d.ktc_r};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto* v : {&c->pev, &c->ev_state, &c->ev_sens})
        for (auto& e : *v)
            if (e) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    delete c;
}

static int setup_impl(const fse_model* m, const fse_opts* o, long long s_begin, long long s_end, int device,
                      fse_ctx** out);

extern "C" int fse_setup(const fse_model* m, const fse_opts* o, int device, fse_ctx** out) {
    return setup_impl(m, o, 0, -1, device, out);
}

extern "C" int fse_setup_shard(const fse_model* m, const fse_opts* o, int s_begin, int s_end, int device,
                               fse_ctx** out) {
    if (out) *out = nullptr;
    if (s_begin < 0 || s_end <= s_begin) return set_err(nullptr, FSE_EINVAL, "need 0 <= s_begin < s_end");
    return setup_impl(m, o, s_begin, s_end, device, out);
}

// s_end < 0: every trajectory (s_begin = 0)
static int setup_impl(const fse_model* m, const fse_opts* o, long long s_begin, long long s_end, int device,
                      fse_ctx** out) {
    if (!out) return set_err(nullptr, FSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!m || !o) return set_err(nullptr, FSE_EINVAL, "model or opts is NULL");
    const int n = m->n;
    if (n < 1 || !m->M || !m->D || !m->K) return set_err(nullptr, FSE_EINVAL, "bad n or matrix pointer");
    if (o->d < 2 || o->d > FSE_MAX_D) return set_err(nullptr, FSE_EINVAL, "d must be in [2, 4]");
    if (m->e < 1 || m->e > o->d || !m->F) return set_err(nullptr, FSE_EINVAL, "need 1 <= e <= d and F");
    if (m->n_nl < 0 || (m->n_nl > 0 && !m->nl)) return set_err(nullptr, FSE_EINVAL, "bad nonlinear element list");
    if (!o->S || !o->H || !o->rho) return set_err(nullptr, FSE_EINVAL, "S, H, rho required");
    if (o->S1 < 2) return set_err(nullptr, FSE_EINVAL, "S1 must be >= 2");
    if (o->newton_maxit < 1 || o->newton_maxit > 64) return set_err(nullptr, FSE_EINVAL, "newton_maxit in [1, 64]");
    if (o->precision != FSE_FP64 && o->precision != FSE_MIXED_FP32)
        return set_err(nullptr, FSE_EINVAL, "unknown precision");
    std::vector<int> S(o->S, o->S + o->d - 1), H(o->H, o->H + o->d - 1);
    long long N = 1, U = 1;
    for (int j = 0; j < o->d - 1; ++j) {
        if (H[j] < 0 || S[j] < 1) return set_err(nullptr, FSE_EINVAL, "bad S_j or H_j");
        if (S[j] < 2 * H[j] + 1)
            return set_err(nullptr, FSE_EINVAL, "sampling rule S_j >= 2 H_j + 1 violated (Sec. 3.1)");
        N *= S[j];
        U *= 2 * H[j] + 1;
    }
    if (N > 65535 || U > 65535) return set_err(nullptr, FSE_EINVAL, "N or U too large");
    // trajectory shard [s_begin, s_end) of the N-sample grid (the whole grid by default)
    const long long Nglob = N;
    if (s_end < 0) {
        s_begin = 0;
        s_end = Nglob;
    }
    if (s_end > Nglob) return set_err(nullptr, FSE_EINVAL, "shard beyond the trajectory grid");
    N = s_end - s_begin;
    for (int j = 0; j < o->d - 1; ++j)
        if (!std::isfinite(o->rho[j])) return set_err(nullptr, FSE_EINVAL, "rho not finite");
    // half-bandwidth from exact zeros and element spans
    int b = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const size_t o2 = (size_t)i * n + j;
            if (m->M[o2] != 0.0 || m->D[o2] != 0.0 || m->K[o2] != 0.0) b = std::max(b, std::abs(i - j));
        }
    for (int e = 0; e < m->n_nl; ++e) {
        const fse_nl_elem& el = m->nl[e];
        if (el.type < 1 || el.type > 4) return set_err(nullptr, FSE_EINVAL, "unknown element type");
        const int nd = host_elem_ndof(el.type);
        for (int a = 0; a < nd; ++a) {
            if (el.dof[a] >= n || el.dof[a] < -1) return set_err(nullptr, FSE_EINVAL, "element dof out of range");
            if (el.type != 3 && el.dof[a] < 0) return set_err(nullptr, FSE_EINVAL, "spring dof must be >= 0");
            for (int c2 = 0; c2 < nd; ++c2)
                if (el.dof[a] >= 0 && el.dof[c2] >= 0) b = std::max(b, std::abs(el.dof[a] - el.dof[c2]));
        }
        if (el.type == 3 && !(el.p[1] > 0.0)) return set_err(nullptr, FSE_EINVAL, "beam element length must be > 0");
    }
    fse_ctx* c = new (std::nothrow) fse_ctx();
    if (!c) return set_err(nullptr, FSE_ENOMEM, "host allocation failed");
    Params& p = c->p;
    p.n = n;
    p.b = b;
    p.d = o->d;
    p.e = m->e;
    p.N = (int)N;
    p.N_glob = (int)Nglob;
    p.s0 = (int)s_begin;
    p.shard = N != Nglob;
    p.U = (int)U;
    p.L = (int)(U - 1) / 2;
    p.S1 = o->S1;
    p.P = 2 * n + 1;
    p.maxit = o->newton_maxit;
    p.prec = o->precision;
    p.tol = o->newton_tol;
    p.n_el = m->n_nl;
    for (int e = 0; e < m->n_nl; ++e)
        if (m->nl[e].type == FSE_NL_VDP) p.has_vel = true;
    const size_t tsz = p.prec == FSE_MIXED_FP32 ? 4 : 8;
    const int nb = b + 1;
    for (int j = 0; j < o->d - 1; ++j) c->rho.push_back(o->rho[j]);
    if (device >= 0) {
        if (cudaSetDevice(device) != cudaSuccess) {
            free_ctx(c);
            return set_err(nullptr, FSE_ECUDA, "cudaSetDevice failed");
        }
        c->device = device;
    } else {
        cudaGetDevice(&c->device);
    }
    int rc = cuda_check(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
    if (rc == FSE_OK) rc = cuda_check(c, cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking), "stream");
    if (rc) {
        g_setup_err = c->err;
        free_ctx(c);
        return rc;
    }
    for (auto& e : c->ev) cudaEventCreateWithFlags(&e, cudaEventDefault);
    // ordering events of the two-stream step loop (one pair per Newmark step)
    c->ev_state.assign(p.S1, nullptr);
    c->ev_sens.assign(p.S1, nullptr);
    for (int k = 0; k < p.S1; ++k) {
        cudaEventCreateWithFlags(&c->ev_state[k], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_sens[k], cudaEventDisableTiming);
    }
    // harmonic table
    auto rows = harmonic_rows(H);
    const int dm1 = p.d - 1;
    c->ktab_host.resize((size_t)rows.size() * dm1);
    for (size_t r = 0; r < rows.size(); ++r)
        for (int j = 0; j < dm1; ++j) c->ktab_host[r * dm1 + j] = rows[r][j];
    // sample grid (Eq. D1): phi_2 fastest
    std::vector<double> phis((size_t)N * dm1);
    for (long long s = 0; s < N; ++s) {
        long long rem = s_begin + s;
        for (int j = 0; j < dm1; ++j) {
            const long long ij = rem % S[j];
            rem /= S[j];
            phis[s * dm1 + j] = 2.0 * M_PI * (double)ij / (double)S[j];
        }
    }
    // rotation angles 2 pi k~_l . rho (Eq. 14)
    std::vector<double> rcv, rsv;
    rotation_tables(c, rcv, rsv);
    // diagonal-major full band of M (for its factor) and the CSR of the union pattern of M, D, K
    const int fb = 2 * b + 1;
    std::vector<double> Mb((size_t)fb * n, 0.0);
    std::vector<int> cptr(n + 1, 0), ccol;
    std::vector<double> cm, cd, ck;
    for (int i = 0; i < n; ++i) {
        for (int j = std::max(0, i - b); j <= std::min(n - 1, i + b); ++j) {
            const size_t o2 = (size_t)i * n + j;
            Mb[(size_t)(j - i + b) * n + i] = m->M[o2];
            if (m->M[o2] != 0.0 || m->D[o2] != 0.0 || m->K[o2] != 0.0) {
                ccol.push_back(j);
                cm.push_back(m->M[o2]);
                cd.push_back(m->D[o2]);
                ck.push_back(m->K[o2]);
            }
        }
        cptr[i + 1] = (int)ccol.size();
    }
    p.nnz = (int)ccol.size();
    // colour the elements so that no two of a colour share a dof
    std::vector<int> color(m->n_nl, 0);
    std::vector<uint64_t> used(n, 0);
    int ncol = 0;
    for (int e = 0; e < m->n_nl; ++e) {
        const fse_nl_elem& el = m->nl[e];
        const int nd = host_elem_ndof(el.type);
        uint64_t mask = 0;
        for (int a = 0; a < nd; ++a)
            if (el.dof[a] >= 0) mask |= used[el.dof[a]];
        int cl = 0;
        while (cl < 64 && (mask >> cl) & 1ull) ++cl;
        if (cl >= 64) {
            free_ctx(c);
            return set_err(nullptr, FSE_EINVAL, "element graph needs more than 64 colours");
        }
        color[e] = cl;
        ncol = std::max(ncol, cl + 1);
        for (int a = 0; a < nd; ++a)
            if (el.dof[a] >= 0) used[el.dof[a]] |= (1ull << cl);
    }
    p.ncolors = ncol;
    std::vector<int> order(m->n_nl);
    for (int e = 0; e < m->n_nl; ++e) order[e] = e;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return color[x] < color[y]; });
    std::vector<int> et(m->n_nl), ed((size_t)6 * m->n_nl), coff(ncol + 1, 0);
    std::vector<double> ep((size_t)6 * m->n_nl);
    for (int k = 0; k < m->n_nl; ++k) {
        const fse_nl_elem& el = m->nl[order[k]];
        et[k] = el.type;
        for (int a = 0; a < 6; ++a) {
            ed[(size_t)6 * k + a] = el.dof[a];
            ep[(size_t)6 * k + a] = el.p[a];
        }
        coff[color[order[k]] + 1]++;
    }
    for (int cl = 0; cl < ncol; ++cl) coff[cl + 1] += coff[cl];
    // CSR pattern of K_t: entry (dof_a, dof_b) for every element and local pair; each entry
    // keeps its sources (element in sorted order, a, b) in increasing element order
    std::vector<std::vector<std::pair<int, int>>> ktrow(n);   // (col, source)
    for (int k = 0; k < m->n_nl; ++k) {
        const int nd = et[k] == 1 ? 1 : (et[k] == 2 ? 2 : 6);
        for (int a = 0; a < nd; ++a)
            for (int bb = 0; bb < nd; ++bb) {
                const int ga = ed[(size_t)6 * k + a], gb = ed[(size_t)6 * k + bb];
                if (ga >= 0 && gb >= 0) ktrow[ga].push_back({gb, k * 36 + a * 6 + bb});
            }
    }
    std::vector<int> kptr(n + 1, 0), kcol, ksoff(1, 0), ksrc;
    for (int i = 0; i < n; ++i) {
        auto& r = ktrow[i];
        std::stable_sort(r.begin(), r.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
            return x.first < y.first;
        });
        for (size_t q = 0; q < r.size(); ++q) {
            if (q == 0 || r[q].first != r[q - 1].first) {
                kcol.push_back(r[q].first);
                ksoff.push_back(ksoff.back());
            }
            ksrc.push_back(r[q].second);
            ksoff.back()++;
        }
        kptr[i + 1] = (int)kcol.size();
    }
    p.nnz_kt = (int)kcol.size();
    p.nblk = (n + FSE_BLK - 1) / FSE_BLK;
    p.RECE = ((b + 3) & ~3) * FSE_BLK + FSE_BLK * FSE_BLK;
    p.ND = (b + FSE_BLK - 1) / FSE_BLK;
    p.tc_ok = p.prec == FSE_MIXED_FP32 && b <= 96;
    p.ld = (p.P + 3) & ~3;
    // row groups: R chosen by the shared-memory wavefronts per 64-column pass of an entry
    // (4 for the X and V elements, RB / 16 for the broadcast record)
    RowGroups grp;
    {
        double best = 0.0;
        for (int R = 1; R <= FSE_RHS_MAXR; ++R) {
            RowGroups cand = group_rows(n, cptr, ccol, R);
            const double cost = (double)cand.col.size() * (4.0 + group_record_bytes(R, tsz) / 16.0);
            if (R == 1 || cost < best) {
                best = cost;
                grp = std::move(cand);
            }
        }
    }
    p.R = grp.R;
    p.ng = (int)grp.ptr.size() - 1;
    p.nE = (int)grp.col.size();
    p.RB = group_record_bytes(p.R, tsz);
    // per pass of FSE_RHS_GPS groups: rows that must be staged (monotone), entries, ring span
    const int npass = (p.ng + FSE_RHS_GPS - 1) / FSE_RHS_GPS;
    std::vector<int> ghi(npass), gmin(npass);
    {
        int hi = 0;
        for (int ps = 0; ps < npass; ++ps) {
            const int g0 = ps * FSE_RHS_GPS, g1 = std::min(p.ng, g0 + FSE_RHS_GPS);
            int mx = 0;
            for (int g = g0; g < g1; ++g)
                for (int r = 0; r < p.R; ++r) mx = std::max(mx, grp.rows[(size_t)g * p.R + r]);
            hi = std::max(hi, std::min(n, mx + b + 1));
            ghi[ps] = hi;
            gmin[ps] = grp.rows[(size_t)g0 * p.R];
            p.ME = std::max(p.ME, grp.ptr[g1] - grp.ptr[g0]);
        }
        // rows are staged in 32-row TMA boxes: the ring (a multiple of 32 rows) holds from the
        // first row a pass reads up to the last box staged for the passes in flight
        const int dep = p.prec == FSE_MIXED_FP32 ? FSE_RHS_DEPTH_F32 : FSE_RHS_DEPTH_F64;
        p.RW = 32;
        for (int ps = 0; ps < npass; ++ps) {
            const int top = (ghi[std::min(ps + dep, npass - 1)] + 31) & ~31;
            p.RW = std::max(p.RW, top - std::max(0, gmin[ps] - b));
        }
        p.RW = (p.RW + 31) & ~31;
    }
    p.RWT = 1;
    while (p.RWT < b + FSE_BLK) p.RWT <<= 1;
    // per pass: {rows to stage, first entry, end entry, first K_t entry}, {K_t entries, first
    // group, 0, 0}; the K_t slice of a pass starts at a multiple of 4 and has a multiple of 4
    // entries (16-byte bulk copies); per group: {first entry relative to its pass, entries};
    // per row: {row, K_t begin, K_t end (relative to the pass's slice), 0}
    p.kt_ld = std::max(4, (p.nnz_kt + 3) & ~3);
    std::vector<int> gpass((size_t)8 * npass, 0), ginfo((size_t)2 * ((p.ng + 1) & ~1), 0);
    std::vector<int> grr((size_t)p.ng * p.R * 4, 0);
    p.MK = 0;
    for (int ps = 0; ps < npass; ++ps) {
        const int g0 = ps * FSE_RHS_GPS, g1 = std::min(p.ng, g0 + FSE_RHS_GPS);
        int k0 = p.nnz_kt, k1 = 0;
        for (int g = g0; g < g1; ++g)
            for (int r = 0; r < p.R; ++r) {
                const int i = grp.rows[(size_t)g * p.R + r];
                if (i < 0) continue;
                k0 = std::min(k0, kptr[i]);
                k1 = std::max(k1, kptr[i + 1]);
            }
        const int kb = k1 > k0 ? (k0 & ~3) : 0;
        const int kn = k1 > k0 ? ((k1 - kb + 3) & ~3) : 0;
        p.MK = std::max(p.MK, kn);
        int* d = &gpass[(size_t)8 * ps];
        d[0] = ghi[ps];
        d[1] = grp.ptr[g0];
        d[2] = grp.ptr[g1];
        d[3] = kb;
        d[4] = kn;
        d[5] = g0;
        for (int g = g0; g < g1; ++g) {
            ginfo[(size_t)2 * g] = grp.ptr[g] - grp.ptr[g0];
            ginfo[(size_t)2 * g + 1] = grp.ptr[g + 1] - grp.ptr[g];
            for (int r = 0; r < p.R; ++r) {
                const size_t q = (size_t)g * p.R + r;
                const int i = grp.rows[q];
                grr[4 * q] = i;
                grr[4 * q + 1] = i >= 0 ? kptr[i] - kb : 0;
                grr[4 * q + 2] = i >= 0 ? kptr[i + 1] - kb : 0;
            }
        }
    }
    std::vector<int> gslot(grp.col.size()), kslot(p.kt_ld, 0);
    for (size_t q = 0; q < grp.col.size(); ++q) gslot[q] = grp.col[q] % p.RW;
    for (size_t q = 0; q < kcol.size(); ++q) kslot[q] = kcol[q] % p.RW;
    // panel Cholesky in the state kernel for FP32 factors with b <= 96 when its window fits
    p.chol_blk = 0;
    if (p.prec == FSE_MIXED_FP32 && b <= 96) {
        p.chol_blk = 1;
        if (fse::state_smem(p) > 220 * 1024) p.chol_blk = 0;
    }
    p.smem_state = fse::state_smem(p);
    p.smem_rhs = fse::rhs_smem(p);
    p.smem_trsm = fse::trsm_smem(p);
    const size_t lim = 220 * 1024;
    if (b > FSE_MAX_BAND || p.smem_state > lim || p.smem_rhs > lim || p.smem_trsm > lim ||
        (size_t)(nb + 9) * nb * sizeof(double) > lim) {
        free_ctx(c);
        return set_err(nullptr, FSE_EINVAL, "n or half-bandwidth too large for the on-chip working set");
    }
    // device allocations
    const size_t Nn = (size_t)N * n, band = (size_t)fb * n, lb = (size_t)n * nb;
    const size_t sensz = (size_t)N * n * p.ld * tsz;
    const size_t ktsz = (size_t)N * p.kt_ld * tsz;
    const size_t dsz = (size_t)N * p.nblk * FSE_BLK * FSE_BLK * tsz;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** ptr, size_t bytes) {
        if (e == cudaSuccess) e = dalloc(ptr, bytes);
    };
    A(&c->d.Mb, band * 8);
    A(&c->d.F, (size_t)m->e * n * 8);
    A(&c->d.el_type, (size_t)std::max(1, m->n_nl) * 4);
    A(&c->d.el_dof, (size_t)std::max(1, m->n_nl) * 24);
    A(&c->d.el_p, (size_t)std::max(1, m->n_nl) * 48);
    A(&c->d.col_off, (size_t)(ncol + 1) * 4);
    A(&c->d.cs_ptr, (size_t)(n + 1) * 4);
    A(&c->d.cs_col, (size_t)p.nnz * 4);
    A(&c->d.g_pass, gpass.size() * 4);
    A(&c->d.g_info, ginfo.size() * 4);
    A(&c->d.g_rr, (size_t)p.ng * p.R * 16);
    A(&c->d.g_map, (size_t)p.nE * p.R * 4);
    A(&c->d.g_slot, (size_t)p.nE * 4);
    A(&c->d.g_rec, (size_t)p.nE * p.RB);
    A(&c->d.kt_slot, (size_t)p.kt_ld * 4);
    A(&c->d.cs_m, (size_t)p.nnz * 8);
    A(&c->d.cs_d, (size_t)p.nnz * 8);
    A(&c->d.cs_k, (size_t)p.nnz * 8);
    A(&c->d.cs_s, (size_t)p.nnz * 8);
    A(&c->d.cs_A, (size_t)p.nnz * tsz);
    A(&c->d.cs_B, (size_t)p.nnz * tsz);
    A(&c->d.kt_ptr, (size_t)(n + 1) * 4);
    // panel factor: K_t entries of the lower triangle grouped by column
    std::vector<int> ktc_ptr(n + 1, 0), ktc_e, ktc_c, ktc_r;
    if (p.chol_blk) {
        for (int i = 0; i < n; ++i)
            for (int e = kptr[i]; e < kptr[i + 1]; ++e)
                if (kcol[e] <= i) ++ktc_ptr[kcol[e] + 1];
        for (int j = 0; j < n; ++j) ktc_ptr[j + 1] += ktc_ptr[j];
        const int nl = ktc_ptr[n];
        ktc_e.assign(std::max(1, nl), 0);
        ktc_c.assign(std::max(1, nl), 0);
        ktc_r.assign(std::max(1, nl), 0);
        std::vector<int> fill(ktc_ptr.begin(), ktc_ptr.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int e = kptr[i]; e < kptr[i + 1]; ++e) {
                const int j = kcol[e];
                if (j > i) continue;
                const int k = fill[j]++;
                ktc_e[k] = e;
                ktc_c[k] = j;
                ktc_r[k] = i - j;
            }
        A(&c->d.Sband, (size_t)n * nb * 4);
        A(&c->d.ktc_ptr, (size_t)(n + 1) * 4);
        A(&c->d.ktc_e, ktc_e.size() * 4);
        A(&c->d.ktc_c, ktc_c.size() * 4);
        A(&c->d.ktc_r, ktc_r.size() * 4);
    }
    A(&c->d.kt_col, (size_t)std::max(1, p.nnz_kt) * 4);
    A(&c->d.kt_soff, (size_t)(p.nnz_kt + 1) * 4);
    A(&c->d.kt_src, (size_t)std::max<size_t>(1, ksrc.size()) * 4);
    A(&c->d.ke, (size_t)N * std::max(1, m->n_nl) * 36 * 8);
    A(&c->d.kt_val, FSE_NBUF_KT * ktsz);
    if (p.has_vel) {
        A(&c->d.ce, (size_t)N * std::max(1, m->n_nl) * 36 * 8);
        A(&c->d.ct_val, FSE_NBUF_KT * ktsz);
    }
    A(&c->d.romega, (size_t)2 * Nn * tsz);
    A(&c->d.phis, (size_t)N * dm1 * 8);
    A(&c->d.G, (size_t)N * U * 8);
    A(&c->d.Gi, (size_t)N * U * 8);
    A(&c->d.RG, (size_t)N * U * 8);
    A(&c->d.rc, rcv.size() * 8);
    A(&c->d.rs, rsv.size() * 8);
    A(&c->d.ktab, c->ktab_host.size() * 4);
    A(&c->d.LMc, lb * 8);
    A(&c->d.LMr, lb * 8);
    A(&c->d.LMinv, (size_t)n * 8);
    A(&c->d.q, Nn * 8);
    A(&c->d.u, Nn * 8);
    A(&c->d.a, Nn * 8);
    A(&c->d.zb, Nn * 16);
    A(&c->d.yb, Nn * 16);
    A(&c->d.Lc, FSE_NBUF_F * (size_t)N * lb * tsz);
    A(&c->d.Lr, FSE_NBUF_F * (size_t)N * lb * tsz);
    A(&c->d.Linv, FSE_NBUF_F * Nn * tsz);
    A(&c->d.Dinv, FSE_NBUF_F * dsz);
    const size_t rsz = (size_t)N * p.nblk * p.RECE * tsz;
    A(&c->d.Rf, FSE_NBUF_F * rsz);
    A(&c->d.Rb, FSE_NBUF_F * rsz);
    if (p.tc_ok) {
        const size_t tcsz = (size_t)2 * N * (p.nblk + 1) * 8 * FSE_BLK * FSE_BLK * 4;   // two step parities
        A(&c->d.Tf, tcsz);
        A(&c->d.Tb, tcsz);
    }
    A(&c->d.X, sensz);
    A(&c->d.V, sensz);
    A(&c->d.Y, sensz);
    const size_t nu = (size_t)2 * n * U;
    A(&c->d.Z0, nu * 8);
    A(&c->d.R, nu * 8);
    A(&c->d.vec, nu * 8);
    A(&c->d.vec2, nu * 8);
    A(&c->d.status, (size_t)N * 4);
    A(&c->d.iters, (size_t)N * 4);
    A(&c->d.nref, (size_t)N * 4);
    A(&c->d.flag, 16);
    if (e != cudaSuccess) {
        rc = cuda_check(c, e, "device allocation");
        g_setup_err = c->err;
        free_ctx(c);
        return rc;
    }
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(c->d.Mb, Mb.data(), band * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.F, m->F, (size_t)m->e * n * 8, cudaMemcpyHostToDevice, st);
    if (m->n_nl > 0) {
        cudaMemcpyAsync(c->d.el_type, et.data(), et.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d.el_dof, ed.data(), ed.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d.el_p, ep.data(), ep.size() * 8, cudaMemcpyHostToDevice, st);
    }
    cudaMemcpyAsync(c->d.col_off, coff.data(), coff.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.cs_ptr, cptr.data(), cptr.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.cs_col, ccol.data(), ccol.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.g_pass, gpass.data(), gpass.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.g_info, ginfo.data(), ginfo.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.g_rr, grr.data(), grr.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.g_map, grp.map.data(), grp.map.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.g_slot, gslot.data(), gslot.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.kt_slot, kslot.data(), kslot.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(c->d.kt_val, 0, FSE_NBUF_KT * ktsz, st);
    if (p.has_vel) cudaMemsetAsync(c->d.ct_val, 0, FSE_NBUF_KT * ktsz, st);
    cudaMemcpyAsync(c->d.cs_m, cm.data(), cm.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.cs_d, cd.data(), cd.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.cs_k, ck.data(), ck.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.kt_ptr, kptr.data(), kptr.size() * 4, cudaMemcpyHostToDevice, st);
    if (p.chol_blk) {
        cudaMemcpyAsync(c->d.ktc_ptr, ktc_ptr.data(), ktc_ptr.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d.ktc_e, ktc_e.data(), ktc_e.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d.ktc_c, ktc_c.data(), ktc_c.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d.ktc_r, ktc_r.data(), ktc_r.size() * 4, cudaMemcpyHostToDevice, st);
    }
    if (p.nnz_kt > 0) {
        cudaMemcpyAsync(c->d.kt_col, kcol.data(), kcol.size() * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(c->d.kt_src, ksrc.data(), ksrc.size() * 4, cudaMemcpyHostToDevice, st);
    }
    cudaMemcpyAsync(c->d.kt_soff, ksoff.data(), ksoff.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.phis, phis.data(), phis.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.rc, rcv.data(), rcv.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.rs, rsv.data(), rsv.size() * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d.ktab, c->ktab_host.data(), c->ktab_host.size() * 4, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(c->d.status, 0, (size_t)N * 4, st);
    cudaMemsetAsync(c->d.iters, 0, (size_t)N * 4, st);
    cudaMemsetAsync(c->d.nref, 0, (size_t)N * 4, st);
    cudaMemsetAsync(c->d.flag, 0, 16, st);
    cudaMemsetAsync(c->d.Rf, 0, FSE_NBUF_F * rsz, st);   // entries outside the band stay zero
    cudaMemsetAsync(c->d.Rb, 0, FSE_NBUF_F * rsz, st);
    if (fse::make_tangent_maps(c) != FSE_OK) {
        rc = set_err(c, FSE_ECUDA, "TMA descriptor encoding failed");
        g_setup_err = c->err;
        free_ctx(c);
        return rc;
    }
    fse::launch_fill_tables(c);
    const int bad = fse::launch_factor_M(c);
    rc = cuda_check(c, cudaStreamSynchronize(st), "setup");
    if (rc == FSE_OK) rc = cuda_check(c, cudaGetLastError(), "setup kernels");
    if (rc == FSE_OK && bad) rc = set_err(c, FSE_ENONPOS_PIVOT, "mass matrix is not positive definite");
    if (rc) {
        g_setup_err = c->err;
        free_ctx(c);
        return rc;
    }
    *out = c;
    return FSE_OK;
}

extern "C" void fse_destroy(fse_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

extern "C" const char* fse_last_error(const fse_ctx* c) {
    return c ? c->err.c_str() : g_setup_err.c_str();
}

extern "C" int fse_sizes(const fse_ctx* c, int* nu, int* U, int* N, int* n, int* band) {
    if (!c) return FSE_EINVAL;
    if (nu) *nu = 2 * c->p.n * c->p.U;
    if (U) *U = c->p.U;
    if (N) *N = c->p.N;
    if (n) *n = c->p.n;
    if (band) *band = c->p.b;
    return FSE_OK;
}

extern "C" int fse_harmonics(const fse_ctx* c, int* kt) {
    if (!c || !kt) return FSE_EINVAL;
    std::memcpy(kt, c->ktab_host.data(), c->ktab_host.size() * sizeof(int));
    return FSE_OK;
}

// Trajectory shards: the partial DFT sums in buf (count doubles) become the whole torus's sums
// through the context's reduction, then sub (nullable) is subtracted.  Without a reduction the
// partial sums are the result.  Synchronous (the reduction runs on the host).
static int shard_complete(fse_ctx* c, double* buf, size_t count, const double* sub) {
    if (!c->p.shard || !c->reduce) return FSE_OK;
    int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "shard partial sums");
    if (rc) return rc;
    if (c->reduce(c->reduce_user, buf, count, (void*)c->stream) != 0) {
        c->reduce_failed = true;
        return set_err(c, FSE_ECUDA, "shard reduction failed");
    }
    if (sub) fse::vec_axpby(c, count, -1.0, sub, 1.0, buf);
    return FSE_OK;
}

// out = (I (x) R Gamma^-1) zb - sub, or on a shard the completed sum minus sub
static int dft_sub(fse_ctx* c, const double* zb, const double* sub, double* out) {
    const size_t nu = (size_t)2 * c->p.n * c->p.U;
    fse::launch_dft_residual(c, zb, sub, out, (sub && !c->p.shard) ? 1 : 0);
    return shard_complete(c, out, nu, sub);
}

// R_T = Gamma R(rho) Gamma^-1 zbar(2 pi) - zbar(0) of Eq. FSES_T from the end points in d.zb:
// DFT + rotation into the coefficient scratch, i-DFT back to the samples, minus the start points
static int hypertime_residual(fse_ctx* c, const double* zb0_dev, double* RT_dev) {
    const Params& p = c->p;
    double* coef = c->ht + (size_t)4 * p.N * 2 * p.n;
    const int rc = dft_sub(c, c->d.zb, nullptr, coef);
    if (rc) return rc;
    fse::launch_idft(c, coef, RT_dev);
    fse::vec_axpby(c, (size_t)p.N * 2 * p.n, -1.0, zb0_dev, 1.0, RT_dev);
    return FSE_OK;
}

// the whole evaluation, asynchronous on the context stream.  The trajectories start from the
// i-DFT of the coefficients Z0_dev (Eq. 20), or, when zb0_dev is given, from the start points
// zbar(0) themselves (the hyper-time form of Sec. 3.4, N x 2n): then R_dev receives R_T.
static int run_eval(fse_ctx* c, const double* Z0_dev, double w, double* R_dev, int sens,
                    const double* zb0_dev = nullptr) {
    if (!(w > 0.0) || !std::isfinite(w)) return set_err(c, FSE_EINVAL, "omega1 must be positive and finite");
    cudaSetDevice(c->device);
    const Params& p = c->p;
    if (w != c->omega_S) {
        fse::launch_build_ops(c, w);
        fse::launch_build_groups(c);
        c->omega_S = w;
    }
    const int steps = (c->n_steps > 0 && c->n_steps < p.S1) ? c->n_steps : p.S1;
    if ((int)c->ev_state.size() < steps) {
        for (int k = (int)c->ev_state.size(); k < steps; ++k) {
            cudaEvent_t a = nullptr, b2 = nullptr;
            cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
            cudaEventCreateWithFlags(&b2, cudaEventDisableTiming);
            c->ev_state.push_back(a);
            c->ev_sens.push_back(b2);
        }
    }
    const bool prof = c->prof && (int)c->pev.size() == 8 * p.S1;
    auto rec = [&](int phase, int k, int end, cudaStream_t st) {
        if (prof) cudaEventRecord(c->pev[((size_t)phase * p.S1 + k) * 2 + end], st);
    };
    cudaStream_t s1 = c->stream, s2 = c->stream2;
    cudaEventRecord(c->ev[0], s1);
    if (zb0_dev)
        cudaMemcpyAsync(c->d.zb, zb0_dev, (size_t)p.N * 2 * p.n * 8, cudaMemcpyDeviceToDevice, s1);
    else
        fse::launch_idft(c, Z0_dev, c->d.zb);
    fse::launch_init_state(c, w);
    if (sens) {
        cudaEventRecord(c->ev[2], s1);
        cudaStreamWaitEvent(s2, c->ev[2], 0);
        fse::launch_sens_init(c, s2);
    }
    // state step k (stream 1) writes the factor and w_1-term buffers k % 2 and the tangent
    // values (k + 1) % 3, which the sensitivity step k - 2 (stream 2) reads: it waits for it.
    // The sensitivity step k waits for the state step k; so state k + 1 overlaps sensitivity k.
    for (int k = 0; k < steps; ++k) {
        if (sens && k >= 2) cudaStreamWaitEvent(s1, c->ev_sens[k - 2], 0);
        rec(0, k, 0, s1);
        fse::launch_state_step(c, k, w, s1, sens != 0);
        rec(0, k, 1, s1);
        if (sens) {
            cudaEventRecord(c->ev_state[k], s1);
            cudaStreamWaitEvent(s2, c->ev_state[k], 0);
            for (int ph = 0; ph < 3; ++ph) {
                rec(1 + ph, k, 0, s2);
                fse::launch_sens_phase(c, k, w, ph, s2);
                rec(1 + ph, k, 1, s2);
            }
            cudaEventRecord(c->ev_sens[k], s2);
        }
    }
    c->prof_pending = prof;
    c->prof_sens = sens != 0;
    c->prof_steps = steps;
    fse::launch_collect_end(c);
    const int rcd = zb0_dev ? hypertime_residual(c, zb0_dev, R_dev) : dft_sub(c, c->d.zb, Z0_dev, R_dev);
    if (rcd) return rcd;
    if (sens) cudaStreamWaitEvent(s1, c->ev_sens[steps - 1], 0);
    cudaEventRecord(c->ev[1], s1);
    c->have_jac = sens != 0;
    c->omega_jac = w;
    return cuda_check(c, cudaGetLastError(), "evaluation launch");
}

static int collect_status(fse_ctx* c, int* ts, int* it) {
    const int N = c->p.N;
    std::vector<int> st(N), its(N);
    int flag = 0;
    cudaMemcpyAsync(st.data(), c->d.status, N * 4, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(its.data(), c->d.iters, N * 4, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&flag, c->d.flag, 4, cudaMemcpyDeviceToHost, c->stream);
    int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "evaluation");
    if (rc) return rc;
    if (flag) {
        cudaMemsetAsync(c->d.flag, 0, 4, c->stream);
        return set_err(c, FSE_ECUDA, "a pipeline wait of the tangent kernels timed out");
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess)
        c->timing[0] = ms;
    else
        cudaGetLastError();   // no timing for an evaluation replayed from a graph: clear that error
    if (c->prof_pending) {
        const int S1 = c->p.S1;
        const int steps = c->prof_steps;
        for (int ph = 0; ph < 4; ++ph) {
            double tot = 0.0;
            if (ph == 0 || c->prof_sens)
                for (int k = 0; k < steps; ++k) {
                    float t = 0.f;
                    cudaEventElapsedTime(&t, c->pev[((size_t)ph * S1 + k) * 2], c->pev[((size_t)ph * S1 + k) * 2 + 1]);
                    tot += t;
                }
            c->timing[1 + ph] = tot;
        }
        c->prof_pending = false;
        std::vector<int> nr(N);
        cudaMemcpy(nr.data(), c->d.nref, N * 4, cudaMemcpyDeviceToHost);
        double tot = 0.0;
        for (int x : nr) tot += x;
        c->timing[5] = steps > 0 ? tot / ((double)N * steps) : 0.0;
    }
    if (ts) std::memcpy(ts, st.data(), N * 4);
    if (it) std::memcpy(it, its.data(), N * 4);
    int worst = FSE_OK;
    for (int s = 0; s < N; ++s)
        if (st[s] != FSE_OK && (worst == FSE_OK || st[s] < worst)) worst = st[s];
    if (worst == FSE_ENOCONV) c->err = "per-step Newton did not converge on some trajectories";
    if (worst == FSE_ENONPOS_PIVOT) c->err = "effective stiffness lost positive definiteness";
    if (worst == FSE_ENAN) c->err = "non-finite values in the trajectory";
    return worst;
}

extern "C" int fse_residual_jacobian_dev(fse_ctx* c, const double* Z0_dev, double w, double* R_dev,
                                         int sens, void* stream) {
    if (!c || !Z0_dev || !R_dev) return FSE_EINVAL;
    // the caller's stream (NULL = the legacy default stream) is ordered before the evaluation
    // and waits for its end; the evaluation itself runs on the context's own streams
    cudaStream_t user = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    cudaEventRecord(c->ev[6], user);
    cudaStreamWaitEvent(c->stream, c->ev[6], 0);
    int rc = run_eval(c, Z0_dev, w, R_dev, sens);
    cudaEventRecord(c->ev[7], c->stream);
    cudaStreamWaitEvent(user, c->ev[7], 0);
    return rc;
}

extern "C" int fse_status(fse_ctx* c, int* ts, int* it) {
    if (!c) return FSE_EINVAL;
    return collect_status(c, ts, it);
}

extern "C" int fse_residual_jacobian(fse_ctx* c, const double* Z0, double w, double* R_out, int sens,
                                     int* ts, int* it) {
    if (!c || !Z0 || !R_out) return FSE_EINVAL;
    cudaSetDevice(c->device);
    const size_t nu = (size_t)2 * c->p.n * c->p.U;
    cudaMemcpyAsync(c->d.Z0, Z0, nu * 8, cudaMemcpyHostToDevice, c->stream);
    int rc = run_eval(c, c->d.Z0, w, c->d.R, sens);
    if (rc) return rc;
    cudaMemcpyAsync(R_out, c->d.R, nu * 8, cudaMemcpyDeviceToHost, c->stream);
    return collect_status(c, ts, it);
}

extern "C" int fse_jacobian_apply(fse_ctx* c, const double* v, double* Jv, int nvec) {
    if (!c || !v || !Jv || nvec < 0) return FSE_EINVAL;
    if (!c->have_jac) return set_err(c, FSE_ENOJAC, "no Jacobian stored: call fse_residual_jacobian with want_jacobian=1");
    cudaSetDevice(c->device);
    const size_t nu = (size_t)2 * c->p.n * c->p.U;
    for (int k = 0; k < nvec; ++k) {
        cudaMemcpyAsync(c->d.vec, v + k * nu, nu * 8, cudaMemcpyHostToDevice, c->stream);
        fse::launch_idft(c, c->d.vec, c->d.zb);
        fse::launch_phi_apply(c, c->d.zb, c->d.yb);
        const int rc = dft_sub(c, c->d.yb, c->d.vec, c->d.vec2);
        if (rc) return rc;
        cudaMemcpyAsync(Jv + k * nu, c->d.vec2, nu * 8, cudaMemcpyDeviceToHost, c->stream);
    }
    return cuda_check(c, cudaStreamSynchronize(c->stream), "jacobian_apply");
}

extern "C" int fse_jacobian_domega(fse_ctx* c, double* out) {
    if (!c || !out) return FSE_EINVAL;
    if (!c->have_jac) return set_err(c, FSE_ENOJAC, "no Jacobian stored");
    cudaSetDevice(c->device);
    const size_t nu = (size_t)2 * c->p.n * c->p.U;
    fse::launch_domega(c, c->d.yb);
    const int rc = dft_sub(c, c->d.yb, nullptr, c->d.vec2);
    if (rc) return rc;
    cudaMemcpyAsync(out, c->d.vec2, nu * 8, cudaMemcpyDeviceToHost, c->stream);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "jacobian_domega");
}

static int ensure_dense(fse_ctx* c, size_t m) {
    if (c->Jd_cap >= m * m) return FSE_OK;
    if (c->Jd) cudaFree(c->Jd);
    if (c->piv) cudaFree(c->piv);
    c->Jd = nullptr;
    c->piv = nullptr;
    c->Jd_cap = 0;
    cudaError_t e = cudaMalloc(&c->Jd, m * m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->piv, m * 4);
    if (e != cudaSuccess) return cuda_check(c, e, "dense Jacobian allocation");
    c->Jd_cap = m * m;
    return FSE_OK;
}

extern "C" int fse_jacobian_dense(fse_ctx* c, double* J) {
    if (c && c->p.shard) return set_err(c, FSE_EINVAL, "not available on a trajectory shard");
    if (!c || !J) return FSE_EINVAL;
    if (!c->have_jac) return set_err(c, FSE_ENOJAC, "no Jacobian stored");
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    if (m * m > (1ull << 31)) return set_err(c, FSE_EINVAL, "dense Jacobian too large");
    cudaSetDevice(c->device);
    int rc = ensure_dense(c, m);
    if (rc) return rc;
    fse::launch_dense_jac(c, c->Jd);
    cudaMemcpyAsync(J, c->Jd, m * m * 8, cudaMemcpyDeviceToHost, c->stream);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "jacobian_dense");
}

extern "C" int fse_monodromy(fse_ctx* c, double* Phi, double* dzdw) {
    if (!c) return FSE_EINVAL;
    if (!c->have_jac) return set_err(c, FSE_ENOJAC, "no Jacobian stored");
    cudaSetDevice(c->device);
    const size_t n2 = 2 * (size_t)c->p.n, N = c->p.N;
    double *dP = nullptr, *dz = nullptr;
    cudaError_t e = cudaMalloc(&dP, N * n2 * n2 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dz, N * n2 * 8);
    if (e != cudaSuccess) {
        if (dP) cudaFree(dP);
        return cuda_check(c, e, "monodromy buffer");
    }
    fse::launch_phi_copy(c, dP, dz);
    if (Phi) cudaMemcpyAsync(Phi, dP, N * n2 * n2 * 8, cudaMemcpyDeviceToHost, c->stream);
    if (dzdw) cudaMemcpyAsync(dzdw, dz, N * n2 * 8, cudaMemcpyDeviceToHost, c->stream);
    int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "monodromy");
    cudaFree(dP);
    cudaFree(dz);
    return rc;
}

extern "C" int fse_monodromy_traj(fse_ctx* c, int s, double* Phi, double* dzdw) {
    if (!c) return FSE_EINVAL;
    if (s < 0 || s >= c->p.N) return set_err(c, FSE_EINVAL, "trajectory index out of range");
    if (!c->have_jac) return set_err(c, FSE_ENOJAC, "no Jacobian stored");
    cudaSetDevice(c->device);
    const size_t n2 = 2 * (size_t)c->p.n;
    double *dP = nullptr, *dz = nullptr;
    cudaError_t e = cudaMalloc(&dP, n2 * n2 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dz, n2 * 8);
    if (e != cudaSuccess) {
        if (dP) cudaFree(dP);
        return cuda_check(c, e, "monodromy buffer");
    }
    fse::launch_phi_copy_one(c, s, dP, dz);
    if (Phi) cudaMemcpyAsync(Phi, dP, n2 * n2 * 8, cudaMemcpyDeviceToHost, c->stream);
    if (dzdw) cudaMemcpyAsync(dzdw, dz, n2 * 8, cudaMemcpyDeviceToHost, c->stream);
    int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "monodromy");
    cudaFree(dP);
    cudaFree(dz);
    return rc;
}

// ||R||_2 and ||Z(0)||_2 of the last evaluation (device reduction, two scalars back)
static int norms_RZ(fse_ctx* c, double* rn, double* zn) {
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    fse::vec_norms2(c, m, c->d.R, c->d.Z0, c->d.vec2);
    double h[2];
    cudaMemcpyAsync(h, c->d.vec2, 16, cudaMemcpyDeviceToHost, c->stream);
    const int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "norms");
    if (rn) *rn = std::sqrt(h[0]);
    if (zn) *zn = std::sqrt(h[1]);
    return rc;
}

// Residual (sens = 0) or residual + Jacobian (sens = 1) at the device iterate d.Z0
static int eval_at_iterate(fse_ctx* c, double w, int sens, double* rn, double* zn) {
    int rc = run_eval(c, c->d.Z0, w, c->d.R, sens);
    if (rc) return rc;
    const int st = collect_status(c, nullptr, nullptr);
    if (st < 0 && st != FSE_ENOCONV) return st;
    rc = norms_RZ(c, rn, zn);
    return rc ? rc : st;
}

// w = J v with the stored monodromies (Eq. 22): i-DFT, blockdiag(Phi_s), DFT + rotation, minus v
// (a failed shard reduction is recorded in c->reduce_failed for the caller)
static void jac_apply_dev(fse_ctx* c, const double* v, double* w) {
    fse::launch_idft(c, v, c->d.zb);
    fse::launch_phi_apply(c, c->d.zb, c->d.yb);
    dft_sub(c, c->d.yb, v, w);
}

// Restarted GMRES(m) on J x = b (b, x on the device, x0 = 0), FP64, classical Gram-Schmidt with
// one re-orthogonalisation pass; the small Hessenberg least-squares problem is reduced by
// Givens rotations on the host.  Returns FSE_OK, or FSE_ENOCONV when it stops above rtol.
static int gmres_dev(fse_ctx* c, size_t n, const std::function<void(const double*, double*)>& Av, const double* b,
                     double* x, double rtol, int m, int maxit, int* iters_out, double* relres_out) {
    if ((size_t)(m + 1) * n > c->kry_cap) {
        if (c->kry) cudaFree(c->kry);
        if (c->kdot) cudaFree(c->kdot);
        c->kry = nullptr;
        c->kdot = nullptr;
        c->kry_cap = 0;
        cudaError_t e = cudaMalloc(&c->kry, (size_t)(m + 1) * n * 8);
        if (e == cudaSuccess) e = cudaMalloc(&c->kdot, (size_t)2 * (m + 2) * 8);
        if (e != cudaSuccess) return cuda_check(c, e, "GMRES basis");
        c->kry_cap = (size_t)(m + 1) * n;
    }
    double* Vb = c->kry;
    double* hd = c->kdot;
    auto norm2 = [&](const double* v, double* out) -> int {
        fse::vec_norms2(c, n, v, nullptr, hd);
        double h2[2];
        cudaMemcpyAsync(h2, hd, 16, cudaMemcpyDeviceToHost, c->stream);
        const int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "GMRES norm");
        *out = std::sqrt(h2[0]);
        return rc;
    };
    cudaMemsetAsync(x, 0, n * 8, c->stream);
    double bn = 0.0;
    int rc = norm2(b, &bn);
    if (rc) return rc;
    int it = 0;
    double rel = 0.0;
    if (!(bn > 0.0)) {
        *iters_out = 0;
        *relres_out = 0.0;
        return FSE_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hcol(m + 2), h2(m + 2);
    bool first = true;
    while (it < maxit) {
        // r = b - J x  (x = 0 on the first cycle)
        double* v0 = Vb;
        if (first) {
            cudaMemcpyAsync(v0, b, n * 8, cudaMemcpyDeviceToDevice, c->stream);
        } else {
            Av(x, v0);
            fse::vec_axpby(c, n, 1.0, b, -1.0, v0);
        }
        first = false;
        double beta = 0.0;
        rc = norm2(v0, &beta);
        if (rc) return rc;
        rel = beta / bn;
        if (rel <= rtol) break;
        fse::vec_axpby(c, n, 0.0, v0, 1.0 / beta, v0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (; k < m && it < maxit; ++k) {
            double* w = Vb + (size_t)(k + 1) * n;
            Av(Vb + (size_t)k * n, w);
            ++it;
            // two passes of classical Gram-Schmidt against v_0..v_k
            std::fill(hcol.begin(), hcol.end(), 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                fse::vec_mdot(c, n, k + 1, Vb, w, hd);
                cudaMemcpyAsync(h2.data(), hd, (size_t)(k + 1) * 8, cudaMemcpyDeviceToHost, c->stream);
                rc = cuda_check(c, cudaStreamSynchronize(c->stream), "GMRES dots");
                if (rc) return rc;
                for (int i = 0; i <= k; ++i) {
                    hcol[i] += h2[i];
                    h2[i] = -h2[i];
                }
                cudaMemcpyAsync(hd + (m + 2), h2.data(), (size_t)(k + 1) * 8, cudaMemcpyHostToDevice, c->stream);
                fse::vec_mupdate(c, n, k + 1, Vb, hd + (m + 2), w);
            }
            double hn = 0.0;
            rc = norm2(w, &hn);
            if (rc) return rc;
            hcol[k + 1] = hn;
            if (hn > 0.0) fse::vec_axpby(c, n, 0.0, w, 1.0 / hn, w);
            // apply the previous rotations, then a new one that zeroes hcol[k + 1]
            for (int i = 0; i < k; ++i) {
                const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = t;
            }
            const double r = std::hypot(hcol[k], hcol[k + 1]);
            cs[k] = r > 0.0 ? hcol[k] / r : 1.0;
            sn[k] = r > 0.0 ? hcol[k + 1] / r : 0.0;
            hcol[k] = r;
            hcol[k + 1] = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = hcol[i];
            rel = std::fabs(g[k + 1]) / bn;
            if (rel <= rtol || hn == 0.0) {
                ++k;
                break;
            }
        }
        // x += V_k y with R y = g (upper triangular back substitution)
        for (int i = k - 1; i >= 0; --i) {
            double t = g[i];
            for (int j = i + 1; j < k; ++j) t -= H[(size_t)i * m + j] * y[j];
            y[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
        }
        cudaMemcpyAsync(hd + (m + 2), y.data(), (size_t)k * 8, cudaMemcpyHostToDevice, c->stream);
        fse::vec_mupdate(c, n, k, Vb, hd + (m + 2), x);
        rc = cuda_check(c, cudaStreamSynchronize(c->stream), "GMRES update");
        if (rc) return rc;
        if (rel <= rtol) break;
    }
    *iters_out = it;
    *relres_out = rel;
    return rel <= rtol ? FSE_OK : FSE_ENOCONV;
}

// Solve J dZ = -R (Jacobian and R of the last evaluation) and update d.Z0 += dZ, on the device.
// Returns FSE_OK, FSE_ENOCONV (GMRES stopped above its tolerance; the update is applied) or an error.
static int newton_solve_update(fse_ctx* c) {
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    const bool dense = !c->p.shard && (c->lin_kind == FSE_LIN_DENSE || (c->lin_kind == FSE_LIN_AUTO && m <= 16384));
    if (c->p.shard && c->lin_kind == FSE_LIN_DENSE)
        return set_err(c, FSE_EINVAL, "a trajectory shard has no dense Jacobian: use GMRES");
    c->reduce_failed = false;
    c->lin_iters = 0;
    c->lin_relres = 0.0;
    if (dense) {
        if (m > 16384) return set_err(c, FSE_EINVAL, "outer solve: dense LU limited to 16384 unknowns");
        int rc = ensure_dense(c, m);
        if (rc) return rc;
        fse::launch_dense_jac(c, c->Jd);
        fse::vec_axpby(c, m, -1.0, c->d.R, 0.0, c->d.vec);       // rhs = -R
        rc = fse::dense_lu_solve(c, c->Jd, c->d.vec, (int)m);
        if (rc) return set_err(c, rc, "singular shooting Jacobian");
        fse::vec_axpby(c, m, 1.0, c->d.vec, 1.0, c->d.Z0);       // Z0 += dZ
        return cuda_check(c, cudaStreamSynchronize(c->stream), "newton update");
    }
    fse::vec_axpby(c, m, -1.0, c->d.R, 0.0, c->d.vec2);          // rhs = -R
    int it = 0;
    double rel = 0.0;
    const int rc = gmres_dev(
        c, m, [c](const double* v, double* w) { jac_apply_dev(c, v, w); }, c->d.vec2, c->d.vec, c->lin_rtol,
        c->lin_restart, c->lin_maxit, &it, &rel);
    c->lin_iters = it;
    c->lin_relres = rel;
    if (c->reduce_failed) return set_err(c, FSE_ECUDA, "shard reduction failed");
    if (rc != FSE_OK && rc != FSE_ENOCONV) return rc;
    fse::vec_axpby(c, m, 1.0, c->d.vec, 1.0, c->d.Z0);           // Z0 += dZ
    const int rc2 = cuda_check(c, cudaStreamSynchronize(c->stream), "newton update");
    if (rc2) return rc2;
    if (rc == FSE_ENOCONV) c->err = "GMRES stopped above its tolerance";
    return rc;
}

extern "C" int fse_set_linear_solver(fse_ctx* c, int kind, double rel_tol, int restart, int max_iters) {
    if (!c) return FSE_EINVAL;
    if (kind != FSE_LIN_AUTO && kind != FSE_LIN_DENSE && kind != FSE_LIN_GMRES)
        return set_err(c, FSE_EINVAL, "unknown linear solver");
    if (restart < 1 || restart > 256 || max_iters < 1 || !(rel_tol > 0.0))
        return set_err(c, FSE_EINVAL, "need rel_tol > 0, 1 <= restart <= 256, max_iters >= 1");
    c->lin_kind = kind;
    c->lin_rtol = rel_tol;
    c->lin_restart = restart;
    c->lin_maxit = max_iters;
    return FSE_OK;
}

extern "C" int fse_linear_stats(const fse_ctx* c, int* iters, double* rel_res) {
    if (!c) return FSE_EINVAL;
    if (iters) *iters = c->lin_iters;
    if (rel_res) *rel_res = c->lin_relres;
    return FSE_OK;
}

extern "C" int fse_newton_step(fse_ctx* c, double* Z0, double w, double* res_norm) {
    if (!c || !Z0) return FSE_EINVAL;
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    cudaSetDevice(c->device);
    cudaMemcpyAsync(c->d.Z0, Z0, m * 8, cudaMemcpyHostToDevice, c->stream);
    const int st = eval_at_iterate(c, w, 1, res_norm, nullptr);
    if (st < 0 && st != FSE_ENOCONV) return st;
    const int lin = newton_solve_update(c);
    if (lin != FSE_OK && lin != FSE_ENOCONV) return lin;
    cudaMemcpyAsync(Z0, c->d.Z0, m * 8, cudaMemcpyDeviceToHost, c->stream);
    const int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "newton_step");
    if (rc) return rc;
    return st != FSE_OK ? st : lin;
}

// ----------------------------------------------------------------------------
// FSE-Shooting in the hyper-time domain (Sec. 3.4, Eq. FSES_T): the start points zbar(0, phi~_s)
// are the unknowns; R_T = (I (x) Gamma R Gamma^-1) zbar(2 pi) - zbar(0), J_T = (I (x) Gamma R
// Gamma^-1) blockdiag(Phi_s) - I.  Vectors are sample-major, N x 2n.
// ----------------------------------------------------------------------------

// device buffers of the hyper-time form, allocated on first use: start points, residual, two
// scratch vectors (N x 2n each), a coefficient vector (2n U~) and Gamma R Gamma^-1 (N x N)
static int ensure_hypertime(fse_ctx* c) {
    if (c->ht) return FSE_OK;
    const Params& p = c->p;
    const size_t m = (size_t)p.N * 2 * p.n;
    const size_t tot = 4 * m + (size_t)2 * p.n * p.U + (size_t)p.N * p.N;
    cudaError_t e = cudaMalloc(&c->ht, tot * 8);
    if (e != cudaSuccess) {
        c->ht = nullptr;
        return cuda_check(c, e, "hyper-time buffers");
    }
    c->ht_pm = false;
    return FSE_OK;
}

// w = J_T v: blockdiag(Phi_s) v, DFT + rotation, i-DFT, minus v
static void jac_apply_ht_dev(fse_ctx* c, const double* v, double* w) {
    const Params& p = c->p;
    const size_t m = (size_t)p.N * 2 * p.n;
    double* coef = c->ht + 4 * m;
    fse::launch_phi_apply(c, v, c->d.yb);
    dft_sub(c, c->d.yb, nullptr, coef);
    fse::launch_idft(c, coef, w);
    fse::vec_axpby(c, m, -1.0, v, 1.0, w);
}

extern "C" int fse_residual_jacobian_hypertime(fse_ctx* c, const double* zbar0, double w, double* RT_out,
                                               int want_jacobian, int* ts, int* it) {
    if (!c || !zbar0 || !RT_out) return FSE_EINVAL;
    cudaSetDevice(c->device);
    int rc = ensure_hypertime(c);
    if (rc) return rc;
    const size_t m = (size_t)c->p.N * 2 * c->p.n;
    cudaMemcpyAsync(c->ht, zbar0, m * 8, cudaMemcpyHostToDevice, c->stream);
    rc = run_eval(c, nullptr, w, c->ht + m, want_jacobian, c->ht);
    if (rc) return rc;
    cudaMemcpyAsync(RT_out, c->ht + m, m * 8, cudaMemcpyDeviceToHost, c->stream);
    return collect_status(c, ts, it);
}

extern "C" int fse_jacobian_apply_hypertime(fse_ctx* c, const double* v, double* Jv, int nvec) {
    if (!c || !v || !Jv || nvec < 0) return FSE_EINVAL;
    if (!c->have_jac) return set_err(c, FSE_ENOJAC, "no Jacobian stored: evaluate with want_jacobian=1 first");
    cudaSetDevice(c->device);
    int rc = ensure_hypertime(c);
    if (rc) return rc;
    const size_t m = (size_t)c->p.N * 2 * c->p.n;
    double* a = c->ht + 2 * m;
    double* b = c->ht + 3 * m;
    for (int k = 0; k < nvec; ++k) {
        cudaMemcpyAsync(a, v + k * m, m * 8, cudaMemcpyHostToDevice, c->stream);
        jac_apply_ht_dev(c, a, b);
        cudaMemcpyAsync(Jv + k * m, b, m * 8, cudaMemcpyDeviceToHost, c->stream);
    }
    return cuda_check(c, cudaStreamSynchronize(c->stream), "jacobian_apply_hypertime");
}

extern "C" int fse_newton_step_hypertime(fse_ctx* c, double* zbar0, double w, double* res_norm) {
    if (!c || !zbar0) return FSE_EINVAL;
    cudaSetDevice(c->device);
    int rc = ensure_hypertime(c);
    if (rc) return rc;
    const Params& p = c->p;
    const size_t m = (size_t)p.N * 2 * p.n;
    double* z0 = c->ht;
    double* rt = c->ht + m;
    double* a = c->ht + 2 * m;
    double* b = c->ht + 3 * m;
    double* Pm = c->ht + 4 * m + (size_t)2 * p.n * p.U;
    cudaMemcpyAsync(z0, zbar0, m * 8, cudaMemcpyHostToDevice, c->stream);
    rc = run_eval(c, nullptr, w, rt, 1, z0);
    if (rc) return rc;
    const int st = collect_status(c, nullptr, nullptr);
    if (st < 0 && st != FSE_ENOCONV) return st;
    fse::vec_norms2(c, m, rt, nullptr, c->d.vec2);
    double h2[2];
    cudaMemcpyAsync(h2, c->d.vec2, 16, cudaMemcpyDeviceToHost, c->stream);
    rc = cuda_check(c, cudaStreamSynchronize(c->stream), "hyper-time residual norm");
    if (rc) return rc;
    if (res_norm) *res_norm = std::sqrt(h2[0]);
    fse::vec_axpby(c, m, -1.0, rt, 0.0, b);   // rhs = -R_T
    if (p.shard && c->lin_kind == FSE_LIN_DENSE)
        return set_err(c, FSE_EINVAL, "a trajectory shard has no dense Jacobian: use GMRES");
    const bool dense = !p.shard && (c->lin_kind == FSE_LIN_DENSE || (c->lin_kind == FSE_LIN_AUTO && m <= 16384));
    c->lin_iters = 0;
    c->lin_relres = 0.0;
    c->reduce_failed = false;
    int lin = FSE_OK;
    if (dense) {
        if (m > 16384) return set_err(c, FSE_EINVAL, "outer solve: dense LU limited to 16384 unknowns");
        rc = ensure_dense(c, m);
        if (rc) return rc;
        if (!c->ht_pm) {
            fse::launch_pmat(c, Pm);
            c->ht_pm = true;
        }
        fse::launch_dense_jac_ht(c, Pm, c->Jd);
        rc = fse::dense_lu_solve(c, c->Jd, b, (int)m);
        if (rc) return set_err(c, rc, "singular hyper-time Jacobian");
        fse::vec_axpby(c, m, 1.0, b, 1.0, z0);
    } else {
        int its = 0;
        double rel = 0.0;
        lin = gmres_dev(
            c, m, [c](const double* v, double* o) { jac_apply_ht_dev(c, v, o); }, b, a, c->lin_rtol,
            c->lin_restart, c->lin_maxit, &its, &rel);
        c->lin_iters = its;
        c->lin_relres = rel;
        if (c->reduce_failed) return set_err(c, FSE_ECUDA, "shard reduction failed");
        if (lin != FSE_OK && lin != FSE_ENOCONV) return lin;
        fse::vec_axpby(c, m, 1.0, a, 1.0, z0);
        if (lin == FSE_ENOCONV) c->err = "GMRES stopped above its tolerance";
    }
    cudaMemcpyAsync(zbar0, z0, m * 8, cudaMemcpyDeviceToHost, c->stream);
    rc = cuda_check(c, cudaStreamSynchronize(c->stream), "newton_step_hypertime");
    if (rc) return rc;
    return st != FSE_OK ? st : lin;
}

// ----------------------------------------------------------------------------
// a priori unknown base frequencies (Sec. 3.2: Eq. Cont1, 18, 19, 23, 24)
// ----------------------------------------------------------------------------

extern "C" int fse_set_rho(fse_ctx* c, const double* rho) {
    if (!c || !rho) return FSE_EINVAL;
    const int dm1 = c->p.d - 1;
    for (int j = 0; j < dm1; ++j)
        if (!std::isfinite(rho[j])) return set_err(c, FSE_EINVAL, "rho not finite");
    bool same = true;
    for (int j = 0; j < dm1; ++j) same = same && c->rho[j] == rho[j];
    if (same) return FSE_OK;
    cudaSetDevice(c->device);
    for (int j = 0; j < dm1; ++j) c->rho[j] = rho[j];
    std::vector<double> rcv, rsv;
    rotation_tables(c, rcv, rsv);
    cudaMemcpyAsync(c->d.rc, rcv.data(), rcv.size() * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d.rs, rsv.data(), rsv.size() * 8, cudaMemcpyHostToDevice, c->stream);
    fse::launch_fill_tables(c);
    c->ht_pm = false;
    c->have_jac = false;   // the stored Jacobian belongs to the previous rotation
    return cuda_check(c, cudaStreamSynchronize(c->stream), "set_rho");
}

extern "C" int fse_newton_step_unknown(fse_ctx* c, double* Z0, double w, double* rho, const int* unknown,
                                       double* res_norm) {
    if (!c || !Z0 || !rho || !unknown) return FSE_EINVAL;
    const Params& p = c->p;
    const int dm1 = p.d - 1;
    int idx[FSE_MAX_D - 1], u = 0;
    for (int j = 0; j < dm1; ++j)
        if (unknown[j]) {
            // forcing component j + 1 (0-based) moves its phase with rho_j (Eq. E1): then w_{j+2} is set
            if (j + 1 < p.e) return set_err(c, FSE_EINVAL, "a forced frequency cannot be an unknown");
            idx[u++] = j;
        }
    int rc = fse_set_rho(c, rho);
    if (rc) return rc;
    cudaSetDevice(c->device);
    const size_t m = (size_t)2 * p.n * p.U, M = m + u;
    if (!c->unk) {
        cudaError_t e = cudaMalloc(&c->unk, (2 * (size_t)(FSE_MAX_D - 1) * m + 2 * (m + FSE_MAX_D)) * 8);
        if (e != cudaSuccess) {
            c->unk = nullptr;
            return cuda_check(c, e, "unknown-frequency buffers");
        }
    }
    double* cols = c->unk;
    double* rows = cols + (size_t)(FSE_MAX_D - 1) * m;
    double* xs = rows + (size_t)(FSE_MAX_D - 1) * m;   // solution (M)
    double* bs = xs + m + FSE_MAX_D;                   // right-hand side (M)
    cudaMemcpyAsync(c->d.Z0, Z0, m * 8, cudaMemcpyHostToDevice, c->stream);
    const int st = eval_at_iterate(c, w, 1, res_norm, nullptr);
    if (st < 0 && st != FSE_ENOCONV) return st;
    for (int a = 0; a < u; ++a)
        fse::launch_unknown_border(c, idx[a], w, c->d.R, c->d.Z0, cols + (size_t)a * m, rows + (size_t)a * m);
    // rhs = -[R; 0]
    fse::vec_axpby(c, m, -1.0, c->d.R, 0.0, bs);
    if (u) cudaMemsetAsync(bs + m, 0, u * 8, c->stream);
    if (p.shard && c->lin_kind == FSE_LIN_DENSE)
        return set_err(c, FSE_EINVAL, "a trajectory shard has no dense Jacobian: use GMRES");
    const bool dense = !p.shard && (c->lin_kind == FSE_LIN_DENSE || (c->lin_kind == FSE_LIN_AUTO && M <= 16384));
    c->lin_iters = 0;
    c->lin_relres = 0.0;
    c->reduce_failed = false;
    int lin = FSE_OK;
    if (dense) {
        if (M > 16384) return set_err(c, FSE_EINVAL, "outer solve: dense LU limited to 16384 unknowns");
        rc = ensure_dense(c, M);
        if (rc) return rc;
        fse::launch_dense_jac_bordered(c, u, cols, rows, c->Jd);
        rc = fse::dense_lu_solve(c, c->Jd, bs, (int)M);
        if (rc) return set_err(c, rc, "singular bordered shooting Jacobian");
        cudaMemcpyAsync(xs, bs, M * 8, cudaMemcpyDeviceToDevice, c->stream);
    } else {
        // [J cols; rows^T 0] x: J x_Z + sum_a cols_a x_a, rows_a . x_Z
        auto Av = [c, m, u, cols, rows](const double* x, double* y) {
            jac_apply_dev(c, x, y);
            if (u) {
                fse::vec_mupdate(c, m, u, cols, x + m, y);
                fse::vec_mdot(c, m, u, rows, x, y + m);
            }
        };
        int its = 0;
        double rel = 0.0;
        lin = gmres_dev(c, M, Av, bs, xs, c->lin_rtol, c->lin_restart, c->lin_maxit, &its, &rel);
        c->lin_iters = its;
        c->lin_relres = rel;
        if (c->reduce_failed) return set_err(c, FSE_ECUDA, "shard reduction failed");
        if (lin != FSE_OK && lin != FSE_ENOCONV) return lin;
        if (lin == FSE_ENOCONV) c->err = "GMRES stopped above its tolerance";
    }
    fse::vec_axpby(c, m, 1.0, xs, 1.0, c->d.Z0);   // Z0 += dZ
    double dw[FSE_MAX_D - 1] = {0.0};
    if (u) cudaMemcpyAsync(dw, xs + m, u * 8, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(Z0, c->d.Z0, m * 8, cudaMemcpyDeviceToHost, c->stream);
    rc = cuda_check(c, cudaStreamSynchronize(c->stream), "newton_step_unknown");
    if (rc) return rc;
    for (int a = 0; a < u; ++a) rho[idx[a]] += dw[a] / w;   // w_{j+2} = rho_j w_1 with w_1 fixed
    return st != FSE_OK ? st : lin;
}

extern "C" int fse_lyapunov(fse_ctx* c, const double* Z0, double w, int N_Ly, int h, double* sigma) {
    if (c && c->p.shard) return set_err(c, FSE_EINVAL, "not available on a trajectory shard");
    if (!c || !Z0 || !sigma) return FSE_EINVAL;
    if (N_Ly < 1 || h < 1 || h > 64 || h > 2 * c->p.n) return set_err(c, FSE_EINVAL, "need N_Ly >= 1, 1 <= h <= min(64, 2n)");
    cudaSetDevice(c->device);
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    cudaMemcpyAsync(c->d.Z0, Z0, m * 8, cudaMemcpyHostToDevice, c->stream);
    int rc = run_eval(c, c->d.Z0, w, c->d.R, 1);
    if (rc) return rc;
    const int st = collect_status(c, nullptr, nullptr);
    if (st < 0 && st != FSE_ENOCONV) return st;
    rc = fse::lyapunov_run(c, w, N_Ly, h, sigma);
    return rc ? rc : st;
}

extern "C" int fse_lyapunov_noalloc(fse_ctx* c, const double* Z0, double w, int N_Ly, int h, double* sigma) {
    if (c && c->p.shard) return set_err(c, FSE_EINVAL, "not available on a trajectory shard");
    if (!c || !Z0 || !sigma) return FSE_EINVAL;
    if (N_Ly < 1 || h < 1 || h > 64 || h > 2 * c->p.n)
        return set_err(c, FSE_EINVAL, "need N_Ly >= 1, 1 <= h <= min(64, 2n)");
    if ((size_t)2 * c->p.n * h > FSE_NOALLOC_MAX_QH)
        return set_err(c, FSE_EINVAL, "2 n h exceeds FSE_NOALLOC_MAX_QH of the static scratch (262144 doubles)");
    if (c->p.N > FSE_NOALLOC_MAX_N)
        return set_err(c, FSE_EINVAL, "number of trajectories exceeds FSE_NOALLOC_MAX_N of the static scratch (65536)");
    cudaSetDevice(c->device);
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    cudaMemcpyAsync(c->d.Z0, Z0, m * 8, cudaMemcpyHostToDevice, c->stream);
    int rc = run_eval(c, c->d.Z0, w, c->d.R, 1);
    if (rc) return rc;
    const int st = collect_status(c, nullptr, nullptr);
    if (st < 0 && st != FSE_ENOCONV) return st;
    rc = fse::lyapunov_run_noalloc(c, w, N_Ly, h, sigma);
    return rc ? rc : st;
}

// ----------------------------------------------------------------------------
// several contexts (continuation points, possibly of different N) evaluated together
// ----------------------------------------------------------------------------

struct fse_batch {
    std::vector<fse_ctx*> ctx;
    int device = 0;
    bool use_graph = false;
    cudaStream_t master = nullptr;   // graph mode: capture origin and launch stream
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double> w;           // w_1 of each context in the captured graph
    int sens = -1;                   // want_jacobian of the captured graph (-1: none)
    std::string err;
};

static void batch_free(fse_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->master) cudaStreamDestroy(b->master);
    delete b;
}

extern "C" int fse_batch_create(fse_ctx* const* ctxs, int count, int use_graph, fse_batch** out) {
    if (!out) return FSE_EINVAL;
    *out = nullptr;
    if (!ctxs || count < 1) return FSE_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) return FSE_EINVAL;
        if (ctxs[i]->device != ctxs[0]->device) return set_err(ctxs[0], FSE_EINVAL, "batch contexts on different devices");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return set_err(ctxs[0], FSE_EINVAL, "a context appears twice in the batch");
    }
    fse_batch* b = new (std::nothrow) fse_batch();
    if (!b) return FSE_ENOMEM;
    b->ctx.assign(ctxs, ctxs + count);
    b->device = ctxs[0]->device;
    b->use_graph = use_graph != 0;
    cudaSetDevice(b->device);
    cudaError_t e = cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    b->join.assign(count, nullptr);
    for (int i = 0; i < count && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        batch_free(b);
        return FSE_ECUDA;
    }
    *out = b;
    return FSE_OK;
}

extern "C" void fse_batch_destroy(fse_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->master) cudaStreamSynchronize(b->master);
    batch_free(b);
}

extern "C" const char* fse_batch_last_error(const fse_batch* b) { return b ? b->err.c_str() : ""; }

// capture the evaluations of all contexts at the current w_1 values into one graph
static int batch_capture(fse_batch* b, const double* w, int sens) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->master, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        b->err = std::string("graph capture: ") + cudaGetErrorString(e);
        return FSE_ECUDA;
    }
    cudaEventRecord(b->fork, b->master);
    int rc = FSE_OK;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        fse_ctx* c = b->ctx[i];
        cudaStreamWaitEvent(c->stream, b->fork, 0);
        const int r = run_eval(c, c->d.Z0, w[i], c->d.R, sens);
        if (r && !rc) {
            rc = r;
            b->err = c->err;
        }
        cudaEventRecord(b->join[i], c->stream);
        cudaStreamWaitEvent(b->master, b->join[i], 0);
    }
    e = cudaStreamEndCapture(b->master, &b->graph);
    if (rc) return rc;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        b->err = std::string("graph capture: ") + cudaGetErrorString(e);
        return FSE_ECUDA;
    }
    b->w.assign(w, w + b->ctx.size());
    b->sens = sens;
    return FSE_OK;
}

extern "C" int fse_batch_residual_jacobian(fse_batch* b, const double* const* Z0, const double* omega1,
                                           double* const* R_out, int sens, int* status_out) {
    if (!b || !Z0 || !omega1 || !R_out) return FSE_EINVAL;
    const int count = (int)b->ctx.size();
    for (int i = 0; i < count; ++i) {
        if (!Z0[i] || !R_out[i]) return FSE_EINVAL;
        if (!(omega1[i] > 0.0) || !std::isfinite(omega1[i])) {
            b->err = "omega1 must be positive and finite";
            return FSE_EINVAL;
        }
    }
    cudaSetDevice(b->device);
    sens = sens ? 1 : 0;
    if (b->use_graph) {
        bool same = b->exec && b->sens == sens;
        for (int i = 0; same && i < count; ++i) same = b->w[i] == omega1[i];
        // the inputs go to the contexts' start buffers on the launch stream, before the graph
        for (int i = 0; i < count; ++i) {
            fse_ctx* c = b->ctx[i];
            cudaMemcpyAsync(c->d.Z0, Z0[i], (size_t)2 * c->p.n * c->p.U * 8, cudaMemcpyHostToDevice, b->master);
        }
        if (!same) {
            // the capture waits for nothing the contexts still run: drain them and the copies first
            for (fse_ctx* c : b->ctx) cudaStreamSynchronize(c->stream);
            cudaStreamSynchronize(b->master);
            const int rc = batch_capture(b, omega1, sens);
            if (rc) return rc;
        }
        cudaError_t e = cudaGraphLaunch(b->exec, b->master);
        if (e != cudaSuccess) {
            b->err = std::string("graph launch: ") + cudaGetErrorString(e);
            return FSE_ECUDA;
        }
        cudaEventRecord(b->done, b->master);
        for (fse_ctx* c : b->ctx) cudaStreamWaitEvent(c->stream, b->done, 0);
    } else {
        for (int i = 0; i < count; ++i) {
            fse_ctx* c = b->ctx[i];
            cudaMemcpyAsync(c->d.Z0, Z0[i], (size_t)2 * c->p.n * c->p.U * 8, cudaMemcpyHostToDevice, c->stream);
            const int rc = run_eval(c, c->d.Z0, omega1[i], c->d.R, sens);
            if (rc) {
                b->err = c->err;
                return rc;
            }
        }
    }
    int worst = FSE_OK;
    for (int i = 0; i < count; ++i) {
        fse_ctx* c = b->ctx[i];
        cudaMemcpyAsync(R_out[i], c->d.R, (size_t)2 * c->p.n * c->p.U * 8, cudaMemcpyDeviceToHost, c->stream);
        const int st = collect_status(c, nullptr, nullptr);
        if (status_out) status_out[i] = st;
        if (st < 0 && st != FSE_ENOCONV) {
            b->err = c->err;
            return st;
        }
        if (st != FSE_OK && worst == FSE_OK) worst = st;
    }
    return worst;
}

// ----------------------------------------------------------------------------
// pseudo-arclength continuation in (Z(0), w_1) (App. C, Eq. C1-C3)
// ----------------------------------------------------------------------------

extern "C" int fse_continue_arclength(fse_ctx* c, const fse_arc_opts* o, const double* Z_start, double* Z_out,
                                      double* omega_out, fse_cont_point* info, int* n_done) {
    if (c && c->p.shard) return set_err(c, FSE_EINVAL, "not available on a trajectory shard");
    if (!c || !o || !Z_start || o->n_points < 1) return FSE_EINVAL;
    if (n_done) *n_done = 0;
    if (!(o->rel_tol > 0.0) || o->max_newton < 1 || !(o->ds > 0.0) || !(o->omega_start > 0.0))
        return set_err(c, FSE_EINVAL, "need rel_tol > 0, max_newton >= 1, ds > 0, omega_start > 0");
    cudaSetDevice(c->device);
    const size_t m = (size_t)2 * c->p.n * c->p.U;
    if (m + 1 > 16384) return set_err(c, FSE_EINVAL, "pseudo-arclength: bordered dense solve limited to 16383 unknowns");
    int rc = ensure_dense(c, m + 1);
    if (rc) return rc;
    double *Zprev = nullptr, *Zpred = nullptr, *tZ = nullptr, *tmp = nullptr, *rhs = nullptr, *dd = nullptr;
    cudaError_t e = cudaMalloc(&Zprev, m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&Zpred, m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&tZ, m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&rhs, (m + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dd, 16);
    auto cleanup = [&]() {
        for (void* q : {(void*)Zprev, (void*)Zpred, (void*)tZ, (void*)tmp, (void*)rhs, (void*)dd})
            if (q) cudaFree(q);
    };
    if (e != cudaSuccess) {
        cleanup();
        return cuda_check(c, e, "arclength buffers");
    }
    auto sq_norm = [&](const double* v) -> double {   // ||v||^2 (m entries)
        fse::vec_norms2(c, m, v, nullptr, dd);
        double h[2];
        cudaMemcpyAsync(h, dd, 16, cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        return h[0];
    };
    auto dot = [&](const double* a, const double* b) -> double {
        fse::vec_mdot(c, m, 1, a, b, dd);
        double h = 0.0;
        cudaMemcpyAsync(&h, dd, 8, cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        return h;
    };
    auto get_last = [&]() -> double {
        double h = 0.0;
        cudaMemcpyAsync(&h, rhs + m, 8, cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        return h;
    };
    auto set_last = [&](double v) { cudaMemcpy(rhs + m, &v, 8, cudaMemcpyHostToDevice); };
    auto dRdw = [&]() {   // dR/dw_1 of the last Jacobian evaluation -> d.vec2 (Eq. 23)
        fse::launch_domega(c, c->d.yb);
        fse::launch_dft_residual(c, c->d.yb, nullptr, c->d.vec2, 0);
    };
    auto record = [&](int j, double w, int it, int evals, double rn, double zn, int pst) {
        if (Z_out) cudaMemcpyAsync(Z_out + (size_t)j * m, c->d.Z0, m * 8, cudaMemcpyDeviceToHost, c->stream);
        cudaEventRecord(c->ev[5], c->stream);
        cudaStreamSynchronize(c->stream);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]);
        if (omega_out) omega_out[j] = w;
        if (info) {
            info[j].newton_iters = it;
            info[j].evals = evals;
            info[j].res = rn;
            info[j].znorm = zn;
            info[j].pred_err = 0.0;
            info[j].ms = ms;
            info[j].status = pst;
            info[j].predictor = FSE_PRED_SECANT;
            info[j].fallback = 0;
        }
        if (n_done) *n_done = j + 1;
    };
    // ---- point 0: Newton at fixed w_1 = omega_start
    double w = o->omega_start, rn = 0.0, zn = 0.0;
    cudaEventRecord(c->ev[4], c->stream);
    cudaMemcpyAsync(c->d.Z0, Z_start, m * 8, cudaMemcpyHostToDevice, c->stream);
    int it = 0, evals = 1;
    int st = eval_at_iterate(c, w, 1, &rn, &zn);
    while (st >= FSE_ENOCONV && rn > o->rel_tol * zn && it < o->max_newton) {
        rc = newton_solve_update(c);
        if (rc && rc != FSE_ENOCONV) {
            cleanup();
            return rc;
        }
        ++it;
        st = eval_at_iterate(c, w, 1, &rn, &zn);
        ++evals;
    }
    int pst = (st < 0) ? st : (rn <= o->rel_tol * zn ? FSE_OK : FSE_ENOCONV);
    record(0, w, it, evals, rn, zn, pst);
    if (pst != FSE_OK) {
        cleanup();
        return pst;
    }
    // metric ||dZ||^2 + (sigma dw)^2 of the arclength
    const double sigma = o->omega_scale > 0.0 ? o->omega_scale : zn / w;
    const double s2 = sigma * sigma;
    // ---- first tangent: [J dR/dw; 0 1] (t_Z; t_w) = (0; 1), oriented by `direction`
    dRdw();
    cudaMemsetAsync(tmp, 0, m * 8, c->stream);
    fse::launch_bordered_jac(c, c->d.vec2, tmp, 1.0, c->Jd);
    cudaMemsetAsync(rhs, 0, (m + 1) * 8, c->stream);
    cudaStreamSynchronize(c->stream);
    set_last(1.0);
    rc = fse::dense_lu_solve(c, c->Jd, rhs, (int)m + 1);
    if (rc) {
        cleanup();
        return set_err(c, rc, "singular bordered system at the start point");
    }
    double tw = get_last();
    {
        const double nrm = std::sqrt(sq_norm(rhs) + s2 * tw * tw);
        const double sg = ((o->direction < 0) ? -1.0 : 1.0) * (tw < 0 ? -1.0 : 1.0) / nrm;
        cudaMemcpyAsync(tZ, rhs, m * 8, cudaMemcpyDeviceToDevice, c->stream);
        fse::vec_axpby(c, m, 0.0, tZ, sg, tZ);
        tw *= sg;
    }
    cudaMemcpyAsync(Zprev, c->d.Z0, m * 8, cudaMemcpyDeviceToDevice, c->stream);
    double wprev = w;
    int worst = FSE_OK;
    double ds = o->ds;
    const double ds_max = std::max(o->ds_max, o->ds), ds_min = o->ds / 64.0;
    for (int j = 1; j < o->n_points; ++j) {
        cudaEventRecord(c->ev[4], c->stream);
        // predictor: y_pred = y_{j-1} + ds t
        const double wpred = wprev + ds * tw;
        cudaMemcpyAsync(Zpred, Zprev, m * 8, cudaMemcpyDeviceToDevice, c->stream);
        fse::vec_axpby(c, m, ds, tZ, 1.0, Zpred);
        cudaMemcpyAsync(c->d.Z0, Zpred, m * 8, cudaMemcpyDeviceToDevice, c->stream);
        w = wpred;
        it = 0;
        evals = 1;
        st = eval_at_iterate(c, w, 1, &rn, &zn);
        // corrector: Newton on R = 0 and t . (y - y_pred) = 0 (bordered system)
        while (st >= FSE_ENOCONV && std::isfinite(rn) && rn > o->rel_tol * zn && it < o->max_newton) {
            dRdw();
            cudaMemcpyAsync(tmp, c->d.Z0, m * 8, cudaMemcpyDeviceToDevice, c->stream);
            fse::vec_axpby(c, m, -1.0, Zpred, 1.0, tmp);
            const double Nres = dot(tZ, tmp) + s2 * tw * (w - wpred);
            fse::launch_bordered_jac(c, c->d.vec2, tZ, s2 * tw, c->Jd);
            fse::vec_axpby(c, m, -1.0, c->d.R, 0.0, rhs);
            cudaStreamSynchronize(c->stream);
            set_last(-Nres);
            rc = fse::dense_lu_solve(c, c->Jd, rhs, (int)m + 1);
            if (rc) {
                st = set_err(c, rc, "singular bordered system");
                break;
            }
            const double dw = get_last();
            fse::vec_axpby(c, m, 1.0, rhs, 1.0, c->d.Z0);
            w += dw;
            ++it;
            st = eval_at_iterate(c, w, 1, &rn, &zn);
            ++evals;
        }
        pst = (st < 0) ? st : ((std::isfinite(rn) && rn <= o->rel_tol * zn) ? FSE_OK : FSE_ENOCONV);
        if (pst == FSE_ENOCONV && ds * 0.5 >= ds_min) {
            // not converged from this prediction: halve the step and predict again from y_{j-1}
            ds *= 0.5;
            --j;
            continue;
        }
        record(j, w, it, evals, rn, zn, pst);
        if (pst != FSE_OK) {
            worst = pst;
            break;
        }
        // step control: grow after an easy correction, shrink after a hard one
        if (it <= 2)
            ds = std::min(ds * 1.5, ds_max);
        else if (it >= 5)
            ds = std::max(ds * 0.7, ds_min);
        // secant tangent through the last two points
        cudaMemcpyAsync(tZ, c->d.Z0, m * 8, cudaMemcpyDeviceToDevice, c->stream);
        fse::vec_axpby(c, m, -1.0, Zprev, 1.0, tZ);
        tw = w - wprev;
        const double nrm = std::sqrt(sq_norm(tZ) + s2 * tw * tw);
        fse::vec_axpby(c, m, 0.0, tZ, 1.0 / nrm, tZ);
        tw /= nrm;
        cudaMemcpyAsync(Zprev, c->d.Z0, m * 8, cudaMemcpyDeviceToDevice, c->stream);
        wprev = w;
        if ((o->omega_max > 0.0 && w > o->omega_max) || w < o->omega_min) break;
    }
    cleanup();
    return worst;
}

extern "C" int fse_set_steps(fse_ctx* c, int n_steps) {
    if (!c || n_steps < 0) return FSE_EINVAL;
    c->n_steps = n_steps;
    return FSE_OK;
}

extern "C" int fse_set_reduce(fse_ctx* c, fse_reduce_fn fn, void* user) {
    if (!c) return FSE_EINVAL;
    if (!c->p.shard) return set_err(c, FSE_EINVAL, "not a trajectory shard");
    c->reduce = fn;
    c->reduce_user = user;
    return FSE_OK;
}

extern "C" int fse_set_tangent_solve(fse_ctx* c, int kind) {
    if (!c) return FSE_EINVAL;
    if (kind != FSE_SOLVE_AUTO && kind != FSE_SOLVE_SIMT && kind != FSE_SOLVE_TC)
        return set_err(c, FSE_EINVAL, "unknown tangent-solve kind");
    if (kind == FSE_SOLVE_TC && !c->p.tc_ok)
        return set_err(c, FSE_EINVAL, "tensor-core solves need FP32 tangents and half-bandwidth <= 96");
    c->solve_kind = kind;
    return FSE_OK;
}

extern "C" int fse_profile(fse_ctx* c, int enable) {
    if (!c) return FSE_EINVAL;
    cudaSetDevice(c->device);
    c->prof = enable != 0;
    if (c->prof && (int)c->pev.size() != 8 * c->p.S1) {
        for (auto& e : c->pev)
            if (e) cudaEventDestroy(e);
        c->pev.assign((size_t)8 * c->p.S1, nullptr);
        for (auto& e : c->pev)
            if (cudaEventCreate(&e) != cudaSuccess) return set_err(c, FSE_ECUDA, "event creation failed");
    }
    return FSE_OK;
}

extern "C" int fse_timings(fse_ctx* c, double* ms, int cap) {
    if (!c || !ms) return FSE_EINVAL;
    for (int k = 0; k < cap && k < 6; ++k) ms[k] = c->timing[k];
    return FSE_OK;
}

// ----------------------------------------------------------------------------
// one-parameter continuation in w_1 with the secant or the learned predictor
// ----------------------------------------------------------------------------

extern "C" int fse_set_fallback(fse_ctx* c, fse_ctx* fb) {
    if (!c) return FSE_EINVAL;
    if (!fb) {
        c->fallback = nullptr;
        return FSE_OK;
    }
    if (fb == c || c->p.prec != FSE_MIXED_FP32 || fb->p.prec != FSE_FP64)
        return set_err(c, FSE_EINVAL, "fallback: an FP64 context for an FSE_MIXED_FP32 one");
    if (c->p.shard || fb->p.shard) return set_err(c, FSE_EINVAL, "fallback: trajectory shards are not supported");
    if (fb->device != c->device || fb->p.n != c->p.n || fb->p.d != c->p.d || fb->p.U != c->p.U ||
        fb->p.N != c->p.N || fb->p.S1 != c->p.S1 || fb->rho != c->rho)
        return set_err(c, FSE_EINVAL, "fallback: a context of another problem (n, d, U, N, S1, rho or device)");
    c->fallback = fb;
    return FSE_OK;
}

extern "C" int fse_continue(fse_ctx* c, fse_mlp* mlp, const fse_cont_opts* o, const double* Z_start,
                            double* Z_out, fse_cont_point* info) {
    if (!c || !o || !Z_start || !o->omega1 || o->n_points < 1) return FSE_EINVAL;
    if (o->predictor == FSE_PRED_MLP && !mlp) return set_err(c, FSE_EINVAL, "learned predictor needs a network");
    if (!(o->rel_tol > 0.0) || o->max_newton < 0) return set_err(c, FSE_EINVAL, "bad tolerance or iteration limit");
    cudaSetDevice(c->device);
    const size_t nu = (size_t)2 * c->p.n * c->p.U;
    const int P = o->n_points;
    if (o->predictor == FSE_PRED_MLP && (o->pod_modes < 1 || fse_mlp_nouts(mlp) != o->pod_modes))
        return set_err(c, FSE_EINVAL, "network outputs must equal pod_modes");
    double *Zs = nullptr, *Zp = nullptr, *Sec = nullptr, *Dsn = nullptr, *Sscr = nullptr, *pmean = nullptr,
           *pbasis = nullptr, *coef = nullptr, *cdev = nullptr;
    cudaError_t e = cudaMalloc(&Zs, (size_t)P * nu * 8);
    if (e == cudaSuccess) e = cudaMalloc(&Zp, nu * 8);
    if (e == cudaSuccess) e = cudaMalloc(&Sec, nu * 8);
    const bool learn = o->predictor == FSE_PRED_MLP;
    const int rmax = std::max(1, o->pod_modes);
    if (learn) {
        if (e == cudaSuccess) e = cudaMalloc(&Dsn, (size_t)P * nu * 8);   // corrections Z_a - S_a, a >= 2
        if (e == cudaSuccess) e = cudaMalloc(&Sscr, (size_t)P * nu * 8);
        if (e == cudaSuccess) e = cudaMalloc(&pmean, nu * 8);
        if (e == cudaSuccess) e = cudaMalloc(&pbasis, (size_t)rmax * nu * 8);
        if (e == cudaSuccess) e = cudaMalloc(&coef, (size_t)P * rmax * 8);
        if (e == cudaSuccess) e = cudaMalloc(&cdev, (size_t)rmax * 8);
    }
    auto cleanup = [&]() {
        for (void* q : {(void*)Zs, (void*)Zp, (void*)Sec, (void*)Dsn, (void*)Sscr, (void*)pmean, (void*)pbasis,
                        (void*)coef, (void*)cdev})
            if (q) cudaFree(q);
    };
    if (e != cudaSuccess) {
        cleanup();
        return cuda_check(c, e, "continuation buffers");
    }
    int r = 0;                                 // current POD rank (0 = no basis yet)
    int reff = 0;                              // modes above the relative threshold 1e-8
    double tmax = 0.0;                         // clamp of the scaled network outputs
    std::vector<double> sing(rmax, 0.0);
    std::vector<double> tsc(rmax, 1.0);        // per-mode scale: RMS of the training coefficients
    const double lo = o->omega_lo, hi = o->omega_hi > o->omega_lo ? o->omega_hi : o->omega_lo + 1.0;
    auto feats = [&](double w, float* x) {
        const double t = 2.0 * (w - lo) / (hi - lo) - 1.0;
        x[0] = (float)t;
        x[1] = (float)t;                        // w_2 = rho w_1: same normalised value
        x[2] = 0.0f;                            // F_1 fixed over the sweep
    };
    // secant prediction S_j = (1 + q) Z_{j-1} - q Z_{j-2} into Sec (j >= 2), or Z_0 (j == 1)
    auto secant = [&](int j) {
        if (j == 1) {
            cudaMemcpyAsync(Sec, Zs, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
            return;
        }
        const double q = (o->omega1[j] - o->omega1[j - 1]) / (o->omega1[j - 1] - o->omega1[j - 2]);
        cudaMemcpyAsync(Sec, Zs + (size_t)(j - 1) * nu, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
        fse::vec_axpby(c, nu, -q, Zs + (size_t)(j - 2) * nu, 1.0 + q, Sec);
    };
    int worst = FSE_OK;
    for (int j = 0; j < P; ++j) {
        const double w = o->omega1[j];
        cudaEventRecord(c->ev[4], c->stream);
        // ---- predictor: secant, plus the network's correction once it has seen enough points
        bool used_mlp = false;
        if (j == 0) {
            cudaMemcpyAsync(c->d.Z0, Z_start, nu * 8, cudaMemcpyHostToDevice, c->stream);
        } else {
            secant(j);
            if (learn && reff > 0 && j >= std::max(4, o->warmup)) {
                float x[3];
                feats(w, x);
                std::vector<float> yy((size_t)rmax);
                int rc = fse_mlp_forward(mlp, x, 1, yy.data());
                if (rc) {
                    cleanup();
                    return set_err(c, rc, "network forward failed");
                }
                std::vector<double> cc(r, 0.0);
                for (int k = 0; k < reff; ++k) {
                    const double t = std::max(-tmax, std::min(tmax, (double)yy[k]));
                    cc[k] = t * tsc[k];
                }
                cudaMemcpyAsync(cdev, cc.data(), r * 8, cudaMemcpyHostToDevice, c->stream);
                fse::pod_expand(c, nu, r, pmean, pbasis, cdev, c->d.Z0);   // predicted correction
                fse::vec_axpby(c, nu, 1.0, Sec, 1.0, c->d.Z0);             // + secant
                used_mlp = true;
            } else {
                cudaMemcpyAsync(c->d.Z0, Sec, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
            }
        }
        cudaMemcpyAsync(Zp, c->d.Z0, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
        // ---- corrector: Newton on Eq. (16) at fixed w_1, accepted when ||R|| <= tol ||Z||
        double rn = 0.0, zn = 0.0;
        int it = 0, evals = 1;
        int st = eval_at_iterate(c, w, 1, &rn, &zn);
        if (used_mlp && (st < FSE_ENOCONV || !std::isfinite(rn))) {
            // the corrected prediction left the basin: fall back to the secant prediction
            cudaMemcpyAsync(c->d.Z0, Sec, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
            cudaMemcpyAsync(Zp, c->d.Z0, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
            used_mlp = false;
            st = eval_at_iterate(c, w, 1, &rn, &zn);
            ++evals;
        }
        while (st >= FSE_ENOCONV && rn > o->rel_tol * zn && it < o->max_newton) {
            int rc = newton_solve_update(c);
            if (rc && rc != FSE_ENOCONV) {
                st = rc;
                break;
            }
            ++it;
            st = eval_at_iterate(c, w, 0, &rn, &zn);
            ++evals;
            if (rn <= o->rel_tol * zn || st < FSE_ENOCONV) break;
            if (o->chord) continue;   // next update with the monodromies of the point's first evaluation
            st = eval_at_iterate(c, w, 1, &rn, &zn);
            ++evals;
        }
        int pst = (st < 0) ? st : (rn <= o->rel_tol * zn ? FSE_OK : FSE_ENOCONV);
        // a point the mixed-precision corrector rejects is corrected again in the FP64 context
        bool fell_back = false;
        if (pst != FSE_OK && pst != FSE_ECUDA && c->fallback) {
            fse_ctx* fb = c->fallback;
            if (fb->rho != c->rho) {
                cleanup();
                return set_err(c, FSE_EINVAL, "fallback context has other rotation numbers");
            }
            int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "continuation point");
            if (!rc) rc = cuda_check(c, cudaMemcpy(fb->d.Z0, Zp, nu * 8, cudaMemcpyDeviceToDevice), "fallback start");
            if (rc) {
                cleanup();
                return rc;
            }
            int fst = eval_at_iterate(fb, w, 1, &rn, &zn);
            ++evals;
            int fit = 0;
            while (fst >= FSE_ENOCONV && rn > o->rel_tol * zn && fit < o->max_newton) {
                const int frc = newton_solve_update(fb);
                if (frc && frc != FSE_ENOCONV) {
                    fst = frc;
                    break;
                }
                ++fit;
                fst = eval_at_iterate(fb, w, 0, &rn, &zn);
                ++evals;
                if (rn <= o->rel_tol * zn || fst < FSE_ENOCONV) break;
                if (o->chord) continue;
                fst = eval_at_iterate(fb, w, 1, &rn, &zn);
                ++evals;
            }
            it += fit;
            pst = (fst < 0) ? fst : (rn <= o->rel_tol * zn ? FSE_OK : FSE_ENOCONV);
            if (fst == FSE_ECUDA) {
                c->err = "fallback context: " + fb->err;
                cleanup();
                return FSE_ECUDA;
            }
            rc = cuda_check(c, cudaStreamSynchronize(fb->stream), "fallback point");
            if (!rc) rc = cuda_check(c, cudaMemcpy(c->d.Z0, fb->d.Z0, nu * 8, cudaMemcpyDeviceToDevice), "fallback torus");
            if (rc) {
                cleanup();
                return rc;
            }
            // the mixed context's monodromies belong to the rejected iterate: the next point's
            // first evaluation recomputes them
            c->have_jac = false;
            fell_back = true;
        }
        if (pst != FSE_OK && (worst == FSE_OK || pst < worst)) worst = pst;
        cudaMemcpyAsync(Zs + (size_t)j * nu, c->d.Z0, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
        if (Z_out) cudaMemcpyAsync(Z_out + (size_t)j * nu, c->d.Z0, nu * 8, cudaMemcpyDeviceToHost, c->stream);
        // prediction error ||Z_pred - Z*|| / ||Z*||
        fse::vec_axpby(c, nu, 1.0, c->d.Z0, -1.0, Zp);
        fse::vec_norms2(c, nu, Zp, c->d.Z0, c->d.vec2);
        double h2[2];
        cudaMemcpyAsync(h2, c->d.vec2, 16, cudaMemcpyDeviceToHost, c->stream);
        cudaEventRecord(c->ev[5], c->stream);
        int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "continuation point");
        if (rc) {
            cleanup();
            return rc;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]);
        if (info) {
            info[j].newton_iters = it;
            info[j].evals = evals;
            info[j].res = rn;
            info[j].znorm = zn;
            info[j].pred_err = std::sqrt(h2[0]) / std::max(std::sqrt(h2[1]), 1e-300);
            info[j].ms = ms;
            info[j].status = pst;
            info[j].predictor = used_mlp ? FSE_PRED_MLP : FSE_PRED_SECANT;
            info[j].fallback = fell_back ? 1 : 0;
        }
        // ---- learning: the secant's correction Z_j - S_j of every accepted point j >= 2, its
        // POD, and the network trained on the scaled coefficients
        if (learn && j >= 2) {
            double* dj = Dsn + (size_t)(j - 2) * nu;
            cudaMemcpyAsync(dj, c->d.Z0, nu * 8, cudaMemcpyDeviceToDevice, c->stream);
            fse::vec_axpby(c, nu, -1.0, Sec, 1.0, dj);
            const int m = j - 1;   // corrections known
            if (m >= 2) {
                const bool rebuild = (m % std::max(1, o->pod_every) == 0) || r == 0;
                if (rebuild) {
                    const int rr = std::min(rmax, m - 1);
                    cudaMemcpyAsync(Sscr, Dsn, (size_t)m * nu * 8, cudaMemcpyDeviceToDevice, c->stream);
                    rc = fse::pod_build_dev(Sscr, (int)nu, m, rr, pmean, pbasis, sing.data(), c->stream);
                    if (rc) {
                        cleanup();
                        return set_err(c, rc, "POD build failed");
                    }
                    r = rr;
                    reff = 0;
                    while (reff < r && sing[reff] > 1e-8 * sing[0]) ++reff;
                }
                fse::pod_project(c, nu, r, m, pmean, pbasis, Dsn, coef);
                std::vector<double> ch((size_t)m * r);
                cudaMemcpyAsync(ch.data(), coef, ch.size() * 8, cudaMemcpyDeviceToHost, c->stream);
                rc = cuda_check(c, cudaStreamSynchronize(c->stream), "POD projection");
                if (rc) {
                    cleanup();
                    return rc;
                }
                const int no = o->pod_modes;
                std::vector<float> X((size_t)m * 3), T((size_t)m * no, 0.0f);
                // targets: coefficients divided by their RMS over the training set, mode by mode
                // (modes below the rank threshold are not learned)
                tmax = 0.0;
                for (int k = 0; k < reff; ++k) {
                    double s2 = 0.0;
                    for (int a = 0; a < m; ++a) s2 += ch[(size_t)a * r + k] * ch[(size_t)a * r + k];
                    tsc[k] = std::max(std::sqrt(s2 / m), 1e-300);
                }
                for (int a = 0; a < m; ++a) {
                    feats(o->omega1[a + 2], &X[(size_t)a * 3]);
                    for (int k = 0; k < reff; ++k) {
                        const double t = ch[(size_t)a * r + k] / tsc[k];
                        T[(size_t)a * no + k] = (float)t;
                        tmax = std::max(tmax, 2.0 * std::fabs(t));
                    }
                }
                float loss = 0.f;
                rc = fse_mlp_train(mlp, X.data(), T.data(), m, o->train_steps, o->lr, &loss);
                if (rc) {
                    cleanup();
                    return set_err(c, rc, "network training failed");
                }
            }
        }
    }
    cleanup();
    return worst;
}
