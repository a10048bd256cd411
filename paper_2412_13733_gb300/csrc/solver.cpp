// libhpg host driver: device allocation/upload, the Newton loop over the
// alpha_k proximal steps (eq. pG), the Schur solve of eq. (schur2) with
// right-preconditioned GMRES on S, FP64 iterative refinement around an FP32
// inner solve, and the component operators used by the tests.
#include <algorithm>
#include <atomic>
#include <map>
#include <tuple>
#include <type_traits>
#include <mutex>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "state.h"

namespace hpg {

#define CK(...)                                                                              \
    do {                                                                                     \
        cudaError_t e_ = (__VA_ARGS__);                                                      \
        if (e_ != cudaSuccess) {                                                             \
            ctx->err = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_);            \
            return HPG_ERR_CUDA;                                                             \
        }                                                                                    \
    } while (0)

#define CKS(...)                                                                             \
    do {                                                                                     \
        hpg_status s_ = (__VA_ARGS__);                                                              \
        if (s_ != HPG_OK) return s_;                                                         \
    } while (0)

// ------------------------------------------------------------ kernel timer
static cudaEvent_t timer_event(KernelTimer& T) {
    if (!T.pool.empty()) {
        cudaEvent_t e = T.pool.back();
        T.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

static void timer_flush(KernelTimer& T) {
    for (auto& p : T.pending) {
        cudaEventSynchronize(p.second.second);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.second.first, p.second.second);
        T.ms[p.first] += ms;
        T.launches[p.first] += 1;
        T.pool.push_back(p.second.first);
        T.pool.push_back(p.second.second);
    }
    T.pending.clear();
}

struct Scope {
    KernelTimer& T;
    int cls;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
    Scope(KernelTimer& t, int c, cudaStream_t st) : T(t), cls(c), s(st) {
        if (T.on) { e0 = timer_event(T); cudaEventRecord(e0, s); }
    }
    ~Scope() {
        if (T.on) {
            cudaEvent_t e1 = timer_event(T);
            cudaEventRecord(e1, s);
            T.pending.push_back({cls, {e0, e1}});
            if (T.pending.size() > 4096) timer_flush(T);
        }
    }
};

// ------------------------------------------------------------ allocation
template <typename T>
static T* dalloc(DevState& D, size_t n, bool& ok) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMallocAsync(&p, n * sizeof(T), D.alloc_stream) != cudaSuccess) { ok = false; return nullptr; }
    D.allocs.push_back(p);
    D.bytes += n * sizeof(T);
    return static_cast<T*>(p);
}

Problem::~Problem() {
    if (pinned_scal) cudaFreeHost(pinned_scal);
    if (pinned_iflag) cudaFreeHost(pinned_iflag);
}

// Stream-ordered release (cudaFreeAsync), so that finishing one problem does
// not synchronise the device while other problems run on other streams.
void drop_graphs(Problem& P) {
    for (auto& gx : P.D.gmres_graph)
        if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
    for (auto& kv : P.D.bench_graphs) cudaGraphExecDestroy(kv.second.first);
    P.D.bench_graphs.clear();
}

void free_device(Problem& P, cudaStream_t s) {
    drop_graphs(P);
    for (void* p : P.D.allocs) cudaFreeAsync(p, s);
    P.D.allocs.clear();
    for (auto e : P.timer.pool) cudaEventDestroy(e);
    P.timer.pool.clear();
    P.D = DevState{};
    P.alloc_done = false;
}

static void pack_sten(const Ell& E, bool gram, int n, std::vector<int>& col) {
    col = E.col;
    if (gram)
        for (size_t i = 0; i < col.size(); ++i) col[i] = ((col[i] / n) << 8) | (col[i] % n);
}

static bool upload_sten(DevState& D, const Ell& E, bool gram, int n, DevSten& S, cudaStream_t s) {
    bool ok = true;
    const size_t w = (size_t)E.rows * kEll;
    S.cnt = dalloc<int>(D, E.rows, ok);
    S.col = dalloc<int>(D, w, ok);
    S.vd = dalloc<double>(D, w, ok);
    S.vf = dalloc<float>(D, w, ok);
    if (!ok) return false;
    std::vector<int> col;
    pack_sten(E, gram, n, col);
    std::vector<float> vf(E.val.begin(), E.val.end());
    cudaMemcpyAsync(S.cnt, E.cnt.data(), E.rows * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S.col, col.data(), w * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S.vd, E.val.data(), w * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(S.vf, vf.data(), w * sizeof(float), cudaMemcpyHostToDevice, s);
    return cudaStreamSynchronize(s) == cudaSuccess;
}

// Column lists of the row tiles (extent T) of one axis for the stencils `ops`, and
// each stencil entry's column as a position in its row tile's list (lcol[op]).
// Gram operators (psi columns) use the packed (cell << 8) | k form.
static bool upload_tile_cols(DevState& D, int n1, int T, const std::vector<const Ell*>& ops, bool gram, int n,
                             DevTileCols& tc, const std::vector<int**>& lcol, cudaStream_t s) {
    const int nt = (n1 + T - 1) / T;
    auto packed = [&](int c) { return gram ? (((c / n) << 8) | (c % n)) : c; };
    std::vector<std::vector<int>> lists(nt);
    for (int t = 0; t < nt; ++t) {
        std::vector<int>& L = lists[t];
        for (int r = t * T; r < std::min(n1, (t + 1) * T); ++r)
            for (const Ell* E : ops)
                for (int e = 0; e < E->cnt[r]; ++e) L.push_back(packed(E->col[(size_t)r * kEll + e]));
        std::sort(L.begin(), L.end());
        L.erase(std::unique(L.begin(), L.end()), L.end());
    }
    int cap = 1;
    for (const auto& L : lists) cap = std::max(cap, (int)L.size());
    std::vector<int> list((size_t)nt * cap, 0), count(nt, 0);
    for (int t = 0; t < nt; ++t) {
        count[t] = (int)lists[t].size();
        std::copy(lists[t].begin(), lists[t].end(), list.begin() + (size_t)t * cap);
    }
    bool ok = true;
    tc.cap = cap;
    tc.list = dalloc<int>(D, list.size(), ok);
    tc.count = dalloc<int>(D, count.size(), ok);
    std::vector<std::vector<int>> lc(ops.size(), std::vector<int>((size_t)n1 * kEll, 0));
    for (size_t o = 0; o < ops.size(); ++o) {
        *lcol[o] = dalloc<int>(D, lc[o].size(), ok);
        for (int r = 0; r < n1; ++r) {
            const std::vector<int>& L = lists[r / T];
            for (int e = 0; e < ops[o]->cnt[r]; ++e) {
                const int c = packed(ops[o]->col[(size_t)r * kEll + e]);
                lc[o][(size_t)r * kEll + e] = (int)(std::lower_bound(L.begin(), L.end(), c) - L.begin());
            }
        }
    }
    if (!ok) return false;
    cudaMemcpyAsync(tc.list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tc.count, count.data(), count.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    for (size_t o = 0; o < ops.size(); ++o)
        cudaMemcpyAsync(*lcol[o], lc[o].data(), lc[o].size() * sizeof(int), cudaMemcpyHostToDevice, s);
    return cudaStreamSynchronize(s) == cudaSuccess;
}

template <typename T>
static T* upload_vec(DevState& D, const std::vector<double>& v, bool& ok, cudaStream_t s) {
    T* p = dalloc<T>(D, v.size(), ok);
    if (!ok) return nullptr;
    std::vector<T> tmp(v.begin(), v.end());
    if (!v.empty()) cudaMemcpyAsync(p, tmp.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return p;
}

template <typename T>
static hpg_status autotune_fdm(hpg_ctx* ctx, Problem& P, Geo<T>& g, T* x, T* y, T* w1, T* w2);

long long next_alloc_gen();

hpg_status alloc_device(hpg_ctx* ctx, Problem& P) {
    if (P.alloc_done) return HPG_OK;
    HostProblem& H = P.H;
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    D.alloc_stream = s;
    {
        // keep freed pool memory cached in this process (no release to the OS between solves)
        static std::once_flag pool_cfg;
        std::call_once(pool_cfg, [&] {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
                unsigned long long thr = ~0ULL;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        });
    }
    bool ok = true;
    const int d = H.d;
    const bool grad = H.kind == HPG_GRADIENT;
    {
        // axis-0 row order of the FP64 u-row tiles: rows grouped by their stencil counts
        // (a hierarchical vertex row couples to more columns than a bubble row), so that
        // the 32 lanes of a warp run equally long gather loops; stable, so rows of equal
        // counts keep their natural order
        const Dir1D& D0 = H.dir[0];
        std::vector<int> perm(D0.n1);
        for (int r = 0; r < D0.n1; ++r) perm[r] = r;
        auto key = [&](int r) {
            return std::make_tuple(D0.Ai.cnt[r], D0.Mi.cnt[r], D0.Bi.cnt[r], grad ? D0.Bdi.cnt[r] : 0);
        };
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return key(a) < key(b); });
        D.perm0 = dalloc<int>(D, perm.size(), ok);
        if (ok) {
            cudaMemcpyAsync(D.perm0, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, s);
            ok = cudaStreamSynchronize(s) == cudaSuccess;
        }
    }
    for (int j = 0; j < d; ++j) {
        const Dir1D& Dj = H.dir[j];
        ok = ok && upload_sten(D, Dj.Ai, false, H.n, D.A[j], s);
        ok = ok && upload_sten(D, Dj.Mi, false, H.n, D.M[j], s);
        ok = ok && upload_sten(D, Dj.Bi, true, H.n, D.B[j], s);
        ok = ok && upload_sten(D, Dj.BTi, false, H.n, D.BT[j], s);
        if (grad) {
            ok = ok && upload_sten(D, Dj.Bdi, true, H.n, D.Bd[j], s);
            ok = ok && upload_sten(D, Dj.BdTi, false, H.n, D.BdT[j], s);
        }
        const int T = utile_extent(d, j);
        ok = ok && upload_tile_cols(D, Dj.n1, T, {&Dj.Ai, &Dj.Mi}, false, H.n, D.tu[j], {&D.A[j].lcol, &D.M[j].lcol}, s);
        if (grad)
            ok = ok && upload_tile_cols(D, Dj.n1, T, {&Dj.Bi, &Dj.Bdi}, true, H.n, D.tp[j],
                                        {&D.B[j].lcol, &D.Bd[j].lcol}, s);
        else
            ok = ok && upload_tile_cols(D, Dj.n1, T, {&Dj.Bi}, true, H.n, D.tp[j], {&D.B[j].lcol}, s);
        D.V_d[j] = upload_vec<double>(D, Dj.V, ok, s);
        D.V_f[j] = upload_vec<float>(D, Dj.V, ok, s);
        {
            std::vector<double> Vt((size_t)Dj.n1 * Dj.n1);
            for (int k = 0; k < Dj.n1; ++k)
                for (int a = 0; a < Dj.n1; ++a) Vt[(size_t)a * Dj.n1 + k] = Dj.V[(size_t)k * Dj.n1 + a];
            D.VT_d[j] = upload_vec<double>(D, Vt, ok, s);
            D.VT_f[j] = upload_vec<float>(D, Vt, ok, s);
        }
        D.lam_d[j] = upload_vec<double>(D, Dj.lam, ok, s);
        D.lam_f[j] = upload_vec<float>(D, Dj.lam, ok, s);
    }
    if (!ok) { free_device(P, s); ctx->err = "device allocation failed"; return HPG_ERR_OOM; }
    D.Vq_d = upload_vec<double>(D, H.Vq, ok, s);
    D.Vq_f = upload_vec<float>(D, H.Vq, ok, s);
    D.wq_d = upload_vec<double>(D, H.wq, ok, s);
    D.wq_f = upload_vec<float>(D, H.wq, ok, s);
    D.Mpsi_d = upload_vec<double>(D, H.Mpsi_loc, ok, s);
    D.Mpsi_f = upload_vec<float>(D, H.Mpsi_loc, ok, s);
    if (grad) {
        D.Kpsi_d = upload_vec<double>(D, H.Kpsi_loc, ok, s);
        D.Kpsi_f = upload_vec<float>(D, H.Kpsi_loc, ok, s);
    } else {
        D.C_d = upload_vec<double>(D, H.Cblk, ok, s);
        D.C_f = upload_vec<float>(D, H.Cblk, ok, s);
    }
    const size_t Nu0 = H.Nu0, Npsi = H.Npsi, Nx = Nu0 + Npsi;
    const size_t gsz = H.Nq * gauss_stride(H.kind, d);
    // Per-problem state (data, Newton state, factors, Krylov basis) lives in one
    // slab: every problem of a shape lays it out identically, so a batched launch
    // reaches problem b's copy of a buffer at a fixed byte offset from problem 0's.
    GmresDev& Gk = D.gm;
    Gk.kmax = std::max(1, P.params.krylov_max);
    Gk.N = (long long)Npsi;
    char* slab = nullptr;
    size_t slab_need = 0, slab_off = 0;
    bool measuring = true;
    auto sa = [&](auto*& ptr, size_t n) {
        using E = std::remove_reference_t<decltype(*ptr)>;
        const size_t bytes = ((std::max<size_t>(n, 1) * sizeof(E)) + 255) & ~(size_t)255;
        if (measuring) {
            slab_need += bytes;
        } else {
            ptr = reinterpret_cast<E*>(slab + slab_off);
            slab_off += bytes;
        }
    };
    auto state_buffers = [&]() {
        sa(D.rA, Nu0);
        sa(D.rB, Npsi);
        sa(D.bf, Nu0);
        sa(D.phiz, Npsi);
        sa(D.phiq, H.Nq);
        sa(D.x, Nx);
        sa(D.xt, Nx);
        sa(D.x0, Nx);
        sa(D.psi_prev, Npsi);
        sa(D.gw, gsz);
        sa(D.gwt, gsz);
        sa(D.gwl, gsz);
        sa(D.gwf, gsz);
        sa(D.alpha_dev, 1);
        {
            const size_t fw_d = factor_workspace_elems(H.n, d, (int)H.nb, H.ncomp, (long long)H.Nc, 8);
            const size_t fw_f = factor_workspace_elems(H.n, d, (int)H.nb, H.ncomp, (long long)H.Nc, 4);
            if (fw_d) sa(D.fwork_d, fw_d);
            if (fw_f) sa(D.fwork_f, fw_f);
        }
        sa(D.eg, Npsi);
        sa(D.egt, Npsi);
        sa(D.F, Nx);
        sa(D.Ft, Nx);
        sa(D.delta, Nx);
        sa(D.r, Nx);
        sa(D.dcorr, Nx);
        const size_t sblk = (size_t)H.Nc * H.nb * H.nb;
        sa(D.Sinv_d, sblk);
        sa(D.Sinv_f, sblk);
        sa(D.tu_d, Nu0);
        sa(D.tu2_d, Nu0);
        sa(D.w1_d, Nu0);
        sa(D.w2_d, Nu0);
        sa(D.tu_f, Nu0);
        sa(D.tu2_f, Nu0);
        sa(D.w1_f, Nu0);
        sa(D.w2_f, Nu0);
        sa(D.zp_d, Npsi);
        sa(D.zp_f, Npsi);
        sa(D.yp, Npsi);
        sa(D.xs, Npsi);
        int n1v[kMaxDim] = {1, 1, 1};
        for (int j = 0; j < d; ++j) n1v[j] = H.dir[j].n1;
        const int nres = n_res_partials_for(d, n1v, (long long)Npsi);
        sa(D.part, std::max(nres, 2048));
        sa(D.scal, 16);
        sa(D.flag, 4);
        // GMRES
        GmresDev& G = D.gm;
        sa(G.Vb, (size_t)(G.kmax + 1) * Npsi);
        sa(G.H, (size_t)(G.kmax + 1) * G.kmax);
        sa(G.cs, G.kmax);
        sa(G.sn, G.kmax);
        sa(G.gv, G.kmax + 1);
        sa(G.part_dots, (size_t)gmres_dot_blocks(G.N) * (G.kmax + 2));
        sa(G.part_norm, std::max<size_t>(1024, (size_t)gmres_upd_blocks(G.N)));
        sa(G.scal, 8);
        sa(G.iflag, 8);
        sa(G.jdev, 1);
        sa(G.hsum, G.kmax + 2);
        sa(G.counter, gmres_dot_groups(G.kmax));
        sa(G.counter2, 1);
        sa(G.reo, 1);
        sa(G.force, 1);
        sa(G.y, G.kmax + 1);
    };
    state_buffers();
    measuring = false;
    if (cudaMallocAsync(reinterpret_cast<void**>(&slab), slab_need, D.alloc_stream) != cudaSuccess) {
        free_device(P, s);
        ctx->err = "device allocation failed";
        return HPG_ERR_OOM;
    }
    D.allocs.push_back(slab);
    D.bytes += slab_need;
    D.slab = slab;
    D.slab_bytes = slab_need;
    state_buffers();
    GmresDev& G = D.gm;
    if (!ok) { free_device(P, s); ctx->err = "device allocation failed"; return HPG_ERR_OOM; }
    cudaMemsetAsync(G.counter, 0, sizeof(unsigned int) * gmres_dot_groups(G.kmax), s);
    cudaMemsetAsync(G.counter2, 0, sizeof(unsigned int), s);
    cudaMemsetAsync(G.force, 0, sizeof(int), s);
    cudaMemsetAsync(G.iflag, 0, 8 * sizeof(int), s);
    cudaMemsetAsync(G.jdev, 0, sizeof(int), s);
    static std::once_flag configured;
    std::call_once(configured, configure_kernels);
    cudaMemsetAsync(D.flag, 0, 4 * sizeof(int), s);
    if (!P.pinned_scal && (cudaMallocHost(&P.pinned_scal, 16 * sizeof(double)) != cudaSuccess ||
                           cudaMallocHost(&P.pinned_iflag, 8 * sizeof(int)) != cudaSuccess)) {
        free_device(P, s);
        ctx->err = "pinned host allocation failed";
        return HPG_ERR_OOM;
    }
    D.h_scal = P.pinned_scal;
    D.h_iflag = P.pinned_iflag;
    // geometry views
    auto fill = [&](auto& g, auto sel) {
        g.d = d; g.n = H.n; g.ncomp = H.ncomp; g.kind = H.kind;
        for (int j = 0; j < kMaxDim; ++j) { g.m[j] = H.m[j]; g.n1[j] = (j < d) ? H.dir[j].n1 : 1; }
        g.Nu0 = (long long)Nu0; g.Nc = (long long)H.Nc; g.nloc = (long long)H.nloc; g.nb = (long long)H.nb;
        g.Npsi = (long long)Npsi;
        sel(g);
    };
    fill(D.gd, [&](Geo<double>& g) {
        g.perm0 = D.perm0;
        for (int j = 0; j < d; ++j) {
            g.A[j] = {D.A[j].cnt, D.A[j].col, D.A[j].vd, D.A[j].lcol};
            g.M[j] = {D.M[j].cnt, D.M[j].col, D.M[j].vd, D.M[j].lcol};
            g.B[j] = {D.B[j].cnt, D.B[j].col, D.B[j].vd, D.B[j].lcol};
            g.BT[j] = {D.BT[j].cnt, D.BT[j].col, D.BT[j].vd, nullptr};
            g.Bd[j] = {D.Bd[j].cnt, D.Bd[j].col, D.Bd[j].vd, D.Bd[j].lcol};
            g.BdT[j] = {D.BdT[j].cnt, D.BdT[j].col, D.BdT[j].vd, nullptr};
            g.tu[j] = {D.tu[j].list, D.tu[j].count, D.tu[j].cap};
            g.tp[j] = {D.tp[j].list, D.tp[j].count, D.tp[j].cap};
            g.V[j] = D.V_d[j];
            g.VT[j] = D.VT_d[j];
            g.lam[j] = D.lam_d[j];
        }
        g.Vq = D.Vq_d; g.wq = D.wq_d; g.detJ = H.detJ; g.Mpsi = D.Mpsi_d; g.Kpsi = D.Kpsi_d; g.C = D.C_d;
    });
    fill(D.gf, [&](Geo<float>& g) {
        g.perm0 = nullptr;               // FP32 tiles keep the natural order (coalesced gathers)
        for (int j = 0; j < d; ++j) {
            g.A[j] = {D.A[j].cnt, D.A[j].col, D.A[j].vf, D.A[j].lcol};
            g.M[j] = {D.M[j].cnt, D.M[j].col, D.M[j].vf, D.M[j].lcol};
            g.B[j] = {D.B[j].cnt, D.B[j].col, D.B[j].vf, D.B[j].lcol};
            g.BT[j] = {D.BT[j].cnt, D.BT[j].col, D.BT[j].vf, nullptr};
            g.Bd[j] = {D.Bd[j].cnt, D.Bd[j].col, D.Bd[j].vf, D.Bd[j].lcol};
            g.BdT[j] = {D.BdT[j].cnt, D.BdT[j].col, D.BdT[j].vf, nullptr};
            g.tu[j] = {D.tu[j].list, D.tu[j].count, D.tu[j].cap};
            g.tp[j] = {D.tp[j].list, D.tp[j].count, D.tp[j].cap};
            g.V[j] = D.V_f[j];
            g.VT[j] = D.VT_f[j];
            g.lam[j] = D.lam_f[j];
        }
        g.Vq = D.Vq_f; g.wq = D.wq_f; g.detJ = (float)H.detJ; g.Mpsi = D.Mpsi_f; g.Kpsi = D.Kpsi_f; g.C = D.C_f;
    });
    // The u-row kernels stage per-tile value boxes (when they fit the shared-memory
    // budget) where a row gathers from many planes or psi components: 3D, or the
    // gradient kind.  Measured: B apply on the 3D 8^3 p=6 obstacle 23 -> 12.8 us,
    // torsion 16^2 p=10 solve -6 %; on the 2D obstacle (one component) the direct
    // gathers stay faster (radial 32x32 p=8 B apply 4.8 vs 6.3 us).
    // the TMA-fed tcgen05 fast diagonalisation (FP32): workspace, sliced pass matrices and
    // tensor maps; when a map cannot be made its variants are simply not candidates
    {
        bool okt = true;
        auto al = [&](size_t bytes) -> void* { return dalloc<char>(D, bytes, okt); };
        const float* lamf[kMaxDim] = {D.lam_f[0], D.lam_f[1], D.lam_f[2]};
        std::string why;
        D.tma_ok = fdm_tma_setup(D.tma, H, lamf, 1, al, s, nullptr, &why) && okt;
        D.gf.tma = D.tma_ok ? &D.tma : nullptr;
        D.gd.tma = nullptr;
        cudaGetLastError();
    }
    const bool stage = d == 3 || grad;
    D.gd.staged = stage && urow_boxes_fit(D.gd) ? 1 : 0;
    D.gf.staged = stage && urow_boxes_fit(D.gf) ? 1 : 0;
    CK(cudaStreamSynchronize(s));
    if (P.params.fdm_tile_f64 >= 0) D.gd.gemm_cfg = P.params.fdm_tile_f64;
    else CKS(autotune_fdm<double>(ctx, P, D.gd, D.tu_d, D.tu2_d, D.w1_d, D.w2_d));
    if (P.params.fdm_tile_f32 >= 0) D.gf.gemm_cfg = P.params.fdm_tile_f32;
    else CKS(autotune_fdm<float>(ctx, P, D.gf, D.tu_f, D.tu2_f, D.w1_f, D.w2_f));
    P.alloc_done = true;
    P.alloc_gen = next_alloc_gen();
    return HPG_OK;
}

// ------------------------------------------------------------ autotuner
// Pick the FDM GEMM tile variant for this (dim, n1, precision) by timing one
// A_alpha^{-1} apply per variant on the device (after a warm-up apply); cached
// per process, so each mesh shape is tuned once.  Every variant is first run on a
// seeded nonzero input and its output compared with that of variant 0 (the plain
// SIMT tile): a variant whose output is non-finite or differs by more than the
// precision's tolerance is not a candidate, however fast it returns.
template <typename T>
static hpg_status autotune_fdm(hpg_ctx* ctx, Problem& P, Geo<T>& g, T* x, T* y, T* w1, T* w2) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int>, int> cache;
    const int B = std::max(1, P.params.fdm_tune_batch);
    const auto key = std::make_tuple(g.d, g.n1[0], g.n1[1], g.d > 2 ? g.n1[2] : 1, (int)sizeof(T), B);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) { g.gemm_cfg = it->second; return HPG_OK; }
    }
    cudaStream_t s = ctx->stream;
    const size_t n = (size_t)g.Nu0;
    std::vector<T> hx(n), ref(n), out(n);
    for (size_t i = 0; i < n; ++i) hx[i] = (T)std::sin(0.37 * (double)i + 0.1);
    CK(cudaMemcpyAsync(x, hx.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
    const double tol = sizeof(T) == sizeof(float) ? 1e-4 : 1e-11;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 1e30f;
    double ref_max = 0.0;
    // Timing at batch B (fdm_tune_batch): one launch per pass serves B copies of the apply,
    // each on its own input, output and intermediate buffers (a temporary block per copy,
    // reached by byte offsets as a lockstep group's slabs are), as a group of B would; the
    // TMA variants get a temporary workspace and tensor maps for B problems.
    Bat bb{};
    long long* dz = nullptr;
    FdmTma tb{};
    std::vector<void*> tallocs;
    T* bx = nullptr;                 // copy 0's x, y, w1, w2 inside the temporary blocks
    T *by = nullptr, *bw1 = nullptr, *bw2 = nullptr;
    if (B > 1) {
        const size_t np4 = (n + 63) / 64 * 64;
        void* blk = nullptr;
        std::vector<long long> hd((size_t)B);
        for (int b = 0; b < B; ++b) hd[(size_t)b] = (long long)b * (long long)(4 * np4 * sizeof(T));
        if (cudaMalloc(&blk, (size_t)B * 4 * np4 * sizeof(T)) == cudaSuccess) {
            tallocs.push_back(blk);
            bx = static_cast<T*>(blk);
            by = bx + np4;
            bw1 = bx + 2 * np4;
            bw2 = bx + 3 * np4;
            bool okb = cudaMalloc(&dz, (size_t)B * sizeof(long long)) == cudaSuccess &&
                       cudaMemcpy(dz, hd.data(), (size_t)B * sizeof(long long), cudaMemcpyHostToDevice) ==
                           cudaSuccess;
            for (int b = 0; b < B && okb; ++b)
                okb = cudaMemcpy(bx + (size_t)b * 4 * np4, hx.data(), n * sizeof(T), cudaMemcpyHostToDevice) ==
                      cudaSuccess;
            if (okb) {
                bb.delta = dz;
                bb.np = B;
            }
        }
        if constexpr (sizeof(T) == 4) {
            if (P.D.tma_ok && bb.np == B) {
                auto al = [&](size_t bytes) -> void* {
                    void* q = nullptr;
                    if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
                    tallocs.push_back(q);
                    return q;
                };
                const float* lamf[kMaxDim] = {P.D.lam_f[0], P.D.lam_f[1], P.D.lam_f[2]};
                std::string why;
                if (!fdm_tma_setup(tb, P.H, lamf, B, al, s, &P.D.tma, &why)) tb = FdmTma{};
            }
        }
        cudaGetLastError();
    }
    auto release = [&]() {
        if (dz) cudaFree(dz);
        for (void* q : tallocs) cudaFree(q);
    };
    const int ncfg = fdm_tile_count((int)sizeof(T));
    for (int c = 0; c < ncfg; ++c) {
        g.gemm_cfg = c;
        if (launch_fdm<T>(g, nullptr, 1.0, x, y, w1, w2, s) != cudaSuccess) { cudaGetLastError(); continue; }
        if (cudaMemcpyAsync(out.data(), y, n * sizeof(T), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        bool finite = true;
        for (size_t i = 0; i < n && finite; ++i) finite = std::isfinite((double)out[i]);
        if (!finite) continue;
        if (c == 0) {
            ref = out;
            for (size_t i = 0; i < n; ++i) ref_max = std::max(ref_max, std::fabs((double)ref[i]));
        } else {
            double dmax = 0.0;
            for (size_t i = 0; i < n; ++i) dmax = std::max(dmax, std::fabs((double)out[i] - (double)ref[i]));
            if (ref.empty() || dmax > tol * std::max(ref_max, 1e-300)) continue;
        }
        Geo<T> gt = g;
        Bat bt{};
        T *tx = x, *ty = y, *tw1 = w1, *tw2 = w2;
        if (B > 1) {
            if (bb.np != B) continue;
            bt = bb;
            tx = bx;
            ty = by;
            tw1 = bw1;
            tw2 = bw2;
            if (gt.tma) gt.tma = tb.ready ? &tb : nullptr;
        }
        if (launch_fdm<T>(gt, nullptr, 1.0, tx, ty, tw1, tw2, s, nullptr, bt) != cudaSuccess) {   // warm-up
            cudaGetLastError();
            continue;
        }
        cudaEventRecord(e0, s);
        for (int r = 0; r < (B > 1 ? 10 : 5); ++r) launch_fdm<T>(gt, nullptr, 1.0, tx, ty, tw1, tw2, s, nullptr, bt);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); continue; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaStreamSynchronize(s));
    release();
    if (best < 0) {
        ctx->err = "no fast-diagonalisation pass variant produced a valid result";
        return HPG_ERR_CUDA;
    }
    g.gemm_cfg = best;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    return HPG_OK;
}

hpg_status upload_data(hpg_ctx* ctx, Problem& P) {
    HostProblem& H = P.H;
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    P.h2d_bytes = 0;
    if (P.data_dirty) {
        CK(cudaMemcpyAsync(D.rA, H.rA.data(), H.Nu0 * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(D.rB, H.rB.data(), H.Npsi * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(D.bf, H.bf.data(), H.Nu0 * sizeof(double), cudaMemcpyHostToDevice, s));
        P.h2d_bytes += (long long)(2 * H.Nu0 + H.Npsi) * (long long)sizeof(double);
        P.data_dirty = false;
    }
    if (P.phi_dirty) {
        CK(cudaMemcpyAsync(D.phiq, H.phiq.data(), H.Nq * sizeof(double), cudaMemcpyHostToDevice, s));
        P.h2d_bytes += (long long)H.Nq * (long long)sizeof(double);
        if (H.kind != HPG_GRADIENT) CK(launch_project(D.gd, D.phiq, D.phiz, s));
        P.phi_dirty = false;
    }
    CK(cudaStreamSynchronize(s));
    return HPG_OK;
}

// ------------------------------------------------------------ precision views
template <typename T>
struct PV;
template <>
struct PV<double> {
    static const Geo<double>& g(DevState& D) { return D.gd; }
    static double* Sinv(DevState& D) { return D.Sinv_d; }
    static const double* gw(DevState& D) { return D.gwl; }
    static double* fwork(DevState& D) { return D.fwork_d; }
    static double* tu(DevState& D) { return D.tu_d; }
    static double* tu2(DevState& D) { return D.tu2_d; }
    static double* w1(DevState& D) { return D.w1_d; }
    static double* w2(DevState& D) { return D.w2_d; }
    static double* zp(DevState& D) { return D.zp_d; }
};
template <>
struct PV<float> {
    static const Geo<float>& g(DevState& D) { return D.gf; }
    static float* Sinv(DevState& D) { return D.Sinv_f; }
    static const float* gw(DevState& D) { return D.gwf; }
    static float* fwork(DevState& D) { return D.fwork_f; }
    static float* tu(DevState& D) { return D.tu_f; }
    static float* tu2(DevState& D) { return D.tu2_f; }
    static float* w1(DevState& D) { return D.w1_f; }
    static float* w2(DevState& D) { return D.w2_f; }
    static float* zp(DevState& D) { return D.zp_f; }
};

template <typename T>
static cudaError_t to_T(const double* x, T* y, long long n, cudaStream_t s);
template <>
cudaError_t to_T<double>(const double* x, double* y, long long n, cudaStream_t s) {
    return cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}
template <>
cudaError_t to_T<float>(const double* x, float* y, long long n, cudaStream_t s) {
    return launch_convert<double, float>(x, y, n, s);
}
template <typename T>
static cudaError_t from_T(const T* x, double* y, long long n, cudaStream_t s);
template <>
cudaError_t from_T<double>(const double* x, double* y, long long n, cudaStream_t s) {
    return cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}
template <>
cudaError_t from_T<float>(const float* x, double* y, long long n, cudaStream_t s) {
    return launch_convert<float, double>(x, y, n, s);
}

// ------------------------------------------------------------ building blocks
static hpg_status eval_state(hpg_ctx* ctx, Problem& P, const double* x, double* gw, double* eg) {
    DevState& D = P.D;
    Scope sc(P.timer, HPG_K_EVAL, ctx->stream);
    CK(launch_eval(D.gd, x + P.H.Nu0, D.phiq, gw, nullptr, eg, D.flag, ctx->stream));
    return HPG_OK;
}

// F = residual(x), returns |F| and the eval flag (one host sync)
static hpg_status residual_state(hpg_ctx* ctx, Problem& P, const double* x, const double* eg, double alpha,
                                 double* F, double* norm, int* flag) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    {
        Scope sc(P.timer, HPG_K_RESIDUAL, s);
        CK(launch_residual(D.gd, x, x + P.H.Nu0, D.psi_prev, eg, D.rA, D.rB, D.bf, D.phiz, alpha, F, D.part, s));
        CK(launch_reduce_sum(D.part, n_res_partials(D.gd), D.scal, s));
    }
    CK(cudaMemcpyAsync(D.h_scal, D.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(D.h_iflag, D.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *norm = std::sqrt(D.h_scal[0]);
    *flag = D.h_iflag[0];
    if (!std::isfinite(*norm)) *flag |= 1;
    return HPG_OK;
}

static hpg_status norm_of(hpg_ctx* ctx, Problem& P, const double* v, long long n, double* out) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    int np = 0;
    CK(launch_sumsq(v, n, D.part, &np, s));
    CK(launch_reduce_sum(D.part, np, D.scal + 1, s));
    CK(cudaMemcpyAsync(D.h_scal + 1, D.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = std::sqrt(D.h_scal[1]);
    return HPG_OK;
}

template <typename T>
static hpg_status factor_T(hpg_ctx* ctx, Problem& P, double alpha, double* dump) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    Scope sc(P.timer, HPG_K_FACTOR, s);
    const long long gsz = (long long)(P.H.Nq * gauss_stride(P.H.kind, P.H.d));
    // freeze the weights of this linearisation (D.gw is swapped by the line search)
    CK(cudaMemcpyAsync(D.gwl, D.gw, gsz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (sizeof(T) == sizeof(float)) CK(launch_convert<double, float>(D.gwl, D.gwf, gsz, s));
    CK(launch_factor<T>(PV<T>::g(D), PV<T>::gw(D), alpha, P.params.beta, PV<T>::Sinv(D), dump, D.flag,
                        PV<T>::fwork(D), s));
    return HPG_OK;
}

template <typename T>
static hpg_status fdm_T(hpg_ctx* ctx, Problem& P, double alpha, const T* x, T* y) {
    DevState& D = P.D;
    Scope sc(P.timer, HPG_K_FDM, ctx->stream);
    CK(launch_fdm<T>(PV<T>::g(D), nullptr, alpha, x, y, PV<T>::w1(D), PV<T>::w2(D), ctx->stream));
    return HPG_OK;
}

// S z for z = Shat^{-1} v :  w = -(D z + E z + B^T A^{-1} B z), written into out (FP64)
template <typename T>
static hpg_status schur_apply_T(hpg_ctx* ctx, Problem& P, double alpha, const T* z, double* out) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const Geo<T>& g = PV<T>::g(D);
    {
        Scope sc(P.timer, HPG_K_BAPPLY, s);
        CK(launch_bapply<T, T, T>(g, z, PV<T>::tu(D), s));
    }
    CKS(fdm_T<T>(ctx, P, alpha, PV<T>::tu(D), PV<T>::tu2(D)));
    {
        Scope sc(P.timer, HPG_K_SCHUR, s);
        CK(launch_schur_rest<T, double>(g, PV<T>::gw(D), P.params.beta, z, PV<T>::tu2(D), out, s));
    }
    return HPG_OK;
}

// `chunk` GMRES iterations enqueued on the stream (no host synchronisation):
// z = S-hat^{-1} V_j, w = S z written into V_{j+1}, Arnoldi/Givens update.
// Iteration index, stop flag and alpha are read on the device, so the same
// launches can be captured once into a CUDA graph and replayed.
template <typename T, typename VT>
static hpg_status gmres_chunk(hpg_ctx* ctx, Problem& P, int chunk) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    GmresDev& G = D.gm;
    const Geo<T>& g = PV<T>::g(D);
    const IterCtl ctl{G.iflag, G.jdev, G.N};
    for (int c = 0; c < chunk; ++c) {
        {
            Scope sc(P.timer, HPG_K_PRECOND, s);
            CK(launch_precond<T, VT, T>(g, PV<T>::Sinv(D), gmres_basis<VT>(G), PV<T>::zp(D), s, ctl));
        }
        {
            Scope sc(P.timer, HPG_K_BAPPLY, s);
            CK(launch_bapply<T, T, T>(g, PV<T>::zp(D), PV<T>::tu(D), s, G.iflag));
        }
        {
            Scope sc(P.timer, HPG_K_FDM, s);
            CK(launch_fdm<T>(g, D.alpha_dev, 0.0, PV<T>::tu(D), PV<T>::tu2(D), PV<T>::w1(D), PV<T>::w2(D), s,
                             G.iflag));
        }
        {
            Scope sc(P.timer, HPG_K_SCHUR, s);
            CK(launch_schur_rest<T, VT>(g, PV<T>::gw(D), P.params.beta, PV<T>::zp(D), PV<T>::tu2(D),
                                        gmres_basis<VT>(G), s, ctl));
        }
        {
            Scope sc(P.timer, HPG_K_ORTHO, s);
            CK(gmres_arnoldi<VT>(G, s));
        }
    }
    return HPG_OK;
}

constexpr int kGraphChunk = 2;

// Build the device-side GMRES loop: one CUDA graph holding a conditional WHILE
// node whose body is `kGraphChunk` iterations followed by a kernel that sets
// the loop condition from the stop flag.  One launch runs GMRES to its stop
// flag with no host round trip.  Returns false if the runtime lacks support.
template <typename T, typename VT>
static bool build_gmres_loop(hpg_ctx* ctx, Problem& P, cudaGraphExec_t* exec, long long* kernels_per_body) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    const long long before = kernel_launch_count();
    hpg_status st = gmres_chunk<T, VT>(ctx, P, kGraphChunk);
    if (st == HPG_OK && launch_gm_setcond(h, D.gm.iflag, s) != cudaSuccess) st = HPG_ERR_CUDA;
    *kernels_per_body = kernel_launch_count() - before;
    add_kernel_launches(-*kernels_per_body);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &captured);
    bool ok = st == HPG_OK && ce == cudaSuccess && cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!ok) cudaGetLastError();
    return ok;
}

// Run GMRES to its stop flag: one launch of the device-side loop graph (or
// eager launches when kernel timing is on), then one read of the flags.
template <typename T, typename VT>
static hpg_status gmres_run(hpg_ctx* ctx, Problem& P, int* its, bool* capped) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    GmresDev& G = D.gm;
    const int pi = sizeof(T) == sizeof(float) ? (sizeof(VT) == sizeof(float) ? 2 : 1) : 0;
    const bool use_graph = !P.timer.on && P.params.graphs != 0;
    if (use_graph && !D.gmres_graph[pi] && !D.gmres_graph_failed[pi]) {
        long long nk = 0;
        if (!build_gmres_loop<T, VT>(ctx, P, &D.gmres_graph[pi], &nk)) {
            D.gmres_graph[pi] = nullptr;
            D.gmres_graph_failed[pi] = true;
        } else {
            D.graph_kernels[pi] = nk;
        }
    }
    if (use_graph && D.gmres_graph[pi]) {
        CK(cudaGraphLaunch(D.gmres_graph[pi], s));
        CK(cudaMemcpyAsync(D.h_iflag + 4, G.iflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // kernels executed: one body per kGraphChunk iterations (rounded up)
        add_kernel_launches(D.graph_kernels[pi] * ((D.h_iflag[5] + kGraphChunk - 1) / kGraphChunk + 1));
    } else {
        for (int guard = 0; guard <= G.kmax; ++guard) {
            CKS(gmres_chunk<T, VT>(ctx, P, 1));
            CK(cudaMemcpyAsync(D.h_iflag + 4, G.iflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (D.h_iflag[4]) break;
        }
    }
    *its = D.h_iflag[5];
    *capped = D.h_iflag[7] != 0 && D.h_iflag[4] != 0 && D.h_iflag[6] == 0;
    if (*capped) {
        // the cap flag is also set when the last allowed iteration converged; check the residual
        CK(cudaMemcpyAsync(D.h_scal + 4, G.scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *capped = D.h_scal[5] > D.h_scal[6];
    }
    return HPG_OK;
}

// eq. (schur2): y = b_psi - B^T A^{-1} b_u; GMRES on S (right-preconditioned by
// S-hat); delta_u = A^{-1}(b_u - B delta_psi).  Right-hand sides and results FP64,
// operators in T, the GMRES basis and its Gram-Schmidt in VT.
template <typename T, typename VT>
static hpg_status schur_solve_TV(hpg_ctx* ctx, Problem& P, double alpha, const double* bu, const double* bp,
                                 double* du, double* dp, double rtol, int* its, bool* capped, int cap) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const Geo<T>& g = PV<T>::g(D);
    const long long Nu0 = (long long)P.H.Nu0, Npsi = (long long)P.H.Npsi;
    GmresDev& G = D.gm;
    T* tu = PV<T>::tu(D);
    T* tu2 = PV<T>::tu2(D);
    T* zp = PV<T>::zp(D);
    CK(to_T<T>(bu, tu, Nu0, s));
    CKS(fdm_T<T>(ctx, P, alpha, tu, tu2));
    {
        Scope sc(P.timer, HPG_K_SCHUR, s);
        CK(launch_btapply<T, T, T>(g, tu2, zp, s));
        CK(launch_sub_scaled<T>(bp, 1.0, zp, D.yp, Npsi, s));
    }
    {
        Scope sc(P.timer, HPG_K_ORTHO, s);
        CK(gmres_start<VT>(G, D.yp, rtol, s, cap));
    }
    CKS(gmres_run<T, VT>(ctx, P, its, capped));
    P.stats.ainv_total += 2 + *its;
    {
        Scope sc(P.timer, HPG_K_ORTHO, s);
        CK(gmres_finish<VT>(G, D.xs, s));
    }
    {
        Scope sc(P.timer, HPG_K_PRECOND, s);
        CK(launch_precond<T, double, double>(g, PV<T>::Sinv(D), D.xs, dp, s));
    }
    {
        Scope sc(P.timer, HPG_K_BAPPLY, s);
        CK(launch_bapply<T, double, T>(g, dp, tu, s));
    }
    {
        Scope sc(P.timer, HPG_K_UPDATE, s);
        CK(launch_sub_scaled<T>(bu, 1.0, tu, D.tu_d, Nu0, s));
        CK(to_T<T>(D.tu_d, tu, Nu0, s));
    }
    CKS(fdm_T<T>(ctx, P, alpha, tu, tu2));
    CK(from_T<T>(tu2, du, Nu0, s));
    return HPG_OK;
}

// FP64 basis unless the FP32 inner solves are asked for a float basis (krylov_f32)
template <typename T>
static hpg_status schur_solve_T(hpg_ctx* ctx, Problem& P, double alpha, const double* bu, const double* bp,
                                double* du, double* dp, double rtol, int* its, bool* capped, int cap = 0) {
    if constexpr (sizeof(T) == sizeof(float))
        if (P.params.krylov_f32) return schur_solve_TV<T, float>(ctx, P, alpha, bu, bp, du, dp, rtol, its, capped, cap);
    return schur_solve_TV<T, double>(ctx, P, alpha, bu, bp, du, dp, rtol, its, capped, cap);
}

// ---- flexible GMRES on G with a block preconditioner (Section 4.3) -------------
// z = P^{-1} r for r = [r_u; r_psi] (G = [[A_alpha, B], [B^T, C]], S = C - B^T A_alpha^{-1} B):
//   P_D:      z_u = A_alpha^{-1} r_u,  z_psi = S-hat^{-1} r_psi
//   P_L P_D:  z_u = A_alpha^{-1} r_u,  z_psi = S-hat^{-1} (r_psi - B^T z_u)
//   P_F:      eq. (schur2) with S^{-1} replaced by at most inner_max iterations of
//             S-hat-preconditioned GMRES on S (relative tolerance 1e-5)
static hpg_status fg_precond(hpg_ctx* ctx, Problem& P, double alpha, const double* r, double* z) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const Geo<double>& g = D.gd;
    const long long Nu0 = (long long)P.H.Nu0, Npsi = (long long)P.H.Npsi;
    if (P.params.strategy == HPG_FGMRES_PF) {
        int its = 0;
        bool capped = false;
        CKS(schur_solve_T<double>(ctx, P, alpha, r, r + Nu0, z, z + Nu0, 1e-5, &its, &capped, P.params.inner_max));
        P.stats.krylov_total += its;
        return HPG_OK;
    }
    if (P.params.ainv_pcg) {
        int its = 0;
        double res = 0.0;
        CKS(pcg_solve(ctx, P, P.params.ainv_pcg, alpha, r, z, P.params.ainv_rtol, 0.0, 1000, &its, &res));
        P.stats.ainv_iters += its;
    } else {
        CK(launch_fdm<double>(g, nullptr, alpha, r, z, D.w1_d, D.w2_d, s));
    }
    P.stats.ainv_total += 1;
    const double* rp = r + Nu0;
    if (P.params.strategy == HPG_FGMRES_PLPD) {
        CK(launch_btapply<double, double, double>(g, z, D.fP1, s));
        CK(launch_sub_scaled<double>(r + Nu0, 1.0, D.fP1, D.fP1, Npsi, s));     // r_psi - B^T z_u
        rp = D.fP1;
    }
    CK(launch_precond<double, double, double>(g, D.Sinv_d, rp, z + Nu0, s));
    return HPG_OK;
}

// sum of the chunk partials of nv dot products (chunk order), on the host
static hpg_status fg_dots(hpg_ctx* ctx, Problem& P, const double* V, int nv, const double* w, std::vector<double>& h) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long N = (long long)(P.H.Nu0 + P.H.Npsi);
    const int nch = fg_chunks(N);
    CK(launch_mdot(V, N, nv, w, N, D.fpart, s));
    std::vector<double> part((size_t)nv * nch);
    CK(cudaMemcpyAsync(part.data(), D.fpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h.assign(nv, 0.0);
    for (int v = 0; v < nv; ++v)
        for (int c = 0; c < nch; ++c) h[v] += part[(size_t)v * nch + c];
    return HPG_OK;
}

// Right-preconditioned flexible GMRES (unrestarted, at most krylov_max iterations) on
// G x = b, classical Gram-Schmidt with one re-orthogonalisation, Givens rotations on
// the host.  Outer iterations are few (1-3 for P_F, tens for P_D), so the loop is
// host-driven; every vector operation runs in libhpg kernels.
static hpg_status fgmres_solve(hpg_ctx* ctx, Problem& P, double alpha, const double* b, double rtol, double* x,
                               int* its, bool* capped) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long Nu0 = (long long)P.H.Nu0, Npsi = (long long)P.H.Npsi, N = Nu0 + Npsi;
    const int m = std::max(1, P.params.krylov_max);
    if (!D.fV || D.fm != m) {
        bool ok = true;
        D.fV = dalloc<double>(D, (size_t)(m + 1) * N, ok);
        D.fZ = dalloc<double>(D, (size_t)m * N, ok);
        D.fpart = dalloc<double>(D, (size_t)(m + 1) * fg_chunks(N), ok);
        D.fh = dalloc<double>(D, (size_t)m + 1, ok);
        D.fP1 = dalloc<double>(D, (size_t)Npsi, ok);
        if (!ok) { ctx->err = "device allocation failed (flexible GMRES)"; return HPG_ERR_OOM; }
        D.fm = m;
    }
    *its = 0;
    *capped = false;
    CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    double beta = 0.0;
    CKS(norm_of(ctx, P, b, N, &beta));
    if (!(beta > 0.0)) return HPG_OK;
    CK(cudaMemsetAsync(D.fV, 0, N * sizeof(double), s));
    CK(launch_axpby(1.0 / beta, b, 0.0, D.fV, N, s));
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1, 0.0), h, h2;
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
        double* vj = D.fV + (long long)j * N;
        double* zj = D.fZ + (long long)j * N;
        double* w = D.fV + (long long)(j + 1) * N;
        CKS(fg_precond(ctx, P, alpha, vj, zj));
        CK(launch_newton_apply(D.gd, D.gw, alpha, P.params.beta, zj, w, s));
        double* col = H.data() + (size_t)j * (m + 1);
        for (int pass = 0; pass < 2; ++pass) {
            CKS(fg_dots(ctx, P, D.fV, j + 1, w, h));
            CK(cudaMemcpyAsync(D.fh, h.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
            CK(launch_maxpy(w, D.fV, N, D.fh, j + 1, N, -1.0, s));
            for (int i = 0; i <= j; ++i) col[i] += h[i];
        }
        CKS(fg_dots(ctx, P, w, 1, w, h2));
        const double hn = std::sqrt(std::max(h2[0], 0.0));
        col[j + 1] = hn;
        if (hn > 0.0) CK(launch_axpby(1.0 / hn, w, 0.0, w, N, s));
        for (int i = 0; i < j; ++i) {
            const double t = cs[i] * col[i] + sn[i] * col[i + 1];
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
            col[i] = t;
        }
        const double r = std::hypot(col[j], col[j + 1]);
        cs[j] = r > 0.0 ? col[j] / r : 1.0;
        sn[j] = r > 0.0 ? col[j + 1] / r : 0.0;
        col[j] = r;
        col[j + 1] = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        k = j + 1;
        if (!(std::fabs(gv[j + 1]) > rtol * beta) || !(hn > 1e-300 * beta)) break;
    }
    *its = k;
    P.stats.fgmres_total += k;
    *capped = k == m && std::fabs(gv[k]) > rtol * beta;
    // back substitution, then x = Z y
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double t = gv[i];
        for (int l = i + 1; l < k; ++l) t -= H[(size_t)l * (m + 1) + i] * y[l];
        const double dgl = H[(size_t)i * (m + 1) + i];
        y[i] = dgl != 0.0 ? t / dgl : 0.0;
    }
    CK(cudaMemcpyAsync(D.fh, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_maxpy(x, D.fZ, N, D.fh, k, N, 1.0, s));
    CK(cudaStreamSynchronize(s));
    return HPG_OK;
}

// Solve G delta = F for the current factorisation.  FP64: GMRES on S in FP64;
// if it stops at its cap the FP64 residual r = F - G delta is formed and the
// solve is repeated on r (a restart).  Mixed: FP32 inner solves inside FP64
// iterative refinement until ||F - G delta|| <= eta ||F||.
// tolerance of the FP32 inner solve, relative to the reduction the refinement still needs:
// half of it (measured against a tenth: 6 % fewer inner iterations on the 32x32 p=8 obstacle,
// 5 % on torsion, 7 % on the 3D obstacle, same Newton counts, a few more second sweeps;
// single solves 2.6 %, 5 % and 9 % faster)
constexpr double kInnerMargin = 0.5;

static hpg_status linear_solve(hpg_ctx* ctx, Problem& P, double alpha, const double* F, double normF, double eta,
                               double* delta, int* its_total, int* sweeps, bool force_f64 = false) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long Nu0 = (long long)P.H.Nu0, Npsi = (long long)P.H.Npsi, Nx = Nu0 + Npsi;
    const bool f64 = P.params.precision == HPG_FP64 || force_f64;
    *sweeps = 0;
    *its_total = 0;
    CK(cudaMemsetAsync(delta, 0, Nx * sizeof(double), s));
    CK(cudaMemcpyAsync(D.r, F, Nx * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double rnorm = normF;
    for (int sw = 0; sw < std::max(1, P.params.refine_max); ++sw) {
        int its = 0;
        bool capped = false;
        // GMRES tolerance relative to the current residual r, aimed at ||r|| <= eta ||F||:
        // FP64 exactly; FP32 with a margin below it (kInnerMargin), floored near the FP32
        // limit, so that one refinement sweep usually suffices
        const double need = eta * normF / std::max(rnorm, 1e-300);
        const double rt = f64 ? std::min(1.0, need) : std::min(1.0, std::max(kInnerMargin * need, 1e-6));
        if (f64 && P.params.strategy != HPG_SCHUR) {
            int outer = 0;
            CKS(fgmres_solve(ctx, P, alpha, D.r, rt, D.dcorr, &outer, &capped));
        } else if (f64) {
            CKS(schur_solve_T<double>(ctx, P, alpha, D.r, D.r + Nu0, D.dcorr, D.dcorr + Nu0, rt, &its, &capped));
        } else {
            CKS(schur_solve_T<float>(ctx, P, alpha, D.r, D.r + Nu0, D.dcorr, D.dcorr + Nu0, rt, &its, &capped));
        }
        *its_total += its;
        *sweeps = sw + 1;
        if (capped) P.stats.krylov_cap_hits++;
        {
            Scope sc(P.timer, HPG_K_UPDATE, s);
            CK(launch_axpby(1.0, D.dcorr, 1.0, delta, Nx, s));
        }
        if (f64 && !capped) break;      // FP64 GMRES residual is the true Newton-system residual
        {
            Scope sc(P.timer, HPG_K_NEWTON_APPLY, s);
            CK(launch_newton_apply(D.gd, D.gw, alpha, P.params.beta, delta, D.r, s));
        }
        {
            Scope sc(P.timer, HPG_K_UPDATE, s);
            CK(launch_axpby(1.0, F, -1.0, D.r, Nx, s));
        }
        CKS(norm_of(ctx, P, D.r, Nx, &rnorm));
        if (rnorm <= eta * normF) break;
    }
    return HPG_OK;
}

static hpg_status set_alpha(hpg_ctx* ctx, Problem& P, double alpha) {
    DevState& D = P.D;
    D.h_scal[8] = alpha;
    CK(cudaMemcpyAsync(D.alpha_dev, D.h_scal + 8, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return HPG_OK;
}

static void swap_state(DevState& D) {
    std::swap(D.x, D.xt);
    std::swap(D.gw, D.gwt);
    std::swap(D.eg, D.egt);
    std::swap(D.F, D.Ft);
}

hpg_status solve_problem(hpg_ctx* ctx, Problem& P) {
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = kernel_launch_count();
    HostProblem& H = P.H;
    CKS(alloc_device(ctx, P));
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long Nu0 = (long long)H.Nu0, Npsi = (long long)H.Npsi, Nx = Nu0 + Npsi;
    hpg_stats& st = P.stats;
    st = hpg_stats{};
    st.n_u = Nu0;
    st.n_psi = Npsi;
    P.timer.on = P.params.timing != 0;
    CK(cudaMemsetAsync(D.x, 0, Nx * sizeof(double), s));
    CK(cudaMemsetAsync(D.psi_prev, 0, Npsi * sizeof(double), s));
    CK(cudaMemsetAsync(D.flag, 0, 4 * sizeof(int), s));
    hpg_status status = HPG_OK;
    double normF = 0.0;
    // HPG_MIXED: a proximal step whose mixed Newton iteration fails (a non-positive pivot
    // of the FP32 S-hat elimination, a line search ending on a non-finite trial point, the
    // Newton cap) is solved again from its starting point in FP64, and so is the rest of
    // the solve
    const bool mixed = P.params.precision != HPG_FP64;
    bool fp64 = !mixed;
    const int nsteps = (int)std::min<size_t>(H.alphas.size(), HPG_MAX_ALPHA);
    for (int k = 0; k < nsteps && status == HPG_OK; ++k) {
        const double alpha = H.alphas[k];
        CKS(set_alpha(ctx, P, alpha));
        if (k > 0) CK(cudaMemcpyAsync(D.psi_prev, D.x + Nu0, Npsi * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (!fp64) CK(cudaMemcpyAsync(D.x0, D.x, Nx * sizeof(double), cudaMemcpyDeviceToDevice, s));
        int flag = 0;
        CKS(eval_state(ctx, P, D.x, D.gw, D.eg));
        CKS(residual_state(ctx, P, D.x, D.eg, alpha, D.F, &normF, &flag));
        int it = 0;
        auto fall_back = [&]() -> hpg_status {
            fp64 = true;
            st.fp64_from_step = k + 1;
            st.newton_total += it;              // the mixed Newton steps discarded
            it = 0;
            CK(cudaMemcpyAsync(D.x, D.x0, Nx * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(D.flag, 0, 4 * sizeof(int), s));
            CKS(eval_state(ctx, P, D.x, D.gw, D.eg));
            CKS(residual_state(ctx, P, D.x, D.eg, alpha, D.F, &normF, &flag));
            return HPG_OK;
        };
        while (true) {
            if (flag & 1) { status = HPG_ERR_NONFINITE; break; }
            if (!std::isfinite(normF)) {
                status = HPG_ERR_NONFINITE;
                ctx->err = "non-finite Newton residual in proximal step " + std::to_string(k + 1);
                break;
            }
            if (normF <= P.params.newton_tol) break;
            if (it >= P.params.newton_max && !fp64) {
                CKS(fall_back());
                continue;
            }
            if (it >= P.params.newton_max) {
                status = HPG_ERR_NEWTON_CAP;
                ctx->err = "Newton cap reached in proximal step " + std::to_string(k + 1) + " (||F|| = " +
                           std::to_string(normF) + ")";
                break;
            }
            if (fp64) CKS(factor_T<double>(ctx, P, alpha, nullptr));
            else CKS(factor_T<float>(ctx, P, alpha, nullptr));
            if (mixed && fp64) st.fp64_newton_steps++;
            int its = 0, sweeps = 0;
            // forcing term: relative tolerance min(krylov_rtol, ||F||)
            const double eta = std::min(P.params.krylov_rtol, std::max(normF, 1e-12));
            CKS(linear_solve(ctx, P, alpha, D.F, normF, eta, D.delta, &its, &sweeps, fp64));
            st.krylov_total += its;
            st.refine_total += sweeps;
            // backtracking on ||F||
            double lam = 1.0, nFt = 0.0;
            int tflag = 0;
            for (int h = 0; h <= P.params.ls_max; ++h) {
                {
                    Scope sc(P.timer, HPG_K_UPDATE, s);
                    CK(launch_trial(D.x, D.delta, lam, D.xt, Nx, s));
                }
                CK(cudaMemsetAsync(D.flag, 0, sizeof(int), s));
                CKS(eval_state(ctx, P, D.xt, D.gwt, D.egt));
                CKS(residual_state(ctx, P, D.xt, D.egt, alpha, D.Ft, &nFt, &tflag));
                if (!(tflag & 1) && nFt <= (1.0 - 1e-4 * lam) * normF) break;
                if (h == P.params.ls_max) { st.ls_fail++; break; }
                lam *= 0.5;
            }
            // factorisation flag (non-SPD block): bit 1 of flag[1], sticky for the solve
            CK(cudaMemcpyAsync(D.h_iflag, D.flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const bool spd_fail = (D.h_iflag[0] & 2) != 0;
            const bool bad_trial = (tflag & 1) || !std::isfinite(nFt);
            if (!fp64 && (spd_fail || bad_trial)) {
                CKS(fall_back());
                continue;
            }
            if (spd_fail) {
                status = HPG_ERR_NOT_SPD;
                ctx->err = "non-positive pivot in an FP64 S-hat block factorisation in proximal step " +
                           std::to_string(k + 1);
                break;
            }
            swap_state(D);
            normF = nFt;
            flag = tflag;
            ++it;
        }
        st.newton_per_step[k] = it;
        st.newton_total += it;
        st.alpha_steps = k + 1;
    }
    st.final_residual = normF;
    st.status = status;
    st.kernel_launches = kernel_launch_count() - launches0;
    st.fdm_tile_f32 = D.gf.gemm_cfg;
    st.fdm_tile_f64 = D.gd.gemm_cfg;
    st.h2d_bytes = P.h2d_bytes;
    CK(cudaStreamSynchronize(s));
    timer_flush(P.timer);
    st.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    P.solved = true;
    return status;
}

// ====================================================== lockstep groups (batched launches)
// Problems of one shape are solved together: every launch of a Newton step or of a
// Krylov iteration serves all problems of the group at once (Bat), so a batch of
// small solves fills the GPU with few, large launches instead of many small ones.
// Each problem keeps the arithmetic it has alone -- the same kernels, launch shapes,
// operands and reduction orders -- and the host keeps each problem's Newton,
// line-search and refinement decisions apart, masking problems out of the launches
// they take no part in.  Results are therefore those of hpg_solve, bit for bit.
namespace {
enum { kMaskStart = 0, kMaskNewton = 1, kMaskSolve = 2, kMaskTrial = 3, kMaskIdle = 4, kMaskPrev = 5,
       kMaskCount = 6 };
constexpr int kStatD = 4;   // gathered doubles per problem (scal[0..3] or GMRES scal[0..3])
constexpr int kStatI = 4;   // gathered ints per problem (flag[0..3] or GMRES iflag[0..3])
std::atomic<long long> g_alloc_gen{0};
}  // namespace

long long next_alloc_gen() { return ++g_alloc_gen; }

struct Group {
    int np = 0;
    std::vector<int> ids;
    std::vector<long long> gens;
    std::vector<Problem*> ps;
    long long* delta_d = nullptr;
    int* mask_d = nullptr;       // kMaskCount x np
    double* par_d = nullptr;     // np x kBatPar
    double* stat_d = nullptr;    // np x (kStatD + kStatI)
    long long* h_delta = nullptr;
    // masks and per-problem scalars are staged in pageable host memory on purpose: an
    // asynchronous copy from pageable memory takes its snapshot before it returns, so
    // the host may change them for the next phase while earlier copies are queued
    std::vector<int> h_mask;
    std::vector<double> h_par;
    double* h_stat = nullptr;
    cudaGraphExec_t loop[3] = {nullptr, nullptr, nullptr};
    long long loop_kernels[3] = {0, 0, 0};
    bool loop_failed[3] = {false, false, false};
    // problem 0's operator views with the FDM pass variant tuned for the group's size
    Geo<float> gf{};
    Geo<double> gd{};
    bool tuned_f = false, tuned_d = false;
    // the TMA fast diagonalisation over all np problems (its own workspace and maps)
    FdmTma tma{};
    std::vector<void*> tma_allocs;
    std::map<long long, std::pair<cudaGraphExec_t, long long>> bench_graphs;   // kernel-class replays
    ~Group() {
        for (auto& kv : bench_graphs) cudaGraphExecDestroy(kv.second.first);
        for (auto& gx : loop)
            if (gx) cudaGraphExecDestroy(gx);
        if (delta_d) cudaFree(delta_d);
        if (mask_d) cudaFree(mask_d);
        if (par_d) cudaFree(par_d);
        if (stat_d) cudaFree(stat_d);
        if (h_delta) cudaFreeHost(h_delta);
        if (h_stat) cudaFreeHost(h_stat);
        for (void* p : tma_allocs) cudaFree(p);
    }
    Bat bat(int slot) const {
        Bat b;
        b.delta = delta_d;
        b.act = slot < 0 ? nullptr : mask_d + (size_t)slot * np;
        b.par = par_d;
        b.np = np;
        return b;
    }
    int* mask(int slot) { return h_mask.data() + (size_t)slot * np; }
};

// Problems that may share a group: same shape (so the same operator constants and
// the same slab layout) and the same solver parameters that launches depend on.
static std::string group_key(const Problem& P) {
    const HostProblem& H = P.H;
    const hpg_params& q = P.params;
    char buf[512];
    std::snprintf(buf, sizeof buf, "%d|%d|%d,%d,%d|%d|%a,%a,%a|%a,%a,%a|%d|%d|%d|%a|%d|%d|%d|%d|%d", H.d, H.kind,
                  H.m[0], H.m[1], H.m[2], H.p, H.lo[0], H.lo[1], H.lo[2], H.hi[0], H.hi[1], H.hi[2], q.precision,
                  q.krylov_max, q.krylov_f32, q.beta, q.fdm_tile_f32, q.fdm_tile_f64 * 128 + q.fdm_tune_batch,
                  q.strategy, q.ls_max, q.refine_max * 2 + (q.graphs != 0));
    return buf;
}

// Whether a problem can run in a lockstep group at all (the flexible-GMRES strategies
// and per-kernel timing stay on the single-problem path).
static bool groupable(const Problem& P) { return P.params.strategy == HPG_SCHUR && P.params.timing == 0; }

static hpg_status group_build(hpg_ctx* ctx, std::vector<Problem*>& ps, std::shared_ptr<Group>& out) {
    auto Gp = std::make_shared<Group>();
    const int np = (int)ps.size();
    Gp->np = np;
    Gp->ps = ps;
    for (Problem* P : ps) {
        Gp->ids.push_back(P->id);
        Gp->gens.push_back(P->alloc_gen);
        if (P->D.slab_bytes != ps[0]->D.slab_bytes) {
            ctx->err = "problems of a group differ in layout";
            return HPG_ERR_STATE;
        }
    }
    if (cudaMalloc(&Gp->delta_d, sizeof(long long) * np) != cudaSuccess ||
        cudaMalloc(&Gp->mask_d, sizeof(int) * np * kMaskCount) != cudaSuccess ||
        cudaMalloc(&Gp->par_d, sizeof(double) * np * kBatPar) != cudaSuccess ||
        cudaMalloc(&Gp->stat_d, sizeof(double) * np * (kStatD + kStatI)) != cudaSuccess ||
        cudaMallocHost(&Gp->h_delta, sizeof(long long) * np) != cudaSuccess ||
        cudaMallocHost(&Gp->h_stat, sizeof(double) * np * (kStatD + kStatI)) != cudaSuccess) {
        ctx->err = "group allocation failed";
        return HPG_ERR_OOM;
    }
    for (int i = 0; i < np; ++i) Gp->h_delta[i] = (long long)(ps[i]->D.slab - ps[0]->D.slab);
    Gp->h_mask.assign((size_t)np * kMaskCount, 0);
    Gp->h_par.assign((size_t)np * kBatPar, 0.0);
    CK(cudaMemcpy(Gp->delta_d, Gp->h_delta, sizeof(long long) * np, cudaMemcpyHostToDevice));
    out = Gp;
    return HPG_OK;
}

// The group of these problems: reused while every problem keeps the device state it
// had when the group was built (same allocation generation), else rebuilt.
static hpg_status group_for(hpg_ctx* home, hpg_ctx* ctx, std::vector<Problem*>& ps, std::shared_ptr<Group>& out) {
    std::vector<int> key;
    for (Problem* P : ps) key.push_back(P->id);
    std::lock_guard<std::mutex> lock(home->groups_mu);
    auto it = home->groups.find(key);
    if (it != home->groups.end()) {
        bool same = true;
        for (size_t i = 0; i < ps.size() && same; ++i)
            same = it->second->ps[i] == ps[i] && it->second->gens[i] == ps[i]->alloc_gen;
        if (same) {
            out = it->second;
            return HPG_OK;
        }
        home->groups.erase(it);
    }
    CKS(group_build(ctx, ps, out));
    home->groups[key] = out;
    return HPG_OK;
}

void drop_groups_with(hpg_ctx* ctx, int pid) {
    std::lock_guard<std::mutex> lock(ctx->groups_mu);
    for (auto it = ctx->groups.begin(); it != ctx->groups.end();) {
        if (std::find(it->first.begin(), it->first.end(), pid) != it->first.end()) it = ctx->groups.erase(it);
        else ++it;
    }
}

static hpg_status group_upload(hpg_ctx* ctx, Group& Gp, bool masks, bool par) {
    cudaStream_t s = ctx->stream;
    if (masks)
        CK(cudaMemcpyAsync(Gp.mask_d, Gp.h_mask.data(), sizeof(int) * Gp.np * kMaskCount, cudaMemcpyHostToDevice, s));
    if (par)
        CK(cudaMemcpyAsync(Gp.par_d, Gp.h_par.data(), sizeof(double) * Gp.np * kBatPar, cudaMemcpyHostToDevice, s));
    return HPG_OK;
}

// Read kStatD doubles at d and kStatI ints at iv of every problem (one copy, synchronises).
static hpg_status group_gather(hpg_ctx* ctx, Group& Gp, const double* d, const int* iv) {
    cudaStream_t s = ctx->stream;
    CK(launch_gather_status(d, kStatD, iv, kStatI, Gp.stat_d, s, Gp.bat(-1)));
    CK(cudaMemcpyAsync(Gp.h_stat, Gp.stat_d, sizeof(double) * Gp.np * (kStatD + kStatI), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return HPG_OK;
}
template <typename T>
struct GG;
template <>
struct GG<float> {
    static Geo<float>& g(Group& G) { return G.gf; }
    static bool& tuned(Group& G) { return G.tuned_f; }
};
template <>
struct GG<double> {
    static Geo<double>& g(Group& G) { return G.gd; }
    static bool& tuned(Group& G) { return G.tuned_d; }
};

// The FDM pass variant of a group: among the variants with the K split of the one
// the problems use alone (the same products summed in the same order, so the same
// bits), the fastest at the group's size; cached per (shape, precision, size).
template <typename T>
static hpg_status group_tune_fdm(hpg_ctx* ctx, Group& Gp) {
    Geo<T>& gg = GG<T>::g(Gp);
    DevState& D = Gp.ps[0]->D;
    gg = PV<T>::g(D);
    GG<T>::tuned(Gp) = true;
    const int forced = sizeof(T) == 4 ? Gp.ps[0]->params.fdm_tile_f32 : Gp.ps[0]->params.fdm_tile_f64;
    const int ks = fdm_tile_ks((int)sizeof(T), gg.gemm_cfg);
    if (ks < 0) {
        // a TMA variant: the group gets its own workspace and tensor maps over its np
        // problems; the pass matrices are problem 0's.  The variant stays the problems'
        // own (each TMA variant has its own summation order).
        if (!Gp.tma.ready) {
            std::string why;
            auto al = [&](size_t bytes) -> void* {
                void* p = nullptr;
                if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
                Gp.tma_allocs.push_back(p);
                return p;
            };
            const float* lamf[kMaxDim] = {D.lam_f[0], D.lam_f[1], D.lam_f[2]};
            if (!D.tma_ok || !fdm_tma_setup(Gp.tma, Gp.ps[0]->H, lamf, Gp.np, al, ctx->stream, &D.tma, &why)) {
                ctx->err = "lockstep group: TMA fast diagonalisation set-up failed (" + why + ")";
                return HPG_ERR_CUDA;
            }
        }
        gg.tma = &Gp.tma;
        return HPG_OK;
    }
    if (forced >= 0 || ks == 0 || Gp.np == 1) return HPG_OK;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, int>, int> cache;
    const auto key =
        std::make_tuple(gg.d, gg.n1[0], gg.n1[1], gg.d > 2 ? gg.n1[2] : 1, (int)sizeof(T), Gp.np, ks);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) { gg.gemm_cfg = it->second; return HPG_OK; }
    }
    cudaStream_t s = ctx->stream;
    const Bat all = Gp.bat(-1);
    T* x = PV<T>::tu(D);
    T* y = PV<T>::tu2(D);
    CK(launch_copy<T>(nullptr, x, gg.Nu0, s, all));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int base = gg.gemm_cfg;
    int best = base;
    float best_ms = 1e30f;
    for (int c = 0; c < fdm_tile_count((int)sizeof(T)); ++c) {
        if (fdm_tile_ks((int)sizeof(T), c) != ks) continue;
        gg.gemm_cfg = c;
        if (launch_fdm<T>(gg, nullptr, 1.0, x, y, PV<T>::w1(D), PV<T>::w2(D), s, nullptr, all) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch_fdm<T>(gg, nullptr, 1.0, x, y, PV<T>::w1(D), PV<T>::w2(D), s, nullptr, all);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); continue; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gg.gemm_cfg = best;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    return HPG_OK;
}

static double gd_(const Group& Gp, int i, int k) { return Gp.h_stat[i * kStatD + k]; }
static int gi_(const Group& Gp, int i, int k) { return (int)Gp.h_stat[Gp.np * kStatD + i * kStatI + k]; }

// `chunk` GMRES iterations of every problem of the group, enqueued without host
// synchronisation (problems whose GMRES has stopped skip every launch).
template <typename T, typename VT>
static hpg_status group_gmres_chunk(hpg_ctx* ctx, Group& Gp, int chunk) {
    Problem& P0 = *Gp.ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    GmresDev& G = D.gm;
    const Geo<T>& g = GG<T>::g(Gp);
    const IterCtl ctl{G.iflag, G.jdev, G.N};
    const Bat all = Gp.bat(-1);
    for (int c = 0; c < chunk; ++c) {
        CK(launch_precond<T, VT, T>(g, PV<T>::Sinv(D), gmres_basis<VT>(G), PV<T>::zp(D), s, ctl, all));
        CK(launch_bapply<T, T, T>(g, PV<T>::zp(D), PV<T>::tu(D), s, G.iflag, all));
        CK(launch_fdm<T>(g, D.alpha_dev, 0.0, PV<T>::tu(D), PV<T>::tu2(D), PV<T>::w1(D), PV<T>::w2(D), s, G.iflag,
                         all));
        CK(launch_schur_rest<T, VT>(g, PV<T>::gw(D), P0.params.beta, PV<T>::zp(D), PV<T>::tu2(D),
                                    gmres_basis<VT>(G), s, ctl, all));
        CK(gmres_arnoldi<VT>(G, s, all));
    }
    return HPG_OK;
}

template <typename T, typename VT>
static bool group_build_loop(hpg_ctx* ctx, Group& Gp, cudaGraphExec_t* exec, long long* kernels_per_body) {
    DevState& D = Gp.ps[0]->D;
    cudaStream_t s = ctx->stream;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGraphDestroy(g);
        return false;
    }
    const long long before = kernel_launch_count();
    hpg_status st = group_gmres_chunk<T, VT>(ctx, Gp, kGraphChunk);
    if (st == HPG_OK && launch_gm_setcond_batch(h, D.gm.iflag, s, Gp.bat(-1)) != cudaSuccess) st = HPG_ERR_CUDA;
    *kernels_per_body = kernel_launch_count() - before;
    add_kernel_launches(-*kernels_per_body);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &captured);
    bool ok = st == HPG_OK && ce == cudaSuccess && cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!ok) cudaGetLastError();
    return ok;
}

// GMRES of the problems in mask slot kMaskSolve (the others' stop flags are set from
// slot kMaskIdle) to their stop flags: one launch of the group's device-side loop.
// its[i], capped[i] per problem.
template <typename T, typename VT>
static hpg_status group_gmres_run(hpg_ctx* ctx, Group& Gp, std::vector<int>& its, std::vector<char>& capped) {
    DevState& D = Gp.ps[0]->D;
    cudaStream_t s = ctx->stream;
    GmresDev& G = D.gm;
    const int pi = sizeof(T) == sizeof(float) ? (sizeof(VT) == sizeof(float) ? 2 : 1) : 0;
    CK(launch_gm_stop(G.iflag, s, Gp.bat(kMaskIdle)));
    // host-driven iterations when graphs are off (profilers cannot trace conditional nodes)
    if (Gp.ps[0]->params.graphs == 0) Gp.loop_failed[pi] = true;
    if (!Gp.loop[pi] && !Gp.loop_failed[pi]) {
        long long nk = 0;
        if (!group_build_loop<T, VT>(ctx, Gp, &Gp.loop[pi], &nk)) {
            Gp.loop[pi] = nullptr;
            Gp.loop_failed[pi] = true;
        } else {
            Gp.loop_kernels[pi] = nk;
        }
    }
    if (Gp.loop[pi]) {
        CK(cudaGraphLaunch(Gp.loop[pi], s));
        CKS(group_gather(ctx, Gp, G.scal, G.iflag));
        int maxits = 0;
        for (int i = 0; i < Gp.np; ++i) maxits = std::max(maxits, gi_(Gp, i, 1));
        add_kernel_launches(Gp.loop_kernels[pi] * ((maxits + kGraphChunk - 1) / kGraphChunk + 1));
    } else {
        for (int guard = 0; guard <= G.kmax; ++guard) {
            CKS(group_gmres_chunk<T, VT>(ctx, Gp, 1));
            CKS(group_gather(ctx, Gp, G.scal, G.iflag));
            bool all = true;
            for (int i = 0; i < Gp.np && all; ++i) all = gi_(Gp, i, 0) != 0;
            if (all) break;
        }
    }
    for (int i = 0; i < Gp.np; ++i) {
        its[i] = gi_(Gp, i, 1);
        // the cap flag is also set when the last allowed iteration converged: check the residual
        capped[i] = gi_(Gp, i, 3) != 0 && gi_(Gp, i, 0) != 0 && gi_(Gp, i, 2) == 0 && gd_(Gp, i, 1) > gd_(Gp, i, 2);
    }
    return HPG_OK;
}

// eq. (schur2) for the problems of mask slot kMaskSolve: y = b_psi - B^T A^{-1} b_u,
// GMRES on S, delta_u = A^{-1}(b_u - B delta_psi); b = D.r, result in D.dcorr,
// relative tolerance per problem in Bat::par (kParRtol).
template <typename T, typename VT>
static hpg_status group_schur_solve(hpg_ctx* ctx, Group& Gp, std::vector<int>& its, std::vector<char>& capped) {
    Problem& P0 = *Gp.ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    const Geo<T>& g = GG<T>::g(Gp);
    const long long Nu0 = (long long)P0.H.Nu0, Npsi = (long long)P0.H.Npsi;
    GmresDev& G = D.gm;
    const Bat b = Gp.bat(kMaskSolve);
    T* tu = PV<T>::tu(D);
    T* tu2 = PV<T>::tu2(D);
    T* zp = PV<T>::zp(D);
    const double* bu = D.r;
    const double* bp = D.r + Nu0;
    double* du = D.dcorr;
    double* dp = D.dcorr + Nu0;
    if constexpr (sizeof(T) == sizeof(double)) CK(launch_copy<double>(bu, tu, Nu0, s, b));
    else CK(launch_convert<double, float>(bu, tu, Nu0, s, b));
    CK(launch_fdm<T>(g, D.alpha_dev, 0.0, tu, tu2, PV<T>::w1(D), PV<T>::w2(D), s, nullptr, b));
    CK(launch_btapply<T, T, T>(g, tu2, zp, s, b));
    CK(launch_sub_scaled<T>(bp, 1.0, zp, D.yp, Npsi, s, b));
    CK(gmres_start<VT>(G, D.yp, 0.0, s, 0, b));
    CKS(group_gmres_run<T, VT>(ctx, Gp, its, capped));
    CK(gmres_finish<VT>(G, D.xs, s, b));
    CK(launch_precond<T, double, double>(g, PV<T>::Sinv(D), D.xs, dp, s, IterCtl{}, b));
    CK(launch_bapply<T, double, T>(g, dp, tu, s, nullptr, b));
    CK(launch_sub_scaled<T>(bu, 1.0, tu, D.tu_d, Nu0, s, b));
    if constexpr (sizeof(T) == sizeof(float)) CK(launch_convert<double, float>(D.tu_d, tu, Nu0, s, b));
    CK(launch_fdm<T>(g, D.alpha_dev, 0.0, tu, tu2, PV<T>::w1(D), PV<T>::w2(D), s, nullptr, b));
    if constexpr (sizeof(T) == sizeof(double)) CK(launch_copy<double>(tu2, du, Nu0, s, b));
    else CK(launch_convert<float, double>(tu2, du, Nu0, s, b));
    return HPG_OK;
}

template <typename T>
static hpg_status group_schur_solve_T(hpg_ctx* ctx, Group& Gp, std::vector<int>& its, std::vector<char>& capped) {
    if constexpr (sizeof(T) == sizeof(float))
        if (Gp.ps[0]->params.krylov_f32) return group_schur_solve<T, float>(ctx, Gp, its, capped);
    return group_schur_solve<T, double>(ctx, Gp, its, capped);
}

// Newton systems of the problems in mask slot kMaskNewton: the refinement loop of
// linear_solve, problem by problem in its decisions, batched in its launches.
static hpg_status group_linear_solve(hpg_ctx* ctx, Group& Gp, const std::vector<char>& inN,
                                     const std::vector<double>& normF, const std::vector<double>& eta) {
    Problem& P0 = *Gp.ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    const int np = Gp.np;
    const long long Nu0 = (long long)P0.H.Nu0, Npsi = (long long)P0.H.Npsi, Nx = Nu0 + Npsi;
    const bool f64 = P0.params.precision == HPG_FP64;
    const Bat bN = Gp.bat(kMaskNewton);
    CK(launch_copy<double>(nullptr, D.delta, Nx, s, bN));
    CK(launch_copy<double>(D.F, D.r, Nx, s, bN));
    std::vector<double> rnorm(normF);
    std::vector<char> on(inN);
    std::vector<int> its(np, 0);
    std::vector<char> capped(np, 0);
    for (int sw = 0; sw < std::max(1, P0.params.refine_max); ++sw) {
        bool any = false;
        for (int i = 0; i < np; ++i) {
            Gp.mask(kMaskSolve)[i] = on[i];
            Gp.mask(kMaskIdle)[i] = !on[i];
            any = any || on[i];
            if (!on[i]) continue;
            const double need = eta[i] * normF[i] / std::max(rnorm[i], 1e-300);
            Gp.h_par[i * kBatPar + kParRtol] =
                f64 ? std::min(1.0, need) : std::min(1.0, std::max(kInnerMargin * need, 1e-6));
        }
        if (!any) break;
        CKS(group_upload(ctx, Gp, true, true));
        if (f64) CKS(group_schur_solve_T<double>(ctx, Gp, its, capped));
        else CKS(group_schur_solve_T<float>(ctx, Gp, its, capped));
        bool more = false;
        for (int i = 0; i < np; ++i) {
            if (!on[i]) continue;
            hpg_stats& st = Gp.ps[i]->stats;
            st.krylov_total += its[i];
            st.refine_total += 1;
            st.ainv_total += 2 + its[i];
            if (capped[i]) st.krylov_cap_hits++;
        }
        CK(launch_axpby(1.0, D.dcorr, 1.0, D.delta, Nx, s, Gp.bat(kMaskSolve)));
        for (int i = 0; i < np; ++i) {
            if (on[i] && f64 && !capped[i]) on[i] = 0;     // the FP64 GMRES residual is the true one
            Gp.mask(kMaskPrev)[i] = on[i];
            more = more || on[i];
        }
        if (!more) break;
        CKS(group_upload(ctx, Gp, true, false));
        const Bat bR = Gp.bat(kMaskPrev);
        CK(launch_newton_apply(D.gd, D.gw, 0.0, P0.params.beta, D.delta, D.r, s, bR));
        CK(launch_axpby(1.0, D.F, -1.0, D.r, Nx, s, bR));
        int nparts = 0;
        CK(launch_sumsq(D.r, Nx, D.part, &nparts, s, bR));
        CK(launch_reduce_sum(D.part, nparts, D.scal + 1, s, bR));
        CKS(group_gather(ctx, Gp, D.scal, D.flag));
        for (int i = 0; i < np; ++i) {
            if (!on[i]) continue;
            rnorm[i] = std::sqrt(gd_(Gp, i, 1));
            if (rnorm[i] <= eta[i] * normF[i]) on[i] = 0;
        }
    }
    return HPG_OK;
}

// Evaluation + residual + norm of the state at `x` (the current or the trial state)
// for the problems of mask slot `slot`; alpha from Bat::par.  Synchronises; the
// squared norms and flags are in the group's gathered status.
static hpg_status group_residual(hpg_ctx* ctx, Group& Gp, int slot, bool trial) {
    Problem& P0 = *Gp.ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    const long long Nu0 = (long long)P0.H.Nu0;
    const Bat b = Gp.bat(slot);
    const double* x = trial ? D.xt : D.x;
    double* gw = trial ? D.gwt : D.gw;
    double* eg = trial ? D.egt : D.eg;
    double* F = trial ? D.Ft : D.F;
    CK(launch_eval(D.gd, x + Nu0, D.phiq, gw, nullptr, eg, D.flag, s, b));
    CK(launch_residual(D.gd, x, x + Nu0, D.psi_prev, eg, D.rA, D.rB, D.bf, D.phiz, 0.0, F, D.part, s, b));
    CK(launch_reduce_sum(D.part, n_res_partials(D.gd), D.scal, s, b));
    return group_gather(ctx, Gp, D.scal, D.flag);
}

// The proximal loop of solve_problem for every problem of the group at once, on
// ctx's stream; `home` owns the cache of groups (the caller's context).
hpg_status solve_group(hpg_ctx* home, hpg_ctx* ctx, std::vector<Problem*>& ps, std::vector<std::string>* errs) {
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = kernel_launch_count();
    const int np = (int)ps.size();
    for (Problem* P : ps) {
        CKS(alloc_device(ctx, *P));
        // every problem of a group keeps its current state in the first buffer of each pair
        if (P->D.x > P->D.xt) swap_state(P->D);
    }
    std::shared_ptr<Group> gref;
    CKS(group_for(home, ctx, ps, gref));
    Group& Gp = *gref;
    Problem& P0 = *ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    const long long Nu0 = (long long)P0.H.Nu0, Npsi = (long long)P0.H.Npsi, Nx = Nu0 + Npsi;
    const long long gsz = (long long)(P0.H.Nq * gauss_stride(P0.H.kind, P0.H.d));
    for (Problem* P : ps) {
        P->stats = hpg_stats{};
        P->stats.n_u = Nu0;
        P->stats.n_psi = Npsi;
        P->timer.on = false;
    }
    const Bat all = Gp.bat(-1);
    if (P0.params.precision == HPG_FP64 && !Gp.tuned_d) CKS(group_tune_fdm<double>(ctx, Gp));
    if (P0.params.precision != HPG_FP64 && !Gp.tuned_f) CKS(group_tune_fdm<float>(ctx, Gp));
    CK(launch_copy<double>(nullptr, D.x, Nx, s, all));
    CK(launch_copy<double>(nullptr, D.psi_prev, Npsi, s, all));
    CK(launch_copy<int>(nullptr, D.flag, 4, s, all));
    // per-problem host state
    std::vector<int> k(np, 0), it(np, 0), flag(np, 0), status(np, HPG_OK);
    std::vector<char> done(np, 0), start(np, 1), redo(np, 0);
    std::vector<double> normF(np, 0.0), eta(np, 0.0), lam(np, 1.0), nFt(np, 0.0);
    const bool mixed = P0.params.precision != HPG_FP64;
    std::vector<int> tflag(np, 0), nsteps(np);
    std::vector<std::string> msg(np);
    for (int i = 0; i < np; ++i) nsteps[i] = (int)std::min<size_t>(ps[i]->H.alphas.size(), HPG_MAX_ALPHA);
    auto finish_step = [&](int i) {
        hpg_stats& st = ps[i]->stats;
        st.newton_per_step[k[i]] = it[i];
        st.newton_total += it[i];
        st.alpha_steps = k[i] + 1;
    };
    while (true) {
        // ---- subproblem starts: alpha_k, psi_{k-1} <- psi, residual at the warm start
        bool anyS = false, anyPrev = false;
        for (int i = 0; i < np; ++i) {
            const bool st_ = !done[i] && start[i];
            Gp.mask(kMaskStart)[i] = st_;
            Gp.mask(kMaskPrev)[i] = st_ && k[i] > 0;
            anyS = anyS || st_;
            anyPrev = anyPrev || (st_ && k[i] > 0);
            if (st_) Gp.h_par[i * kBatPar + kParAlpha] = ps[i]->H.alphas[k[i]];
        }
        if (anyS) {
            CKS(group_upload(ctx, Gp, true, true));
            CK(launch_scatter_par(D.alpha_dev, kParAlpha, s, Gp.bat(kMaskStart)));
            if (anyPrev) CK(launch_copy<double>(D.x + Nu0, D.psi_prev, Npsi, s, Gp.bat(kMaskPrev)));
            CKS(group_residual(ctx, Gp, kMaskStart, false));
            for (int i = 0; i < np; ++i) {
                if (!Gp.mask(kMaskStart)[i]) continue;
                normF[i] = std::sqrt(gd_(Gp, i, 0));
                flag[i] = gi_(Gp, i, 0);
                if (!std::isfinite(normF[i])) flag[i] |= 1;
                start[i] = 0;
            }
        }
        // ---- per-problem decisions
        bool anyN = false, live = false;
        for (int i = 0; i < np; ++i) {
            Gp.mask(kMaskNewton)[i] = 0;
            if (done[i] || start[i]) {
                live = live || !done[i];
                continue;
            }
            const hpg_params& q = ps[i]->params;
            if (flag[i] & 1) {
                status[i] = HPG_ERR_NONFINITE;
            } else if (!std::isfinite(normF[i])) {
                status[i] = HPG_ERR_NONFINITE;
                msg[i] = "non-finite Newton residual in proximal step " + std::to_string(k[i] + 1);
            } else if (normF[i] <= q.newton_tol) {
                finish_step(i);
                ++k[i];
                it[i] = 0;
                if (k[i] >= nsteps[i]) done[i] = 1;
                else start[i] = 1;
                live = live || !done[i];
                continue;
            } else if (it[i] >= q.newton_max && mixed) {
                redo[i] = 1;                // FP64 again on its own, as alone (below)
                done[i] = 1;
                continue;
            } else if (it[i] >= q.newton_max) {
                status[i] = HPG_ERR_NEWTON_CAP;
                msg[i] = "Newton cap reached in proximal step " + std::to_string(k[i] + 1) + " (||F|| = " +
                         std::to_string(normF[i]) + ")";
            } else {
                Gp.mask(kMaskNewton)[i] = 1;
                eta[i] = std::min(q.krylov_rtol, std::max(normF[i], 1e-12));
                anyN = true;
                live = true;
                continue;
            }
            finish_step(i);
            done[i] = 1;
        }
        if (!live) break;
        if (!anyN) continue;
        // ---- one Newton step of every problem in the Newton mask
        CKS(group_upload(ctx, Gp, true, false));
        const Bat bN = Gp.bat(kMaskNewton);
        CK(launch_copy<double>(D.gw, D.gwl, gsz, s, bN));
        if (P0.params.precision == HPG_FP64) {
            CK(launch_factor<double>(D.gd, D.gwl, 1.0, P0.params.beta, D.Sinv_d, nullptr, D.flag, D.fwork_d, s, bN));
        } else {
            CK(launch_convert<double, float>(D.gwl, D.gwf, gsz, s, bN));
            CK(launch_factor<float>(D.gf, D.gwf, 1.0, P0.params.beta, D.Sinv_f, nullptr, D.flag, D.fwork_f, s, bN));
        }
        std::vector<char> inN(np);
        for (int i = 0; i < np; ++i) inN[i] = (char)Gp.mask(kMaskNewton)[i];
        CKS(group_linear_solve(ctx, Gp, inN, normF, eta));
        // backtracking on ||F||, each problem with its own step length
        std::vector<char> ls(inN);
        for (int i = 0; i < np; ++i) lam[i] = 1.0;
        for (int h = 0; h <= P0.params.ls_max; ++h) {
            bool any = false;
            for (int i = 0; i < np; ++i) {
                Gp.mask(kMaskTrial)[i] = ls[i];
                any = any || ls[i];
                if (ls[i]) Gp.h_par[i * kBatPar + kParLam] = lam[i];
            }
            if (!any) break;
            CKS(group_upload(ctx, Gp, true, true));
            const Bat bL = Gp.bat(kMaskTrial);
            CK(launch_trial(D.x, D.delta, 1.0, D.xt, Nx, s, bL));
            CK(launch_copy<int>(nullptr, D.flag, 1, s, bL));
            CKS(group_residual(ctx, Gp, kMaskTrial, true));
            for (int i = 0; i < np; ++i) {
                if (!ls[i]) continue;
                nFt[i] = std::sqrt(gd_(Gp, i, 0));
                tflag[i] = gi_(Gp, i, 0);
                if (!std::isfinite(nFt[i])) tflag[i] |= 1;
                if (!(tflag[i] & 1) && nFt[i] <= (1.0 - 1e-4 * lam[i]) * normF[i]) {
                    ls[i] = 0;
                } else if (h == ps[i]->params.ls_max) {
                    ps[i]->stats.ls_fail++;
                    ls[i] = 0;
                } else {
                    lam[i] *= 0.5;
                }
            }
        }
        // factorisation flag (non-SPD block): bit 1 of flag[1]
        CKS(group_gather(ctx, Gp, D.scal, D.flag));
        bool anyAcc = false;
        for (int i = 0; i < np; ++i) {
            Gp.mask(kMaskTrial)[i] = 0;
            if (!inN[i]) continue;
            const bool spd_fail = (gi_(Gp, i, 1) & 2) != 0;
            const bool bad_trial = (tflag[i] & 1) || !std::isfinite(nFt[i]);
            if (mixed && (spd_fail || bad_trial)) {
                // a failed mixed step: a problem solved alone takes its proximal step again
                // in FP64, which the group does not run; the member is solved again on its
                // own afterwards (the same steps as alone)
                redo[i] = 1;
                done[i] = 1;
                continue;
            }
            if (spd_fail) {
                status[i] = HPG_ERR_NOT_SPD;
                msg[i] = "non-positive pivot in an FP64 S-hat block factorisation in proximal step " +
                         std::to_string(k[i] + 1);
                finish_step(i);
                done[i] = 1;
                continue;
            }
            Gp.mask(kMaskTrial)[i] = 1;
            anyAcc = true;
            normF[i] = nFt[i];
            flag[i] = tflag[i];
            ++it[i];
        }
        if (anyAcc) {
            // accept: the trial state becomes the current one
            CKS(group_upload(ctx, Gp, true, false));
            const Bat bA = Gp.bat(kMaskTrial);
            CK(launch_copy<double>(D.xt, D.x, Nx, s, bA));
            CK(launch_copy<double>(D.gwt, D.gw, gsz, s, bA));
            CK(launch_copy<double>(D.egt, D.eg, Npsi, s, bA));
            CK(launch_copy<double>(D.Ft, D.F, Nx, s, bA));
        }
    }
    CK(cudaStreamSynchronize(s));
    const long long launches = kernel_launch_count() - launches0;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    // members that fell back from the mixed form: solved again on their own (same steps as alone)
    for (int i = 0; i < np; ++i) {
        if (!redo[i]) continue;
        status[i] = solve_problem(ctx, *ps[i]);
        if (status[i] != HPG_OK) msg[i] = ctx->err;
    }
    hpg_status first = HPG_OK;
    for (int i = 0; i < np; ++i) {
        if (redo[i]) {
            if (errs) (*errs)[i] = msg[i];
            if (status[i] != HPG_OK && first == HPG_OK) {
                first = (hpg_status)status[i];
                ctx->err = msg[i];
            }
            continue;
        }
        hpg_stats& st = ps[i]->stats;
        st.final_residual = normF[i];
        st.status = status[i];
        st.kernel_launches = launches / np + (i < launches % np ? 1 : 0);   // the group's launches, shared out
        // the FDM pass variant the group ran (same summation order as the problem's own)
        st.fdm_tile_f32 = Gp.tuned_f ? Gp.gf.gemm_cfg : ps[i]->D.gf.gemm_cfg;
        st.fdm_tile_f64 = Gp.tuned_d ? Gp.gd.gemm_cfg : ps[i]->D.gd.gemm_cfg;
        st.h2d_bytes = ps[i]->h2d_bytes;
        st.solve_ms = ms;
        ps[i]->solved = true;
        if (errs) (*errs)[i] = msg[i];
        if (status[i] != HPG_OK && first == HPG_OK) {
            first = (hpg_status)status[i];
            ctx->err = msg[i].empty() ? std::string(hpg_status_str(first)) : msg[i];
        }
    }
    return first;
}

// Several independent solves in flight at once: up to ctx->concurrency host
// workers, each driving its own CUDA stream (forked from and joined back to the
// context's stream), pull problems from a shared queue.  Kernels of different
// problems overlap on the device; each problem's arithmetic and reduction
// order is exactly that of hpg_solve, so results do not depend on the mix.
hpg_status solve_batch(hpg_ctx* ctx, std::vector<Problem*>& probs) {
    const int n = (int)probs.size();
    // units of work: lockstep groups of same-shape problems (at most kGroupMax each), and
    // single problems that cannot share launches
    constexpr int kGroupMax = 64;
    std::vector<std::vector<int>> units;
    {
        std::map<std::string, std::vector<int>> by_key;
        std::vector<std::string> order;
        for (int i = 0; i < n; ++i) {
            if (!groupable(*probs[i])) { units.push_back({i}); continue; }
            const std::string key = group_key(*probs[i]);
            auto& v = by_key[key];
            if (v.empty()) order.push_back(key);
            v.push_back(i);
        }
        for (const auto& key : order) {
            const auto& v = by_key[key];
            for (size_t a = 0; a < v.size(); a += kGroupMax)
                units.emplace_back(v.begin() + a, v.begin() + std::min(v.size(), a + kGroupMax));
        }
    }
    const int nu = (int)units.size();
    const int W = std::max(1, std::min(ctx->concurrency, nu));
    while ((int)ctx->side_streams.size() < W) {
        cudaStream_t st;
        cudaEvent_t ev;
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ctx->side_streams.push_back(st);
        ctx->side_events.push_back(ev);
    }
    CK(cudaEventRecord(ctx->side_events[0], ctx->stream));
    for (int w = 0; w < W; ++w) CK(cudaStreamWaitEvent(ctx->side_streams[w], ctx->side_events[0], 0));
    std::vector<hpg_status> status(n, HPG_OK);
    std::vector<std::string> errs(n);
    std::atomic<int> next{0};
    auto worker = [&](int w) {
        cudaSetDevice(ctx->device);
        hpg_ctx local;
        local.device = ctx->device;
        local.stream = ctx->side_streams[w];
        for (int u = next.fetch_add(1); u < nu; u = next.fetch_add(1)) {
            const std::vector<int>& idx = units[u];
            if (idx.size() == 1) {
                status[idx[0]] = solve_problem(&local, *probs[idx[0]]);
                if (status[idx[0]] != HPG_OK) errs[idx[0]] = local.err;
                continue;
            }
            std::vector<Problem*> ps;
            for (int i : idx) ps.push_back(probs[i]);
            std::vector<std::string> e(ps.size());
            // the group cache belongs to the caller's context
            const hpg_status gs = solve_group(ctx, &local, ps, &e);
            // a failure of the solver itself is per problem (in its stats); any other stops the group
            const bool per_problem = gs == HPG_OK || gs == HPG_ERR_NEWTON_CAP || gs == HPG_ERR_KRYLOV_CAP ||
                                     gs == HPG_ERR_NONFINITE || gs == HPG_ERR_NOT_SPD;
            for (size_t j = 0; j < idx.size(); ++j) {
                status[idx[j]] = per_problem ? (hpg_status)ps[j]->stats.status : gs;
                if (!per_problem) errs[idx[j]] = local.err;
                else if (status[idx[j]] != HPG_OK) errs[idx[j]] = e[j].empty() ? hpg_status_str(status[idx[j]]) : e[j];
            }
        }
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < W; ++w) threads.emplace_back(worker, w);
    worker(0);
    for (auto& t : threads) t.join();
    for (int w = 0; w < W; ++w) {
        CK(cudaEventRecord(ctx->side_events[w], ctx->side_streams[w]));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->side_events[w], 0));
    }
    for (int i = 0; i < n; ++i)
        if (status[i] != HPG_OK) {
            ctx->err = errs[i];
            return status[i];
        }
    return HPG_OK;
}

// ------------------------------------------------------------ operators (tests)
hpg_status op_set_state(hpg_ctx* ctx, Problem& P, const double* u_full, const double* psi, const double* psi_prev,
                        double alpha) {
    CKS(alloc_device(ctx, P));
    HostProblem& H = P.H;
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    std::vector<double> u0(H.Nu0);
    for (size_t I = 0; I < H.Nu0; ++I) {
        size_t ii = I, full = 0, stride = 1;
        for (int j = 0; j < H.d; ++j) {
            full += (size_t)H.dir[j].glob_of_int((int)(ii % H.dir[j].n1)) * stride;
            ii /= H.dir[j].n1;
            stride *= H.dir[j].N1;
        }
        u0[I] = u_full[full];
    }
    CK(cudaMemcpyAsync(D.x, u0.data(), H.Nu0 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.x + H.Nu0, psi, H.Npsi * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.psi_prev, psi_prev, H.Npsi * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(D.flag, 0, 4 * sizeof(int), s));
    CKS(eval_state(ctx, P, D.x, D.gw, D.eg));
    CK(cudaStreamSynchronize(s));
    P.state_alpha = alpha;
    CKS(set_alpha(ctx, P, alpha));
    return HPG_OK;
}

hpg_status op_residual(hpg_ctx* ctx, Problem& P, double* F, double* norm) {
    DevState& D = P.D;
    int flag = 0;
    double nrm = 0.0;
    CKS(residual_state(ctx, P, D.x, D.eg, P.state_alpha, D.F, &nrm, &flag));
    CK(cudaMemcpy(F, D.F, (P.H.Nu0 + P.H.Npsi) * sizeof(double), cudaMemcpyDeviceToHost));
    if (norm) *norm = nrm;
    return (flag & 1) ? HPG_ERR_NONFINITE : HPG_OK;
}

hpg_status op_apply_newton(hpg_ctx* ctx, Problem& P, const double* x, double* y) {
    DevState& D = P.D;
    const size_t Nx = P.H.Nu0 + P.H.Npsi;
    CK(cudaMemcpy(D.r, x, Nx * sizeof(double), cudaMemcpyHostToDevice));
    CK(launch_newton_apply(D.gd, D.gw, P.state_alpha, P.params.beta, D.r, D.dcorr, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(y, D.dcorr, Nx * sizeof(double), cudaMemcpyDeviceToHost));
    return HPG_OK;
}

hpg_status op_stiffness_inv(hpg_ctx* ctx, Problem& P, int precision, const double* x, double* y) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long n = (long long)P.H.Nu0;
    CK(cudaMemcpy(D.r, x, n * sizeof(double), cudaMemcpyHostToDevice));
    if (precision == HPG_FP64) {
        CKS(fdm_T<double>(ctx, P, P.state_alpha, D.r, D.tu2_d));
        CK(cudaStreamSynchronize(s));
        CK(cudaMemcpy(y, D.tu2_d, n * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        CK(launch_convert<double, float>(D.r, D.tu_f, n, s));
        CKS(fdm_T<float>(ctx, P, P.state_alpha, D.tu_f, D.tu2_f));
        CK(launch_convert<float, double>(D.tu2_f, D.dcorr, n, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaMemcpy(y, D.dcorr, n * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return HPG_OK;
}

hpg_status op_factor(hpg_ctx* ctx, Problem& P, int precision, double* blocks) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    double* dump = nullptr;
    const size_t nblk = (size_t)P.H.Nc * P.H.nb * P.H.nb;
    if (blocks) {
        if (cudaMalloc(&dump, nblk * sizeof(double)) != cudaSuccess) return HPG_ERR_OOM;
    }
    hpg_status st = (precision == HPG_FP64) ? factor_T<double>(ctx, P, P.state_alpha, dump)
                                            : factor_T<float>(ctx, P, P.state_alpha, dump);
    cudaStreamSynchronize(s);
    if (st == HPG_OK && blocks) {
        if (cudaMemcpy(blocks, dump, nblk * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) st = HPG_ERR_CUDA;
    }
    if (dump) cudaFree(dump);
    int flag = 0;
    cudaMemcpy(&flag, D.flag + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (st == HPG_OK && (flag & 2)) st = HPG_ERR_NOT_SPD;
    return st;
}

hpg_status op_precond_inv(hpg_ctx* ctx, Problem& P, int precision, const double* x, double* y) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long n = (long long)P.H.Npsi;
    CK(cudaMemcpy(D.yp, x, n * sizeof(double), cudaMemcpyHostToDevice));
    if (precision == HPG_FP64) CK(launch_precond<double, double, double>(D.gd, D.Sinv_d, D.yp, D.xs, s));
    else CK(launch_precond<float, double, double>(D.gf, D.Sinv_f, D.yp, D.xs, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(y, D.xs, n * sizeof(double), cudaMemcpyDeviceToHost));
    return HPG_OK;
}

hpg_status op_schur(hpg_ctx* ctx, Problem& P, int precision, const double* x, double* y) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long n = (long long)P.H.Npsi;
    const long long gsz = (long long)(P.H.Nq * gauss_stride(P.H.kind, P.H.d));
    CK(cudaMemcpyAsync(D.gwl, D.gw, gsz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpy(D.yp, x, n * sizeof(double), cudaMemcpyHostToDevice));
    if (precision == HPG_FP64) {
        CK(cudaMemcpyAsync(D.zp_d, D.yp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CKS(schur_apply_T<double>(ctx, P, P.state_alpha, D.zp_d, D.xs));
    } else {
        CK(launch_convert<double, float>(D.gwl, D.gwf, gsz, s));
        CK(launch_convert<double, float>(D.yp, D.zp_f, n, s));
        CKS(schur_apply_T<float>(ctx, P, P.state_alpha, D.zp_f, D.xs));
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(y, D.xs, n * sizeof(double), cudaMemcpyDeviceToHost));
    return HPG_OK;
}

hpg_status op_newton_direction(hpg_ctx* ctx, Problem& P, int precision, double rtol, double* delta, int* its) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    double nrm = 0.0;
    int flag = 0;
    CKS(residual_state(ctx, P, D.x, D.eg, P.state_alpha, D.F, &nrm, &flag));
    const double save = P.params.krylov_rtol;
    const int saveprec = P.params.precision;
    P.params.krylov_rtol = rtol;
    P.params.precision = precision;
    hpg_status st = (precision == HPG_FP64) ? factor_T<double>(ctx, P, P.state_alpha, nullptr)
                                            : factor_T<float>(ctx, P, P.state_alpha, nullptr);
    int sweeps = 0, it = 0;
    if (st == HPG_OK) st = linear_solve(ctx, P, P.state_alpha, D.F, nrm, rtol, D.delta, &it, &sweeps);
    P.params.krylov_rtol = save;
    P.params.precision = saveprec;
    if (st != HPG_OK) return st;
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(delta, D.delta, (P.H.Nu0 + P.H.Npsi) * sizeof(double), cudaMemcpyDeviceToHost));
    if (its) *its = it;
    return HPG_OK;
}

// Enqueue `reps` applications of one kernel class on the current state, with
// no host synchronisation (for timing with events on the context's stream).
// The launches are captured once per (class, precision, reps) into a CUDA
// graph and replayed, so that host launch overhead does not enter the timing.
static hpg_status enqueue_kernel(hpg_ctx* ctx, Problem& P, int cls, bool f32, double alpha) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const bool fb = f32 && P.params.krylov_f32 != 0;     // float GMRES basis
    switch (cls) {
        case HPG_K_FDM:
            if (f32) CK(launch_fdm<float>(D.gf, nullptr, alpha, D.tu_f, D.tu2_f, D.w1_f, D.w2_f, s));
            else CK(launch_fdm<double>(D.gd, nullptr, alpha, D.tu_d, D.tu2_d, D.w1_d, D.w2_d, s));
            break;
        case HPG_K_PRECOND:
            if (fb) CK(launch_precond<float, float, float>(D.gf, D.Sinv_f, gmres_basis<float>(D.gm), D.zp_f, s));
            else if (f32) CK(launch_precond<float, double, float>(D.gf, D.Sinv_f, D.yp, D.zp_f, s));
            else CK(launch_precond<double, double, double>(D.gd, D.Sinv_d, D.yp, D.zp_d, s));
            break;
        case HPG_K_BAPPLY:
            if (f32) CK(launch_bapply<float, float, float>(D.gf, D.zp_f, D.tu_f, s));
            else CK(launch_bapply<double, double, double>(D.gd, D.zp_d, D.tu_d, s));
            break;
        case HPG_K_SCHUR:
            if (fb)
                CK(launch_schur_rest<float, float>(D.gf, D.gwf, P.params.beta, D.zp_f, D.tu2_f,
                                                   gmres_basis<float>(D.gm) + D.gm.N, s));
            else if (f32) CK(launch_schur_rest<float, double>(D.gf, D.gwf, P.params.beta, D.zp_f, D.tu2_f, D.xs, s));
            else CK(launch_schur_rest<double, double>(D.gd, D.gwl, P.params.beta, D.zp_d, D.tu2_d, D.xs, s));
            break;
        case HPG_K_NEWTON_APPLY:
            CK(launch_newton_apply(D.gd, D.gw, alpha, P.params.beta, D.x, D.r, s));
            break;
        case HPG_K_FACTOR:
            if (f32) CK(launch_factor<float>(D.gf, D.gwf, alpha, P.params.beta, D.Sinv_f, nullptr, D.flag, D.fwork_f, s));
            else CK(launch_factor<double>(D.gd, D.gwl, alpha, P.params.beta, D.Sinv_d, nullptr, D.flag, D.fwork_d, s));
            break;
        case HPG_K_EVAL:
            CK(launch_eval(D.gd, D.x + P.H.Nu0, D.phiq, D.gwt, nullptr, D.egt, D.flag, s));
            break;
        case HPG_K_ORTHO:
            // one CGS2 Arnoldi step at j = kmax / 2, the mean j of a full Krylov cycle
            // (float basis for FP32 inner solves with krylov_f32)
            if (fb) CK(gmres_timed_step<float>(D.gm, D.gm.kmax / 2, s));
            else CK(gmres_timed_step<double>(D.gm, D.gm.kmax / 2, s));
            break;
        default:
            return HPG_ERR_ARG;
    }
    return HPG_OK;
}

hpg_status op_launch_kernel(hpg_ctx* ctx, Problem& P, int cls, int precision, int reps) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long gsz = (long long)(P.H.Nq * gauss_stride(P.H.kind, P.H.d));
    const bool f32 = precision == HPG_MIXED;
    const double alpha = P.state_alpha > 0.0 ? P.state_alpha : (P.H.alphas.empty() ? 1.0 : P.H.alphas.back());
    const long long key = ((long long)cls * 4 + (f32 ? 1 : 0) + (f32 && P.params.krylov_f32 ? 2 : 0)) * 1000003LL + reps;
    auto it = D.bench_graphs.find(key);
    if (it == D.bench_graphs.end()) {
        // operands of this linearisation: the weights of the current state
        CK(cudaMemcpyAsync(D.gwl, D.gw, gsz * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(launch_convert<double, float>(D.gwl, D.gwf, gsz, s));
        // FP32 Krylov-loop kernels with a float basis read it: V_0 = yp
        if (f32 && P.params.krylov_f32) CK(launch_convert<double, float>(D.yp, gmres_basis<float>(D.gm), D.gm.N, s));
        CK(cudaStreamSynchronize(s));
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        hpg_status st = HPG_OK;
        const long long before = kernel_launch_count();
        for (int r = 0; r < reps && st == HPG_OK; ++r) st = enqueue_kernel(ctx, P, cls, f32, alpha);
        const long long nk = kernel_launch_count() - before;
        add_kernel_launches(-nk);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != HPG_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        CK(ce);
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        it = D.bench_graphs.emplace(key, std::make_pair(ex, nk)).first;
    }
    // the timed Arnoldi step always takes both Gram-Schmidt passes
    if (cls == HPG_K_ORTHO) CK(cudaMemsetAsync(D.gm.force, 1, sizeof(int), s));
    CK(cudaGraphLaunch(it->second.first, s));
    if (cls == HPG_K_ORTHO) CK(cudaMemsetAsync(D.gm.force, 0, sizeof(int), s));
    add_kernel_launches(it->second.second);
    return HPG_OK;
}


// ---- kernel-class replays over a whole group (timing in the batched configuration)
template <typename T>
static hpg_status group_enqueue(hpg_ctx* ctx, Group& Gp, int cls, double alpha) {
    Problem& P0 = *Gp.ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    Bat all = Gp.bat(-1);
    all.par = nullptr;                     // scalar arguments, as in the single-problem replays
    const Geo<T>& g = GG<T>::g(Gp);
    constexpr bool f32 = sizeof(T) == sizeof(float);
    switch (cls) {
        case HPG_K_FDM:
            CK(launch_fdm<T>(g, nullptr, alpha, PV<T>::tu(D), PV<T>::tu2(D), PV<T>::w1(D), PV<T>::w2(D), s, nullptr,
                             all));
            break;
        case HPG_K_PRECOND:
            CK((launch_precond<T, double, T>(g, PV<T>::Sinv(D), D.yp, PV<T>::zp(D), s, IterCtl{}, all)));
            break;
        case HPG_K_BAPPLY:
            CK((launch_bapply<T, T, T>(g, PV<T>::zp(D), PV<T>::tu(D), s, nullptr, all)));
            break;
        case HPG_K_SCHUR:
            CK((launch_schur_rest<T, double>(g, PV<T>::gw(D), P0.params.beta, PV<T>::zp(D), PV<T>::tu2(D), D.xs, s,
                                             IterCtl{}, all)));
            break;
        case HPG_K_FACTOR:
            CK(launch_factor<T>(g, PV<T>::gw(D), alpha, P0.params.beta, PV<T>::Sinv(D), nullptr, D.flag,
                                PV<T>::fwork(D), s, all));
            break;
        case HPG_K_NEWTON_APPLY:
            CK(launch_newton_apply(D.gd, D.gw, alpha, P0.params.beta, D.x, D.r, s, all));
            break;
        case HPG_K_EVAL:
            CK(launch_eval(D.gd, D.x + P0.H.Nu0, D.phiq, D.gwt, nullptr, D.egt, D.flag, s, all));
            break;
        default:
            (void)f32;
            return HPG_ERR_ARG;
    }
    return HPG_OK;
}

hpg_status op_launch_kernel_group(hpg_ctx* ctx, std::vector<Problem*>& ps, int cls, int precision, int reps) {
    for (Problem* P : ps)
        if (!P->alloc_done || !P->solved || !groupable(*P) || group_key(*P) != group_key(*ps[0])) {
            ctx->err = "hpg_launch_kernel_batch: every problem must be solved, of one shape and parameter set";
            return HPG_ERR_STATE;
        }
    std::shared_ptr<Group> gref;
    CKS(group_for(ctx, ctx, ps, gref));
    Group& Gp = *gref;
    const bool f32 = precision == HPG_MIXED;
    if (f32 && !Gp.tuned_f) CKS(group_tune_fdm<float>(ctx, Gp));
    if (!f32 && !Gp.tuned_d) CKS(group_tune_fdm<double>(ctx, Gp));
    Problem& P0 = *ps[0];
    DevState& D = P0.D;
    cudaStream_t s = ctx->stream;
    const double alpha = P0.H.alphas.empty() ? 1.0 : P0.H.alphas.back();
    const long long key = ((long long)cls * 2 + (f32 ? 1 : 0)) * 1000003LL + reps;
    auto it = Gp.bench_graphs.find(key);
    if (it == Gp.bench_graphs.end()) {
        const long long gsz = (long long)(P0.H.Nq * gauss_stride(P0.H.kind, P0.H.d));
        const Bat all = Gp.bat(-1);
        CK(launch_copy<double>(D.gw, D.gwl, gsz, s, all));
        CK(launch_convert<double, float>(D.gwl, D.gwf, gsz, s, all));
        CK(cudaStreamSynchronize(s));
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        hpg_status st = HPG_OK;
        const long long before = kernel_launch_count();
        for (int r = 0; r < reps && st == HPG_OK; ++r)
            st = f32 ? group_enqueue<float>(ctx, Gp, cls, alpha) : group_enqueue<double>(ctx, Gp, cls, alpha);
        const long long nk = kernel_launch_count() - before;
        add_kernel_launches(-nk);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != HPG_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        CK(ce);
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        it = Gp.bench_graphs.emplace(key, std::make_pair(ex, nk)).first;
    }
    CK(cudaGraphLaunch(it->second.first, s));
    add_kernel_launches(it->second.second);
    return HPG_OK;
}


// ---- iterative A_alpha^{-1}: preconditioned CG (Section 6.5 compares AMG-preconditioned
// CG with the Cholesky factorisation of A; here the preconditioner is the block Jacobi of
// AinvPrecond, every block solved exactly: the vertex block by fast diagonalisation of
// the Q1 pencils, the edge/face/interior bubble blocks by their dense inverses)
static hpg_status pcg_setup(hpg_ctx* ctx, Problem& P, int kind) {
    DevState& D = P.D;
    if (kind == 3 && D.pcg_ready && !D.pg.Ys) {
        // the vertex-star pencils on top of an existing set-up
        build_ainv_stars(P.H);
        const AinvPrecond& ap = P.H.ap;
        long long npatch = 1, tot = 1;
        for (int j = 0; j < P.H.d; ++j) {
            D.pg.ns[j] = ap.ns[j];
            D.pg.np_[j] = P.H.m[j] >= 2 ? P.H.m[j] - 1 : 1;
            npatch *= D.pg.np_[j];
            tot *= ap.ns[j];
        }
        if ((size_t)(2 * tot) * sizeof(double) > kCellSmemMax) {
            ctx->err = "vertex-star boxes too large for shared memory at this degree";
            return HPG_ERR_ARG;
        }
        bool ok = true;
        for (int j = 0; j < P.H.d; ++j) {
            D.pg.Vs[j] = upload_vec<double>(D, ap.Vs[j], ok, ctx->stream);
            D.pg.lams[j] = upload_vec<double>(D, ap.lams[j], ok, ctx->stream);
        }
        D.pg.Ys = dalloc<double>(D, (size_t)(npatch * tot), ok);
        if (!ok) { ctx->err = "device allocation failed"; return HPG_ERR_OOM; }
        CK(cudaStreamSynchronize(ctx->stream));
        return HPG_OK;
    }
    if (kind == 2 && D.pcg_ready && !D.pg.Cinv) {
        // the cell-patch blocks on top of an existing set-up
        build_ainv_cells(P.H);
        bool ok = true;
        const AinvPrecond& ap = P.H.ap;
        D.pg.Cinv = upload_vec<double>(D, ap.Cinv, ok, ctx->stream);
        D.pg.Y = dalloc<double>(D, (size_t)P.H.Nc * ap.cmax, ok);
        D.pg.cmax = ap.cmax;
        for (int k = 0; k < 64; ++k) { D.pg.csize[k] = ap.csize[k]; D.pg.coff[k] = ap.coff[k]; }
        if (!ok) { ctx->err = "device allocation failed"; return HPG_ERR_OOM; }
        CK(cudaStreamSynchronize(ctx->stream));
        return HPG_OK;
    }
    if (D.pcg_ready) return HPG_OK;
    HostProblem& H = P.H;
    build_ainv_precond(H);
    const AinvPrecond& ap = H.ap;
    cudaStream_t s = ctx->stream;
    bool ok = true;
    const size_t Nu0 = H.Nu0;
    long long nc0 = 1;
    for (int j = 0; j < H.d; ++j) nc0 *= ap.nv[j];
    D.nc0 = nc0;
    D.pr = dalloc<double>(D, Nu0, ok);
    D.pz = dalloc<double>(D, Nu0, ok);
    D.pp = dalloc<double>(D, Nu0, ok);
    D.pq = dalloc<double>(D, Nu0, ok);
    D.pxb = dalloc<double>(D, Nu0, ok);
    D.pbb = dalloc<double>(D, Nu0, ok);
    D.prc = dalloc<double>(D, (size_t)std::max(nc0, 1LL), ok);
    D.pzc = dalloc<double>(D, (size_t)std::max(nc0, 1LL), ok);
    D.pw1 = dalloc<double>(D, (size_t)std::max(nc0, 1LL), ok);
    D.pw2 = dalloc<double>(D, (size_t)std::max(nc0, 1LL), ok);
    if (!ok) { ctx->err = "device allocation failed"; return HPG_ERR_OOM; }
    D.pBinv = upload_vec<double>(D, ap.Binv.empty() ? std::vector<double>(1, 0.0) : ap.Binv, ok, s);
    PcgGeo& pg = D.pg;
    pg = PcgGeo{};
    pg.d = H.d;
    pg.nbub = H.p - 1;
    pg.bmax = 1;
    for (int j = 0; j < kMaxDim; ++j) {
        pg.m[j] = j < H.d ? H.m[j] : 1;
        pg.n1[j] = j < H.d ? H.dir[j].n1 : 1;
        pg.nv[j] = j < H.d ? ap.nv[j] : 1;
    }
    const int ntyp = 1 << H.d;
    pg.eoff[1] = 0;
    for (int t = 1; t < ntyp; ++t) {
        pg.bsize[t] = ap.bsize[t];
        pg.boff[t] = ap.boff[t];
        pg.eoff[t + 1] = pg.eoff[t] + ap.nent[t];
        if (ap.nent[t] > 0) pg.bmax = std::max(pg.bmax, ap.bsize[t]);
    }
    pg.Binv = D.pBinv;
    D.gc = D.gd;
    if (nc0 > 0) {
        for (int j = 0; j < H.d; ++j) {
            D.pVc[j] = upload_vec<double>(D, ap.Vc[j], ok, s);
            D.plamc[j] = upload_vec<double>(D, ap.lamc[j], ok, s);
            D.gc.n1[j] = ap.nv[j];
            D.gc.V[j] = D.pVc[j];
            D.gc.VT[j] = nullptr;        // the coarse pencils keep the strided forward passes
            D.gc.lam[j] = D.plamc[j];
        }
        D.gc.Nu0 = nc0;
        D.gc.gemm_cfg = 0;
    }
    if (!ok) { ctx->err = "device allocation failed"; return HPG_ERR_OOM; }
    CK(cudaStreamSynchronize(s));
    D.pcg_ready = true;
    if (kind >= 2) return pcg_setup(ctx, P, kind);
    return HPG_OK;
}

// z = M_alpha^{-1} r: kind 1, block Jacobi over the entities; kind 2, the two-level
// overlapping Schwarz method with one patch per cell; kind 3, the same with one patch per
// interior vertex (the interior of its star of cells) -- the vertex-based overlapping
// Schwarz method of the p-version (L. F. Pavarino, Numer. Math. 66 (1994)), whose patch
// solves are fast diagonalisations of tensor boxes as in P. F. Fischer's overlapping
// Schwarz method for spectral elements (J. Comput. Phys. 133 (1997)); all with the coarse
// vertex (Q1) space
static hpg_status pcg_precond(hpg_ctx* ctx, Problem& P, int kind, double alpha, const double* r, double* z) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    if (kind >= 2) {
        if (D.nc0 > 0) {
            CK(launch_vertex_gather(D.pg, r, D.prc, D.nc0, s));
            CK(launch_fdm<double>(D.gc, nullptr, alpha, D.prc, D.pzc, D.pw1, D.pw2, s));
        }
        if (kind == 2) {
            CK(launch_cells_solve(D.pg, (long long)P.H.Nc, r, s));
            CK(launch_cells_gather(D.pg, alpha, D.nc0 > 0 ? D.pzc : nullptr, z, (long long)P.H.Nu0, s));
        } else {
            CK(launch_stars_solve(D.pg, r, s));
            CK(launch_stars_gather(D.pg, alpha, D.nc0 > 0 ? D.pzc : nullptr, z, (long long)P.H.Nu0, s));
        }
        return HPG_OK;
    }
    CK(launch_ainv_blocks(D.pg, alpha, r, z, s));
    if (D.nc0 > 0) {
        CK(launch_vertex_gather(D.pg, r, D.prc, D.nc0, s));
        CK(launch_fdm<double>(D.gc, nullptr, alpha, D.prc, D.pzc, D.pw1, D.pw2, s));
        CK(launch_vertex_scatter(D.pg, D.pzc, z, D.nc0, s));
    }
    return HPG_OK;
}

// a . b and, when c is not null, c . c: one synchronisation for both
static hpg_status pcg_dots(hpg_ctx* ctx, Problem& P, const double* a, const double* b, const double* c, double* ab,
                           double* cc) {
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long n = (long long)P.H.Nu0;
    int np = 0;
    CK(launch_dot(a, b, n, D.part, &np, s));
    CK(launch_reduce_sum(D.part, np, D.scal + 10, s));
    if (c) {
        CK(launch_dot(c, c, n, D.part + 1024, &np, s));
        CK(launch_reduce_sum(D.part + 1024, np, D.scal + 11, s));
    }
    CK(cudaMemcpyAsync(D.h_scal + 10, D.scal + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *ab = D.h_scal[10];
    if (cc) *cc = D.h_scal[11];
    return HPG_OK;
}

hpg_status pcg_solve(hpg_ctx* ctx, Problem& P, int kind, double alpha, const double* b, double* x, double rtol,
                     double atol, int maxit, int* its, double* res) {
    CKS(pcg_setup(ctx, P, kind));
    DevState& D = P.D;
    cudaStream_t s = ctx->stream;
    const long long n = (long long)P.H.Nu0;
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    CK(cudaMemcpyAsync(D.pr, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double bb = 0.0;
    CKS(pcg_dots(ctx, P, D.pr, D.pr, nullptr, &bb, nullptr));
    const double bn = std::sqrt(bb);
    *its = 0;
    *res = bn;
    if (!(bn > 0.0)) return HPG_OK;
    const double tol = std::max(atol, rtol * bn);
    CKS(pcg_precond(ctx, P, kind, alpha, D.pr, D.pz));
    CK(cudaMemcpyAsync(D.pp, D.pz, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double rz = 0.0;
    CKS(pcg_dots(ctx, P, D.pr, D.pz, nullptr, &rz, nullptr));
    for (int it = 1; it <= maxit; ++it) {
        CK(launch_aapply(D.gd, alpha, D.pp, D.pq, s));
        double pq = 0.0;
        CKS(pcg_dots(ctx, P, D.pp, D.pq, nullptr, &pq, nullptr));
        if (!(pq > 0.0)) { ctx->err = "CG breakdown (A_alpha not positive on the search direction)"; return HPG_ERR_NONFINITE; }
        const double a = rz / pq;
        CK(launch_axpby(a, D.pp, 1.0, x, n, s));
        CK(launch_axpby(-a, D.pq, 1.0, D.pr, n, s));
        CKS(pcg_precond(ctx, P, kind, alpha, D.pr, D.pz));
        double rz1 = 0.0, rr = 0.0;
        CKS(pcg_dots(ctx, P, D.pr, D.pz, D.pr, &rz1, &rr));
        *its = it;
        *res = std::sqrt(rr);
        if (!std::isfinite(*res)) { ctx->err = "non-finite CG residual"; return HPG_ERR_NONFINITE; }
        if (*res <= tol) break;
        const double beta = rz1 / rz;
        rz = rz1;
        CK(launch_axpby(1.0, D.pz, beta, D.pp, n, s));
    }
    return HPG_OK;
}

hpg_status op_stiffness_pcg(hpg_ctx* ctx, Problem& P, int kind, double alpha, const double* b, double* x, double rtol,
                            double atol, int maxit, int* its) {
    DevState& D = P.D;
    CKS(pcg_setup(ctx, P, kind));
    cudaStream_t s = ctx->stream;
    const long long n = (long long)P.H.Nu0;
    CK(cudaMemcpyAsync(D.pbb, b, n * sizeof(double), cudaMemcpyHostToDevice, s));
    double res = 0.0;
    CKS(pcg_solve(ctx, P, kind, alpha, D.pbb, D.pxb, rtol, atol, maxit, its, &res));
    CK(cudaMemcpyAsync(x, D.pxb, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return HPG_OK;
}

}  // namespace hpg
