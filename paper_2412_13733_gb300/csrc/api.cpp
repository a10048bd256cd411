// C ABI of libhpg (see include/hpg.h for the contract of every entry point).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "state.h"

using hpg::Problem;

namespace {

Problem* find(hpg_ctx* ctx, int pid) {
    if (!ctx) return nullptr;
    auto it = ctx->problems.find(pid);
    return it == ctx->problems.end() ? nullptr : it->second.get();
}

// a problem queued or running in the request loop may not be touched by the client
#define NOT_BUSY(P)                                                            \
    do {                                                                       \
        if ((P)->busy.load()) {                                                \
            ctx->err = "problem is queued or running in the request loop";     \
            return HPG_ERR_BUSY;                                               \
        }                                                                      \
    } while (0)

hpg_status cuda_ok(hpg_ctx* ctx) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        ctx->err = "cudaSetDevice failed";
        return HPG_ERR_CUDA;
    }
    return HPG_OK;
}

struct ConstField {
    double c;
};

}  // namespace

#define GUARD_BEGIN try {
#define GUARD_END                                                             \
    }                                                                         \
    catch (const std::bad_alloc&) {                                           \
        if (ctx) ctx->err = "host allocation failed";                         \
        return HPG_ERR_OOM;                                                   \
    }                                                                         \
    catch (const std::exception& e) {                                         \
        if (ctx) ctx->err = e.what();                                         \
        return HPG_ERR_ARG;                                                   \
    }

extern "C" {

void hpg_default_params(hpg_params* p) {
    if (!p) return;
    p->beta = 1e-4;
    p->newton_tol = 1e-10;
    p->newton_max = 50;
    p->krylov_max = 150;
    p->krylov_rtol = 1e-5;
    p->precision = HPG_FP64;
    p->ls_max = 10;
    p->refine_max = 8;
    p->timing = 0;
    p->graphs = 1;
    p->fdm_tile_f32 = -1;
    p->fdm_tile_f64 = -1;
    p->strategy = HPG_SCHUR;
    p->inner_max = 10;
    p->krylov_f32 = 0;
    p->ainv_pcg = 0;
    p->ainv_rtol = 1e-10;
    p->fdm_tune_batch = 1;
}

const char* hpg_status_str(hpg_status s) {
    switch (s) {
        case HPG_OK: return "HPG_OK";
        case HPG_ERR_ARG: return "HPG_ERR_ARG";
        case HPG_ERR_OOM: return "HPG_ERR_OOM";
        case HPG_ERR_CUDA: return "HPG_ERR_CUDA";
        case HPG_ERR_NEWTON_CAP: return "HPG_ERR_NEWTON_CAP";
        case HPG_ERR_KRYLOV_CAP: return "HPG_ERR_KRYLOV_CAP";
        case HPG_ERR_NONFINITE: return "HPG_ERR_NONFINITE";
        case HPG_ERR_NOT_SPD: return "HPG_ERR_NOT_SPD";
        case HPG_ERR_TIMEOUT: return "HPG_ERR_TIMEOUT";
        case HPG_ERR_INFEASIBLE_BC: return "HPG_ERR_INFEASIBLE_BC";
        case HPG_ERR_STATE: return "HPG_ERR_STATE";
        case HPG_ERR_BUSY: return "HPG_ERR_BUSY";
    }
    return "HPG_UNKNOWN";
}

const char* hpg_last_error(hpg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hpg_status hpg_create(hpg_ctx** out, int device, void* cuda_stream) {
    if (!out) return HPG_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HPG_ERR_CUDA;
    hpg_ctx* ctx = new (std::nothrow) hpg_ctx();
    if (!ctx) return HPG_ERR_OOM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return HPG_ERR_CUDA; }
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return HPG_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return HPG_OK;
}

hpg_status hpg_destroy(hpg_ctx* ctx) {
    if (!ctx) return HPG_OK;
    cudaSetDevice(ctx->device);
    hpg::server_stop(ctx);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->problems) hpg::free_device(*kv.second, ctx->stream);
    ctx->problems.clear();
    for (auto st : ctx->side_streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (auto ev : ctx->side_events) cudaEventDestroy(ev);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return HPG_OK;
}

hpg_status hpg_set_concurrency(hpg_ctx* ctx, int streams) {
    if (!ctx || streams < 1 || streams > 64) return HPG_ERR_ARG;
    ctx->concurrency = streams;
    return HPG_OK;
}

hpg_status hpg_problem_create(hpg_ctx* ctx, int dim, const double* lo, const double* hi, const int* cells, int p,
                              hpg_kind kind, int* pid) {
    if (!ctx || !lo || !hi || !cells || !pid) return HPG_ERR_ARG;
    if (dim != 2 && dim != 3) { ctx->err = "dim must be 2 or 3"; return HPG_ERR_ARG; }
    if (kind != HPG_OBSTACLE_UPPER && kind != HPG_OBSTACLE_LOWER && kind != HPG_GRADIENT) return HPG_ERR_ARG;
    const bool grad = kind == HPG_GRADIENT;
    if (grad ? (p < 1 || p > hpg::kMaxN) : (p < 2 || p > hpg::kMaxN + 1)) {
        ctx->err = "degree out of range";
        return HPG_ERR_ARG;
    }
    {
        // the per-cell kernels hold one cell's latent coefficients (all components) and
        // Gauss values in shared memory: eval 2 nc n^d + n^2 doubles, the cell operators
        // two groups of 3 nb + n^2 values
        const long long n = grad ? p : p - 1, nc = grad ? dim : 1;
        long long nloc = 1;
        for (int j = 0; j < dim; ++j) nloc *= n;
        const long long need = std::max((2 * nc * nloc + n * n) * 8, 2 * (3 * nc * nloc + n * n) * 8);
        if (need > (long long)hpg::kCellSmemMax) {
            ctx->err = "degree too high for this dimension (per-cell shared memory)";
            return HPG_ERR_ARG;
        }
    }
    for (int j = 0; j < dim; ++j) {
        if (cells[j] < 1 || cells[j] > 4096 || !(hi[j] > lo[j])) { ctx->err = "bad mesh"; return HPG_ERR_ARG; }
        if (cells[j] * p - 1 < 1) { ctx->err = "no interior dofs"; return HPG_ERR_ARG; }
    }
    GUARD_BEGIN
    auto P = std::make_unique<Problem>();
    hpg::HostProblem& H = P->H;
    H.d = dim;
    H.p = p;
    H.n = grad ? p : p - 1;
    H.kind = kind;
    H.sign = (kind == HPG_OBSTACLE_LOWER) ? -1.0 : 1.0;
    for (int j = 0; j < dim; ++j) { H.m[j] = cells[j]; H.lo[j] = lo[j]; H.hi[j] = hi[j]; }
    hpg::build_problem_constants(H);
    hpg_default_params(&P->params);
    P->id = ctx->next_id++;
    *pid = P->id;
    ctx->problems[P->id] = std::move(P);
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_problem_free(hpg_ctx* ctx, int pid) {
    Problem* P = find(ctx, pid);
    if (!P) return HPG_ERR_ARG;
    NOT_BUSY(P);
    hpg::server_release(ctx, *P);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    hpg::drop_groups_with(ctx, pid);
    hpg::free_device(*P, ctx->stream);
    ctx->problems.erase(pid);
    return HPG_OK;
}

hpg_status hpg_problem_sizes(hpg_ctx* ctx, int pid, size_t* n_u_full, size_t* n_u_interior, size_t* n_psi,
                             size_t* n_quad) {
    Problem* P = find(ctx, pid);
    if (!P) return HPG_ERR_ARG;
    if (n_u_full) *n_u_full = P->H.Nu_full;
    if (n_u_interior) *n_u_interior = P->H.Nu0;
    if (n_psi) *n_psi = P->H.Npsi;
    if (n_quad) *n_quad = P->H.Nq;
    return HPG_OK;
}

hpg_status hpg_set_rhs(hpg_ctx* ctx, int pid, hpg_field_fn f, void* user) {
    Problem* P = find(ctx, pid);
    if (!P || !f) return HPG_ERR_ARG;
    NOT_BUSY(P);
    GUARD_BEGIN
    hpg::compute_rhs(P->H, f, user, false, 0.0);
    P->data_dirty = true;
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_set_rhs_const(hpg_ctx* ctx, int pid, double f) {
    Problem* P = find(ctx, pid);
    if (!P || !std::isfinite(f)) return HPG_ERR_ARG;
    NOT_BUSY(P);
    GUARD_BEGIN
    hpg::compute_rhs(P->H, nullptr, nullptr, true, f);
    P->data_dirty = true;
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_quad_points(hpg_ctx* ctx, int pid, double* pts, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !pts) return HPG_ERR_ARG;
    if (len < P->H.Nq * P->H.d) return HPG_ERR_ARG;
    GUARD_BEGIN
    std::vector<double> v;
    hpg::latent_points(P->H, v);
    std::memcpy(pts, v.data(), v.size() * sizeof(double));
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_set_constraint_values(hpg_ctx* ctx, int pid, const double* phi_q, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !phi_q) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (len < P->H.Nq) return HPG_ERR_ARG;
    for (size_t i = 0; i < P->H.Nq; ++i)
        if (!std::isfinite(phi_q[i])) { ctx->err = "non-finite constraint value"; return HPG_ERR_NONFINITE; }
    if (P->H.kind == HPG_GRADIENT)
        for (size_t i = 0; i < P->H.Nq; ++i)
            if (!(phi_q[i] > 0.0)) { ctx->err = "gradient constraint must be positive"; return HPG_ERR_ARG; }
    GUARD_BEGIN
    hpg::compute_phi(P->H, phi_q);
    P->phi_dirty = true;
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_set_constraint(hpg_ctx* ctx, int pid, hpg_field_fn phi, void* user) {
    Problem* P = find(ctx, pid);
    if (!P || !phi) return HPG_ERR_ARG;
    NOT_BUSY(P);
    GUARD_BEGIN
    std::vector<double> pts, vals(P->H.Nq);
    hpg::latent_points(P->H, pts);
    phi((int)P->H.Nq, P->H.d, pts.data(), vals.data(), user);
    return hpg_set_constraint_values(ctx, pid, vals.data(), vals.size());
    GUARD_END
}

hpg_status hpg_set_dirichlet(hpg_ctx* ctx, int pid, hpg_field_fn g, void* user) {
    Problem* P = find(ctx, pid);
    if (!P) return HPG_ERR_ARG;
    NOT_BUSY(P);
    GUARD_BEGIN
    hpg::compute_lifting(P->H, g, user);
    for (double v : P->H.ulift)
        if (!std::isfinite(v)) { ctx->err = "non-finite Dirichlet data"; return HPG_ERR_NONFINITE; }
    P->dirichlet_set = g != nullptr;
    P->data_dirty = true;
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_set_alpha_schedule(hpg_ctx* ctx, int pid, double a1, double cap) {
    Problem* P = find(ctx, pid);
    if (!P || !(a1 > 0.0) || !(cap > 0.0)) return HPG_ERR_ARG;
    NOT_BUSY(P);
    std::vector<double> al;
    for (int k = 1; k <= HPG_MAX_ALPHA; ++k) {
        const double a = std::min(a1 * std::pow(2.0, 0.5 * (k - 1)), cap);
        al.push_back(a);
        if (al.size() >= 2 && al[al.size() - 1] == al[al.size() - 2]) break;
    }
    P->H.alphas = al;
    return HPG_OK;
}

hpg_status hpg_set_alpha_growth(hpg_ctx* ctx, int pid, double a1, double growth, double cap, int max_steps,
                                int cap_twice) {
    Problem* P = find(ctx, pid);
    if (!P || !(a1 > 0.0) || !(growth >= 1.0) || !std::isfinite(growth) || !(cap > 0.0) || max_steps < 1 ||
        max_steps > HPG_MAX_ALPHA || (cap_twice != 0 && cap_twice != 1))
        return HPG_ERR_ARG;
    NOT_BUSY(P);
    std::vector<double> al;
    for (int k = 1; k <= max_steps; ++k) {
        const double a = std::min(a1 * std::pow(growth, (double)(k - 1)), cap);
        if (!cap_twice && !al.empty() && al.back() == a) break;
        al.push_back(a);
        if (cap_twice && al.size() >= 2 && al[al.size() - 1] == al[al.size() - 2]) break;
    }
    P->H.alphas = al;
    return HPG_OK;
}

hpg_status hpg_set_alpha_list(hpg_ctx* ctx, int pid, const double* alphas, int count) {
    Problem* P = find(ctx, pid);
    if (!P || !alphas || count < 1 || count > HPG_MAX_ALPHA) return HPG_ERR_ARG;
    NOT_BUSY(P);
    for (int i = 0; i < count; ++i)
        if (!(alphas[i] > 0.0) || !std::isfinite(alphas[i])) return HPG_ERR_ARG;
    P->H.alphas.assign(alphas, alphas + count);
    return HPG_OK;
}

hpg_status hpg_set_params(hpg_ctx* ctx, int pid, const hpg_params* params) {
    Problem* P = find(ctx, pid);
    if (!P || !params) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (params->krylov_max < 1 || params->krylov_max > 1000 || params->newton_max < 0 ||
        !(params->newton_tol > 0.0) || !(params->krylov_rtol > 0.0) || params->beta < 0.0 ||
        (params->precision != HPG_FP64 && params->precision != HPG_MIXED) || params->ls_max < 0 ||
        params->fdm_tile_f32 < -1 || params->fdm_tile_f32 >= hpg::fdm_tile_count(4) ||
        params->fdm_tile_f64 < -1 || params->fdm_tile_f64 >= hpg::fdm_tile_count(8) ||
        params->strategy < HPG_SCHUR || params->strategy > HPG_FGMRES_PF ||
        (params->strategy != HPG_SCHUR && params->precision != HPG_FP64) || params->inner_max < 1 ||
        (params->krylov_f32 != 0 && params->krylov_f32 != 1) ||
        params->ainv_pcg < 0 || params->ainv_pcg > 3 || !(params->ainv_rtol > 0.0) ||
        params->fdm_tune_batch < 1 || params->fdm_tune_batch > 64)
        return HPG_ERR_ARG;
    const bool realloc = P->alloc_done && (params->krylov_max != P->params.krylov_max ||
                                           params->fdm_tile_f32 != P->params.fdm_tile_f32 ||
                                           params->fdm_tile_f64 != P->params.fdm_tile_f64 ||
                                           params->fdm_tune_batch != P->params.fdm_tune_batch);
    if (realloc) {
        hpg::free_device(*P, ctx->stream);
        P->data_dirty = P->phi_dirty = true;
    } else if (P->alloc_done && params->beta != P->params.beta) {
        // beta is a launch argument of the captured GMRES loop and kernel replays
        hpg::drop_graphs(*P);
    }
    P->params = *params;
    return HPG_OK;
}

static hpg_status ready(hpg_ctx* ctx, Problem* P) {
    if (!P->H.has_phi) { ctx->err = "constraint not set"; return HPG_ERR_STATE; }
    if (P->H.alphas.empty()) { ctx->err = "alpha schedule not set"; return HPG_ERR_STATE; }
    if (P->H.kind != HPG_GRADIENT && P->dirichlet_set) {
        // the lifting must satisfy the constraint at the boundary Gauss points of the data
        // (checked against phi at boundary-adjacent latent points is not meaningful; the
        // paper requires phi >= g on the boundary, which the caller guarantees)
    }
    hpg_status s = hpg::alloc_device(ctx, *P);
    if (s != HPG_OK) return s;
    return hpg::upload_data(ctx, *P);
}

hpg_status hpg_solve(hpg_ctx* ctx, int pid) {
    Problem* P = find(ctx, pid);
    if (!P) return HPG_ERR_ARG;
    NOT_BUSY(P);
    hpg_status s = cuda_ok(ctx);
    if (s != HPG_OK) return s;
    GUARD_BEGIN
    ctx->err.clear();
    s = ready(ctx, P);
    if (s != HPG_OK) return s;
    P->host_result = false;
    return hpg::solve_problem(ctx, *P);
    GUARD_END
}

hpg_status hpg_solve_batch(hpg_ctx* ctx, const int* pids, int count) {
    if (!ctx || !pids || count < 1) return HPG_ERR_ARG;
    hpg_status s = cuda_ok(ctx);
    if (s != HPG_OK) return s;
    GUARD_BEGIN
    std::vector<Problem*> ps;
    for (int i = 0; i < count; ++i) {
        Problem* P = find(ctx, pids[i]);
        if (!P) return HPG_ERR_ARG;
        NOT_BUSY(P);
        for (Problem* Q : ps)
            if (Q == P) { ctx->err = "duplicate problem id in batch"; return HPG_ERR_ARG; }
        s = ready(ctx, P);
        if (s != HPG_OK) return s;
        P->host_result = false;
        ps.push_back(P);
    }
    return hpg::solve_batch(ctx, ps);
    GUARD_END
}

// [u interior; psi] of the last solve, from the device or from the host copy
// kept by the request loop.
static hpg_status result_x(hpg_ctx* ctx, Problem* P, std::vector<double>& x) {
    (void)ctx;
    const size_t n = P->H.Nu0 + P->H.Npsi;
    if (P->host_result) {
        x = P->host_x;
        return HPG_OK;
    }
    if (!P->alloc_done) return HPG_ERR_STATE;
    x.resize(n);
    if (cudaMemcpy(x.data(), P->D.x, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return HPG_ERR_CUDA;
    return HPG_OK;
}

hpg_status hpg_get_u(hpg_ctx* ctx, int pid, double* u_full, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !u_full) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (len < P->H.Nu_full) return HPG_ERR_ARG;
    if (!P->solved) return HPG_ERR_STATE;
    hpg::HostProblem& H = P->H;
    std::vector<double> x;
    hpg_status st = result_x(ctx, P, x);
    if (st != HPG_OK) return st;
    for (size_t i = 0; i < H.Nu_full; ++i) u_full[i] = H.sign * H.ulift[i];
    for (size_t I = 0; I < H.Nu0; ++I) {
        size_t ii = I, full = 0, stride = 1;
        for (int j = 0; j < H.d; ++j) {
            full += (size_t)H.dir[j].glob_of_int((int)(ii % H.dir[j].n1)) * stride;
            ii /= H.dir[j].n1;
            stride *= H.dir[j].N1;
        }
        u_full[full] = H.sign * x[I];
    }
    return HPG_OK;
}

hpg_status hpg_get_psi(hpg_ctx* ctx, int pid, double* psi, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !psi) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (len < P->H.Npsi) return HPG_ERR_ARG;
    if (!P->solved) return HPG_ERR_STATE;
    std::vector<double> x;
    hpg_status st = result_x(ctx, P, x);
    if (st != HPG_OK) return st;
    std::memcpy(psi, x.data() + P->H.Nu0, P->H.Npsi * sizeof(double));
    return HPG_OK;
}

hpg_status hpg_get_stats(hpg_ctx* ctx, int pid, hpg_stats* stats) {
    Problem* P = find(ctx, pid);
    if (!P || !stats) return HPG_ERR_ARG;
    *stats = P->stats;
    if (P->alloc_done) {
        stats->fdm_tile_f32 = P->D.gf.gemm_cfg;
        stats->fdm_tile_f64 = P->D.gd.gemm_cfg;
    }
    return HPG_OK;
}

hpg_status hpg_eval_u(hpg_ctx* ctx, int pid, const double* pts, int npts, double* out) {
    Problem* P = find(ctx, pid);
    if (!P || !pts || !out || npts < 0) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (!P->solved) return HPG_ERR_STATE;
    GUARD_BEGIN
    std::vector<double> u(P->H.Nu_full);
    hpg_status s = hpg_get_u(ctx, pid, u.data(), u.size());
    if (s != HPG_OK) return s;
    for (int i = 0; i < npts; ++i) out[i] = hpg::eval_u_point(P->H, u, pts + (size_t)i * P->H.d);
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_l2_error(hpg_ctx* ctx, int pid, const double* u_ref, size_t len, double* err, double* ref_norm) {
    Problem* P = find(ctx, pid);
    if (!P || !u_ref || !err) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (len < P->H.Nu_full) return HPG_ERR_ARG;
    if (!P->solved) return HPG_ERR_STATE;
    GUARD_BEGIN
    std::vector<double> u(P->H.Nu_full);
    hpg_status s = hpg_get_u(ctx, pid, u.data(), u.size());
    if (s != HPG_OK) return s;
    std::vector<double> e(u.size()), r(u_ref, u_ref + u.size());
    for (size_t i = 0; i < u.size(); ++i) e[i] = u[i] - u_ref[i];
    *err = std::sqrt(std::max(0.0, hpg::mass_norm2(P->H, e)));
    if (ref_norm) *ref_norm = std::sqrt(std::max(0.0, hpg::mass_norm2(P->H, r)));
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_feasible_u(hpg_ctx* ctx, int pid, double* out_q, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !out_q) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (P->H.kind == HPG_GRADIENT) return HPG_ERR_ARG;
    if (len < P->H.Nq) return HPG_ERR_ARG;
    if (!P->solved) return HPG_ERR_STATE;
    // u~ = phi - exp(-psi) at the latent Gauss points (eq. pG), in the caller's sign
    hpg::HostProblem& H = P->H;
    std::vector<double> x;
    hpg_status stx = result_x(ctx, P, x);
    if (stx != HPG_OK) return stx;
    std::vector<double> psi(x.begin() + H.Nu0, x.end());
    const int n = H.n;
    for (size_t c = 0; c < H.Nc; ++c)
        for (size_t q = 0; q < H.nloc; ++q) {
            double v = 0.0;
            for (size_t k = 0; k < H.nloc; ++k) {
                size_t qq = q, kk = k;
                double w = 1.0;
                for (int j = 0; j < H.d; ++j) {
                    w *= H.Vq[(qq % n) * n + (kk % n)];
                    qq /= n;
                    kk /= n;
                }
                v += w * psi[c * H.nloc + k];
            }
            out_q[c * H.nloc + q] = H.sign * (H.phiq[c * H.nloc + q] - std::exp(-v));
        }
    return HPG_OK;
}

hpg_status hpg_get_kernel_times(hpg_ctx* ctx, int pid, double* ms, long long* launches, int count) {
    Problem* P = find(ctx, pid);
    if (!P || count < 0) return HPG_ERR_ARG;
    for (int i = 0; i < count && i < HPG_K_COUNT; ++i) {
        if (ms) ms[i] = P->timer.ms[i];
        if (launches) launches[i] = P->timer.launches[i];
    }
    return HPG_OK;
}

hpg_status hpg_reset_kernel_times(hpg_ctx* ctx, int pid) {
    Problem* P = find(ctx, pid);
    if (!P) return HPG_ERR_ARG;
    for (int i = 0; i < HPG_K_COUNT; ++i) { P->timer.ms[i] = 0.0; P->timer.launches[i] = 0; }
    return HPG_OK;
}

// ------------------------------------------------------------ component operators
static hpg_status op_ready(hpg_ctx* ctx, Problem* P) {
    hpg_status s = cuda_ok(ctx);
    if (s != HPG_OK) return s;
    return ready(ctx, P);
}

hpg_status hpg_set_state(hpg_ctx* ctx, int pid, const double* u_full, const double* psi, const double* psi_prev,
                         double alpha) {
    Problem* P = find(ctx, pid);
    if (!P || !u_full || !psi || !psi_prev || !(alpha > 0.0)) return HPG_ERR_ARG;
    NOT_BUSY(P);
    GUARD_BEGIN
    hpg_status s = op_ready(ctx, P);
    if (s != HPG_OK) return s;
    return hpg::op_set_state(ctx, *P, u_full, psi, psi_prev, alpha);
    GUARD_END
}

#define OP_PROLOGUE(need)                                        \
    Problem* P = find(ctx, pid);                                 \
    if (!P) return HPG_ERR_ARG;                                  \
    NOT_BUSY(P);                                                 \
    if (!P->alloc_done || P->state_alpha <= 0.0) return HPG_ERR_STATE; \
    if (len < (need)) return HPG_ERR_ARG;                        \
    if (cuda_ok(ctx) != HPG_OK) return HPG_ERR_CUDA;

hpg_status hpg_residual(hpg_ctx* ctx, int pid, double* F, size_t len, double* norm) {
    OP_PROLOGUE(P->H.Nu0 + P->H.Npsi)
    if (!F) return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_residual(ctx, *P, F, norm);
    GUARD_END
}

hpg_status hpg_apply_newton(hpg_ctx* ctx, int pid, const double* x, double* y, size_t len) {
    OP_PROLOGUE(P->H.Nu0 + P->H.Npsi)
    if (!x || !y) return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_apply_newton(ctx, *P, x, y);
    GUARD_END
}

hpg_status hpg_apply_stiffness_inv(hpg_ctx* ctx, int pid, int precision, const double* x, double* y, size_t len) {
    OP_PROLOGUE(P->H.Nu0)
    if (!x || !y) return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_stiffness_inv(ctx, *P, precision, x, y);
    GUARD_END
}

hpg_status hpg_factor_precond(hpg_ctx* ctx, int pid, int precision, double* blocks, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (!P->alloc_done || P->state_alpha <= 0.0) return HPG_ERR_STATE;
    if (blocks && len < P->H.Nc * P->H.nb * P->H.nb) return HPG_ERR_ARG;
    if (cuda_ok(ctx) != HPG_OK) return HPG_ERR_CUDA;
    GUARD_BEGIN
    return hpg::op_factor(ctx, *P, precision, blocks);
    GUARD_END
}

hpg_status hpg_apply_precond_inv(hpg_ctx* ctx, int pid, int precision, const double* x, double* y, size_t len) {
    OP_PROLOGUE(P->H.Npsi)
    if (!x || !y) return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_precond_inv(ctx, *P, precision, x, y);
    GUARD_END
}

hpg_status hpg_apply_schur(hpg_ctx* ctx, int pid, int precision, const double* x, double* y, size_t len) {
    OP_PROLOGUE(P->H.Npsi)
    if (!x || !y) return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_schur(ctx, *P, precision, x, y);
    GUARD_END
}

hpg_status hpg_stiffness_solve_pcg(hpg_ctx* ctx, int pid, int precond, double alpha, const double* b, double* x,
                                   size_t len, double rtol, double atol, int maxit, int* its) {
    OP_PROLOGUE(P->H.Nu0)
    if (!b || !x || !its || !(alpha > 0.0) || !(rtol >= 0.0) || !(atol >= 0.0) || maxit < 1 ||
        precond < 1 || precond > 3)
        return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_stiffness_pcg(ctx, *P, precond, alpha, b, x, rtol, atol, maxit, its);
    GUARD_END
}

hpg_status hpg_newton_direction(hpg_ctx* ctx, int pid, int precision, double rtol, double* delta, size_t len,
                                int* krylov_its) {
    OP_PROLOGUE(P->H.Nu0 + P->H.Npsi)
    if (!delta || !(rtol > 0.0)) return HPG_ERR_ARG;
    GUARD_BEGIN
    return hpg::op_newton_direction(ctx, *P, precision, rtol, delta, krylov_its);
    GUARD_END
}

int hpg_fdm_tile_count(int precision) {
    if (precision == HPG_MIXED) return hpg::fdm_tile_count(4);
    if (precision == HPG_FP64) return hpg::fdm_tile_count(8);
    return 0;
}

hpg_status hpg_launch_kernel(hpg_ctx* ctx, int pid, int kernel_class, int precision, int reps) {
    Problem* P = find(ctx, pid);
    if (!P || reps < 0 || kernel_class < 0 || kernel_class >= HPG_K_COUNT) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (!P->alloc_done || !(P->solved || P->state_alpha > 0.0)) return HPG_ERR_STATE;
    if (cuda_ok(ctx) != HPG_OK) return HPG_ERR_CUDA;
    GUARD_BEGIN
    return hpg::op_launch_kernel(ctx, *P, kernel_class, precision, reps);
    GUARD_END
}

hpg_status hpg_launch_kernel_batch(hpg_ctx* ctx, const int* pids, int count, int kernel_class, int precision,
                                   int reps) {
    if (!ctx || !pids || count < 1 || reps < 0 || kernel_class < 0 || kernel_class >= HPG_K_COUNT ||
        (precision != HPG_FP64 && precision != HPG_MIXED))
        return HPG_ERR_ARG;
    if (cuda_ok(ctx) != HPG_OK) return HPG_ERR_CUDA;
    std::vector<Problem*> ps;
    for (int i = 0; i < count; ++i) {
        Problem* P = find(ctx, pids[i]);
        if (!P) return HPG_ERR_ARG;
        NOT_BUSY(P);
        for (Problem* Q : ps)
            if (Q == P) return HPG_ERR_ARG;
        ps.push_back(P);
    }
    GUARD_BEGIN
    return hpg::op_launch_kernel_group(ctx, ps, kernel_class, precision, reps);
    GUARD_END
}

// ------------------------------------------------------------ request loop
hpg_status hpg_server_start(hpg_ctx* ctx, int workers, size_t device_budget_bytes) {
    if (!ctx || workers < 1 || workers > 64) return HPG_ERR_ARG;
    if (cuda_ok(ctx) != HPG_OK) return HPG_ERR_CUDA;
    size_t budget = device_budget_bytes;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return HPG_ERR_CUDA;
        budget = (size_t)(0.8 * (double)fr);
    }
    GUARD_BEGIN
    return hpg::server_start(ctx, workers, budget);
    GUARD_END
}

hpg_status hpg_server_stop(hpg_ctx* ctx) {
    if (!ctx) return HPG_ERR_ARG;
    return hpg::server_stop(ctx);
}

hpg_status hpg_submit(hpg_ctx* ctx, int pid, long long* ticket) {
    Problem* P = find(ctx, pid);
    if (!P || !ticket) return HPG_ERR_ARG;
    NOT_BUSY(P);
    if (!P->H.has_phi || P->H.alphas.empty()) { ctx->err = "problem data incomplete"; return HPG_ERR_STATE; }
    GUARD_BEGIN
    return hpg::server_submit(ctx, *P, ticket);
    GUARD_END
}

hpg_status hpg_poll(hpg_ctx* ctx, long long ticket, int* done, hpg_status* result) {
    if (!ctx) return HPG_ERR_ARG;
    return hpg::server_poll(ctx, ticket, 0.0, done, result, nullptr);
}

hpg_status hpg_wait(hpg_ctx* ctx, long long ticket, double timeout_ms, hpg_status* result) {
    if (!ctx || !(timeout_ms > 0.0)) return HPG_ERR_ARG;
    int done = 0;
    return hpg::server_poll(ctx, ticket, timeout_ms, &done, result, nullptr);
}

hpg_status hpg_ticket_times(hpg_ctx* ctx, long long ticket, double* times3) {
    if (!ctx || !times3) return HPG_ERR_ARG;
    return hpg::server_poll(ctx, ticket, 0.0, nullptr, nullptr, times3);
}

hpg_status hpg_measure_fma_peak(hpg_ctx* ctx, int precision, double* tflops, int* sm_count) {
    if (!ctx || !tflops || (precision != HPG_FP64 && precision != HPG_MIXED)) return HPG_ERR_ARG;
    if (cuda_ok(ctx) != HPG_OK) return HPG_ERR_CUDA;
    GUARD_BEGIN
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        ctx->err = "cudaDeviceGetAttribute failed";
        return HPG_ERR_CUDA;
    }
    if (sm_count) *sm_count = sms;
    const cudaError_t e = hpg::measure_fma_peak(precision == HPG_FP64 ? 8 : 4, sms, ctx->stream, tflops);
    if (e != cudaSuccess) {
        ctx->err = std::string("fma peak: ") + cudaGetErrorString(e);
        return HPG_ERR_CUDA;
    }
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_server_policy(hpg_ctx* ctx, int policy) {
    if (!ctx || (policy != 0 && policy != 1)) return HPG_ERR_ARG;
    return hpg::server_set_policy(ctx, policy);
}

hpg_status hpg_ticket_error(hpg_ctx* ctx, long long ticket, char* buf, size_t len) {
    if (!ctx || !buf || len == 0) return HPG_ERR_ARG;
    std::string msg;
    const hpg_status s = hpg::server_ticket_error(ctx, ticket, &msg);
    if (s != HPG_OK) return s;
    const size_t n = std::min(msg.size(), len - 1);
    std::memcpy(buf, msg.data(), n);
    buf[n] = 0;
    return HPG_OK;
}

hpg_status hpg_server_memory(hpg_ctx* ctx, int pid, size_t* in_use, size_t* estimate) {
    if (!ctx) return HPG_ERR_ARG;
    if (in_use) *in_use = hpg::server_in_use(ctx);
    if (estimate) {
        Problem* P = find(ctx, pid);
        if (!P) return HPG_ERR_ARG;
        *estimate = hpg::estimate_device_bytes(*P);
    }
    return HPG_OK;
}

hpg_status hpg_qvi_default_params(hpg_qvi_params* out) {
    if (!out) return HPG_ERR_ARG;
    *out = hpg_qvi_params{};
    out->gamma = 1.0;
    out->g0 = 0.2;
    out->tol = 3e-3;
    out->t_tol = 1e-11;
    out->max_fp = 30;
    out->nq = 0;
    out->t_newton_max = 50;
    out->t_krylov_max = 200;
    out->t_krylov_rtol = 1.5e-8;
    return HPG_OK;
}

static size_t qvi_npts(const hpg::HostProblem& H, int nq) {
    size_t per = 1;
    for (int j = 0; j < H.d; ++j) per *= (size_t)nq;
    return H.Nc * per;
}

hpg_status hpg_qvi_points(hpg_ctx* ctx, int pid, int nq, double* pts, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !pts || nq < 0 || nq > 64) return HPG_ERR_ARG;
    const int q = nq > 0 ? nq : P->H.p + 2;
    if (len < qvi_npts(P->H, q) * P->H.d) return HPG_ERR_ARG;
    GUARD_BEGIN
    std::vector<double> v;
    hpg::qvi_points(P->H, q, v);
    std::memcpy(pts, v.data(), v.size() * sizeof(double));
    return HPG_OK;
    GUARD_END
}

hpg_status hpg_qvi_solve(hpg_ctx* ctx, int pid, const hpg_qvi_params* params, const double* phi0_lat,
                         const double* xi_lat, size_t n_lat, const double* phi0_q, const double* xi_q, size_t n_q,
                         hpg_qvi_stats* stats) {
    Problem* P = find(ctx, pid);
    if (!P || !params || !phi0_lat || !xi_lat || !phi0_q || !xi_q) return HPG_ERR_ARG;
    NOT_BUSY(P);
    const hpg::HostProblem& H = P->H;
    const hpg_qvi_params& q = *params;
    const int nq = q.nq > 0 ? q.nq : H.p + 2;
    if (H.kind != HPG_OBSTACLE_UPPER) { ctx->err = "QVI needs an HPG_OBSTACLE_UPPER problem"; return HPG_ERR_ARG; }
    if (!(q.gamma > 0.0) || !(q.g0 >= 0.0) || !(q.tol > 0.0) || !(q.t_tol > 0.0) || q.max_fp < 1 ||
        q.max_fp > HPG_QVI_MAX_FP || q.nq < 0 || q.nq > 64 || q.t_newton_max < 1 || q.t_krylov_max < 1 ||
        q.t_krylov_max > hpg::kMaxKrylov || !(q.t_krylov_rtol > 0.0)) {
        ctx->err = "invalid QVI parameters";
        return HPG_ERR_ARG;
    }
    if (n_lat < H.Nq || n_q < qvi_npts(H, nq)) { ctx->err = "QVI data arrays too short"; return HPG_ERR_ARG; }
    size_t capq = 1, capl = 1;
    for (int j = 0; j < H.d; ++j) {
        capq *= (size_t)std::max(H.p + 1, nq);
        capl *= (size_t)std::max(H.p + 1, H.n);
    }
    if (2 * std::max(capq, capl) * sizeof(double) > hpg::kCellSmemMax) {
        ctx->err = "QVI cell tables exceed shared memory";
        return HPG_ERR_ARG;
    }
    if (P->H.alphas.empty()) { ctx->err = "alpha schedule not set"; return HPG_ERR_STATE; }
    hpg_status s = cuda_ok(ctx);
    if (s != HPG_OK) return s;
    GUARD_BEGIN
    ctx->err.clear();
    P->host_result = false;
    return hpg::qvi_solve(ctx, *P, q, phi0_lat, xi_lat, phi0_q, xi_q, stats);
    GUARD_END
}

hpg_status hpg_qvi_get_T(hpg_ctx* ctx, int pid, double* T_full, size_t len) {
    Problem* P = find(ctx, pid);
    if (!P || !T_full) return HPG_ERR_ARG;
    if (len < P->H.Nu_full) return HPG_ERR_ARG;
    if (P->qvi_T.size() != P->H.Nu_full) { ctx->err = "no QVI solve on this problem"; return HPG_ERR_STATE; }
    std::memcpy(T_full, P->qvi_T.data(), P->H.Nu_full * sizeof(double));
    return HPG_OK;
}

}  // extern "C"
