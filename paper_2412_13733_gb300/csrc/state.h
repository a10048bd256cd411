// Per-problem device state and the solver driver of libhpg.
#pragma once

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "device.h"

namespace hpg {

// Device copy of one 1D stencil for both precisions.
struct DevSten {
    int* cnt = nullptr;
    int* col = nullptr;
    double* vd = nullptr;
    float* vf = nullptr;
    int* lcol = nullptr;
};

struct DevTileCols {
    int* list = nullptr;
    int* count = nullptr;
    int cap = 0;
};

struct DevState {
    // flexible GMRES on G (allocated on first use): basis, preconditioned directions,
    // dot partials, coefficients, block scratch
    double *fV = nullptr, *fZ = nullptr, *fpart = nullptr, *fh = nullptr;
    double *fT1 = nullptr, *fT2 = nullptr, *fP1 = nullptr;
    int fm = 0;
    // constant operators
    DevSten A[kMaxDim], M[kMaxDim], B[kMaxDim], BT[kMaxDim], Bd[kMaxDim], BdT[kMaxDim];
    DevTileCols tu[kMaxDim], tp[kMaxDim];
    double *Vq_d = nullptr, *wq_d = nullptr, *Mpsi_d = nullptr, *Kpsi_d = nullptr, *C_d = nullptr;
    float *Vq_f = nullptr, *wq_f = nullptr, *Mpsi_f = nullptr, *Kpsi_f = nullptr, *C_f = nullptr;
    double *V_d[kMaxDim] = {}, *lam_d[kMaxDim] = {};
    float *V_f[kMaxDim] = {}, *lam_f[kMaxDim] = {};
    double* VT_d[kMaxDim] = {};
    float* VT_f[kMaxDim] = {};
    FdmTma tma{};                 // TMA/tcgen05 fast diagonalisation of this problem (FP32)
    bool tma_ok = false;
    Geo<double> gd{};
    Geo<float> gf{};
    // data
    double *rA = nullptr, *rB = nullptr, *bf = nullptr, *phiz = nullptr, *phiq = nullptr;
    // state: x = [u (interior); psi] contiguous so Newton updates are one axpy
    double *x = nullptr, *xt = nullptr;          // current and trial
    double* x0 = nullptr;                        // HPG_MIXED: x at the start of the proximal step
    double *psi_prev = nullptr;
    double *gw = nullptr, *gwt = nullptr;        // Gauss weights (current, trial)
    double* gwl = nullptr;                       // weights of the current linearisation (FP64)
    float* gwf = nullptr;                        // FP32 copy of gwl
    double* fwork_d = nullptr;                   // factor workspace when blocks exceed shared memory
    float* fwork_f = nullptr;
    double* alpha_dev = nullptr;                 // alpha of the current proximal step (device)
    int* perm0 = nullptr;                        // axis-0 row order of the FP64 u-row tiles
    // captured GMRES loop per (operator, basis) precision: FP64/FP64, FP32/FP64, FP32/FP32
    cudaGraphExec_t gmres_graph[3] = {nullptr, nullptr, nullptr};
    long long graph_kernels[3] = {0, 0, 0};                 // kernels in one loop body
    bool gmres_graph_failed[3] = {false, false, false};     // conditional graphs unsupported
    std::map<long long, std::pair<cudaGraphExec_t, long long>> bench_graphs;   // hpg_launch_kernel replays
    double *eg = nullptr, *egt = nullptr;
    double *F = nullptr, *Ft = nullptr, *delta = nullptr, *r = nullptr, *dcorr = nullptr;
    double* Sinv_d = nullptr;
    float* Sinv_f = nullptr;
    // Schur temporaries
    double *tu_d = nullptr, *w1_d = nullptr, *w2_d = nullptr, *tu2_d = nullptr;
    float *tu_f = nullptr, *tu2_f = nullptr, *w1_f = nullptr, *w2_f = nullptr;
    double *zp_d = nullptr, *yp = nullptr, *xs = nullptr;
    float *zp_f = nullptr;
    double* part = nullptr;      // residual partials
    double* scal = nullptr;      // [0] |F|^2 reduce target, ...
    int* flag = nullptr;         // eval/factor flags
    GmresDev gm{};
    // pinned host mirror for scalars (owned by the Problem, kept across re-allocation)
    double* h_scal = nullptr;
    int* h_iflag = nullptr;
    // iterative A_alpha^{-1} (preconditioned CG, allocated on first use)
    double *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr, *pxb = nullptr, *pbb = nullptr;
    double *prc = nullptr, *pzc = nullptr, *pw1 = nullptr, *pw2 = nullptr, *pBinv = nullptr;
    double* pVc[kMaxDim] = {};
    double* plamc[kMaxDim] = {};
    PcgGeo pg{};
    Geo<double> gc{};
    long long nc0 = 0;
    bool pcg_ready = false;
    char* slab = nullptr;                  // one allocation holding every per-problem buffer (layout fixed
    size_t slab_bytes = 0;                 // by the problem's shape), see alloc_device
    cudaStream_t alloc_stream = nullptr;   // stream the stream-ordered allocations were made on
    std::vector<void*> allocs;
    size_t bytes = 0;
};

struct Group;

struct KernelTimer {
    bool on = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    std::vector<cudaEvent_t> pool;
    double ms[HPG_K_COUNT] = {};
    long long launches[HPG_K_COUNT] = {};
};

struct Server;

struct Problem {
    int id = 0;
    std::atomic<bool> busy{false};   // queued or running in the request loop
    bool host_result = false;        // result copied to host_x and device memory released
    std::vector<double> host_x;      // [u interior; psi] of the last solve when host_result
    HostProblem H;
    hpg_params params{};
    bool alloc_done = false;
    long long alloc_gen = 0;     // changes whenever the device state is (re)allocated
    bool dirichlet_set = false;
    bool data_dirty = true;      // f load / lifting terms changed since the last upload
    bool phi_dirty = true;       // constraint values changed since the last upload
    long long h2d_bytes = 0;     // bytes uploaded by the last upload_data
    DevState D;
    hpg_stats stats{};
    bool solved = false;
    double state_alpha = 0.0;
    KernelTimer timer;
    double* pinned_scal = nullptr;   // 16 doubles + 8 ints of pinned host memory, lazily allocated
    int* pinned_iflag = nullptr;
    std::vector<double> qvi_T;       // temperature of the last QVI solve (full u numbering)
    ~Problem();
};

}  // namespace hpg

struct hpg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::map<int, std::unique_ptr<hpg::Problem>> problems;
    int next_id = 1;
    std::string err;
    int concurrency = 8;                       // streams/host workers used by hpg_solve_batch
    std::vector<cudaStream_t> side_streams;    // owned; forked from / joined to `stream`
    std::vector<cudaEvent_t> side_events;
    hpg::Server* server = nullptr;             // request loop (hpg_server_start)
    // lockstep groups of hpg_solve_batch, by problem ids (their launch tables and loop graphs)
    std::map<std::vector<int>, std::shared_ptr<hpg::Group>> groups;
    std::mutex groups_mu;
};

namespace hpg {

hpg_status alloc_device(hpg_ctx* ctx, Problem& P);
// Release the problem's device buffers, stream-ordered on `s`.
void free_device(Problem& P, cudaStream_t s);
// Destroy the problem's captured CUDA graphs (they hold launch arguments such as beta);
// they are re-captured on next use.
void drop_graphs(Problem& P);
hpg_status upload_data(hpg_ctx* ctx, Problem& P);
hpg_status solve_problem(hpg_ctx* ctx, Problem& P);
hpg_status solve_batch(hpg_ctx* ctx, std::vector<Problem*>& probs);
// Same-shape problems in lockstep (every launch serves all of them); `home` owns the
// group cache, ctx gives the stream.  Per-problem status in each problem's stats.
hpg_status solve_group(hpg_ctx* home, hpg_ctx* ctx, std::vector<Problem*>& ps, std::vector<std::string>* errs);
// Forget the cached groups that contain problem pid.
void drop_groups_with(hpg_ctx* ctx, int pid);
// component operators
hpg_status op_set_state(hpg_ctx* ctx, Problem& P, const double* u_full, const double* psi, const double* psi_prev,
                        double alpha);
hpg_status op_residual(hpg_ctx* ctx, Problem& P, double* F, double* norm);
hpg_status op_apply_newton(hpg_ctx* ctx, Problem& P, const double* x, double* y);
hpg_status op_stiffness_inv(hpg_ctx* ctx, Problem& P, int precision, const double* x, double* y);
hpg_status op_factor(hpg_ctx* ctx, Problem& P, int precision, double* blocks);
hpg_status op_precond_inv(hpg_ctx* ctx, Problem& P, int precision, const double* x, double* y);
hpg_status op_schur(hpg_ctx* ctx, Problem& P, int precision, const double* x, double* y);
hpg_status op_newton_direction(hpg_ctx* ctx, Problem& P, int precision, double rtol, double* delta, int* its);
hpg_status op_launch_kernel(hpg_ctx* ctx, Problem& P, int cls, int precision, int reps);
// Preconditioned CG on A_alpha x = b (device vectors of n_u interior entries), stopping at
// ||r|| <= max(atol, rtol ||b||) or maxit; *its iterations, *res the final ||r||.
// kind 1: block Jacobi over the basis entities; 2: overlapping cell patches; 3: overlapping
// vertex-star patches (both two-level, with the coarse vertex space).
hpg_status pcg_solve(hpg_ctx* ctx, Problem& P, int kind, double alpha, const double* b, double* x, double rtol,
                     double atol, int maxit, int* its, double* res);
hpg_status op_stiffness_pcg(hpg_ctx* ctx, Problem& P, int kind, double alpha, const double* b, double* x, double rtol,
                            double atol, int maxit, int* its);
hpg_status op_launch_kernel_group(hpg_ctx* ctx, std::vector<Problem*>& ps, int cls, int precision, int reps);
// request loop
size_t estimate_device_bytes(const Problem& P);
hpg_status server_start(hpg_ctx* ctx, int workers, size_t budget);
hpg_status server_stop(hpg_ctx* ctx);
hpg_status server_submit(hpg_ctx* ctx, Problem& P, long long* ticket);
hpg_status server_poll(hpg_ctx* ctx, long long ticket, double wait_ms, int* done, hpg_status* result,
                       double* times3);
void server_release(hpg_ctx* ctx, Problem& P);
hpg_status server_ticket_error(hpg_ctx* ctx, long long ticket, std::string* msg);
hpg_status server_set_policy(hpg_ctx* ctx, int policy);
size_t server_in_use(hpg_ctx* ctx);
// thermoforming QVI (Section 6.4): T-equation Gauss points (Nc nq^d x d, cell-major,
// x fastest) and the fixed point of obstacle and temperature solves
void qvi_points(const HostProblem& H, int nq, std::vector<double>& pts);
hpg_status qvi_solve(hpg_ctx* ctx, Problem& P, const hpg_qvi_params& q, const double* phi0_lat, const double* xi_lat,
                     const double* phi0_q, const double* xi_q, hpg_qvi_stats* st);

}  // namespace hpg
