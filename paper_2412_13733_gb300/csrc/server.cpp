// Request loop of libhpg: continuous batching of independent hpG solves.
//
// Requests (problems already set up by the client) are admitted in arrival
// order as soon as a worker is free and their device footprint fits in the
// memory budget (first fit, so a large request does not block smaller ones
// behind it).  Each worker owns a CUDA stream; its problem's Newton/Krylov state
// stays resident on the device for the whole solve, and the kernels of all
// running requests overlap on the GPU.  A request's device memory is counted
// against the budget from admission until its solve ends; then the result is
// copied to the host and the device buffers are released.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>

#include "state.h"

namespace hpg {

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct Request {
    long long ticket = 0;
    Problem* P = nullptr;
    size_t bytes = 0;
    int state = 0;              // 0 queued, 1 running, 2 done
    hpg_status result = HPG_OK;
    std::string err;            // the solver's message when result != HPG_OK
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Server {
    hpg_ctx* ctx = nullptr;
    int workers = 1;
    size_t budget = 0;
    size_t in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<long long, Request> reqs;
    std::map<Problem*, size_t> charged;   // admitted problems and their bytes
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    bool stopping = false;
    long long next_ticket = 1;
    int policy = 0;                       // 0: arrival order; 1: largest work first
};

// Work of a request for the largest-first policy: unknowns times the degree (the Krylov
// and factorisation work per Newton step grows with both).
static double request_work(const Problem& P) {
    return (double)(P.H.Nu0 + P.H.Npsi) * (double)P.H.p;
}

// Device bytes of a problem's buffers (the allocations of alloc_device).
size_t estimate_device_bytes(const Problem& P) {
    const HostProblem& H = P.H;
    const size_t Nu0 = H.Nu0, Npsi = H.Npsi, Nx = Nu0 + Npsi;
    const size_t gsz = H.Nq * (size_t)gauss_stride(H.kind, H.d);
    const size_t kmax = (size_t)std::max(1, P.params.krylov_max);
    size_t b = 0;
    for (int j = 0; j < H.d; ++j) {
        const size_t n1 = H.dir[j].n1;
        b += n1 * n1 * 24 + n1 * 12;                      // V, V^T, lam (FP64 + FP32)
        b += (size_t)kEll * 20 * (4 * n1 + 2 * H.m[j] * H.n);   // stencils
    }
    b += Nu0 * (8 * 8 + 4 * 4);                          // rA, bf, tu/w buffers
    b += Npsi * 8 * 10 + Npsi * 4;                       // psi-sized vectors
    b += Nx * 8 * 8;                                     // x, xt, x0, F, Ft, delta, r, dcorr
    b += gsz * (8 * 3 + 4);                              // Gauss weights
    b += H.Nq * 8;
    b += H.Nc * H.nb * H.nb * 12;                        // S-hat inverses (FP64 + FP32)
    b += factor_workspace_elems(H.n, H.d, (int)H.nb, H.ncomp, (long long)H.Nc, 8) * 8;
    b += factor_workspace_elems(H.n, H.d, (int)H.nb, H.ncomp, (long long)H.Nc, 4) * 4;
    {
        // TMA fast diagonalisation: four sliced workspace buffers and the sliced pass matrices
        size_t ws = 0;
        for (int j = 0; j < H.d; ++j) {
            const size_t n1 = H.dir[j].n1, R = Nu0 / n1;
            ws = std::max(ws, ((n1 + 15) / 16 * 16) * ((R + 127) / 128 * 128));
            b += 4 * ((n1 + 15) / 16 * 16) * ((n1 + 255) / 256 * 256) * 4 + 4096;
        }
        b += 4 * ws * 4;
    }
    b += (kmax + 1) * Npsi * 8;                          // Krylov basis
    b += (kmax + 1) * kmax * 8 + (size_t)gmres_dot_blocks((long long)Npsi) * (kmax + 2) * 8 + (kmax + 2) * 8;
    if (P.params.strategy != HPG_SCHUR)                   // flexible GMRES on G: V, Z, partials
        b += (2 * kmax + 1) * Nx * 8 + (kmax + 1) * (size_t)fg_chunks((long long)Nx) * 8 + Npsi * 8;
    return b + (1u << 20);
}

static void worker_loop(Server* S, int w) {
    cudaSetDevice(S->ctx->device);
    hpg_ctx local;
    local.device = S->ctx->device;
    local.stream = S->streams[w];
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        Request* R = nullptr;
        S->cv_work.wait(lock, [&] {
            if (S->stopping) return true;
            for (Request* q : S->queue)
                if (S->in_use + q->bytes <= S->budget || S->charged.count(q->P)) return true;
            return false;
        });
        if (S->stopping && S->queue.empty()) return;
        // admission: the first request in arrival order that fits the memory budget, or
        // (policy 1) the largest one that fits, so that long solves start early and the
        // small ones fill the gaps
        auto pick = S->queue.end();
        for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
            Request* q = *it;
            const bool fits = S->charged.count(q->P) != 0 || S->in_use + q->bytes <= S->budget;
            if (!fits) continue;
            if (pick == S->queue.end()) {
                pick = it;
                if (S->policy == 0) break;
            } else if (request_work(*q->P) > request_work(*(*pick)->P)) {
                pick = it;
            }
        }
        if (pick != S->queue.end()) {
            Request* q = *pick;
            if (S->charged.count(q->P) == 0) {
                S->in_use += q->bytes;
                S->charged[q->P] = q->bytes;
            }
            R = q;
            S->queue.erase(pick);
        }
        if (!R) {
            if (S->stopping) return;
            continue;
        }
        R->state = 1;
        R->t_start = now_ms();
        lock.unlock();
        Problem& P = *R->P;
        P.host_result = false;
        hpg_status st = alloc_device(&local, P);
        if (st == HPG_OK) st = upload_data(&local, P);
        if (st == HPG_OK) st = solve_problem(&local, P);
        if (st != HPG_OK) P.stats.status = st;
        // keep the result on the host and hand the device memory back to the budget
        if (P.alloc_done) {
            P.host_x.resize(P.H.Nu0 + P.H.Npsi);
            if (cudaMemcpyAsync(P.host_x.data(), P.D.x, P.host_x.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                local.stream) == cudaSuccess &&
                cudaStreamSynchronize(local.stream) == cudaSuccess)
                P.host_result = P.solved;
            free_device(P, local.stream);
            P.data_dirty = P.phi_dirty = true;
        }
        lock.lock();
        auto ch = S->charged.find(R->P);
        if (ch != S->charged.end()) {
            S->in_use -= ch->second;
            S->charged.erase(ch);
        }
        R->result = st;
        if (st != HPG_OK) R->err = local.err.empty() ? std::string(hpg_status_str(st)) : local.err;
        R->t_done = now_ms();
        R->state = 2;
        R->P->busy = false;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

hpg_status server_start(hpg_ctx* ctx, int workers, size_t budget) {
    if (ctx->server) return HPG_ERR_STATE;
    auto* S = new Server();
    S->ctx = ctx;
    S->workers = workers;
    S->budget = budget;
    for (int w = 0; w < workers; ++w) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto s2 : S->streams) cudaStreamDestroy(s2);
            delete S;
            ctx->err = "stream creation failed";
            return HPG_ERR_CUDA;
        }
        S->streams.push_back(st);
    }
    for (int w = 0; w < workers; ++w) S->threads.emplace_back(worker_loop, S, w);
    ctx->server = S;
    return HPG_OK;
}

hpg_status server_stop(hpg_ctx* ctx) {
    Server* S = ctx->server;
    if (!S) return HPG_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->threads) t.join();
    for (auto st : S->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (auto& kv : S->reqs)
        if (kv.second.state != 2) kv.second.P->busy = false;
    delete S;
    ctx->server = nullptr;
    return HPG_OK;
}

hpg_status server_submit(hpg_ctx* ctx, Problem& P, long long* ticket) {
    Server* S = ctx->server;
    if (!S) return HPG_ERR_STATE;
    const size_t bytes = P.alloc_done ? P.D.bytes : estimate_device_bytes(P);
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) return HPG_ERR_STATE;
    if (bytes > S->budget) {
        ctx->err = "request larger than the device memory budget";
        return HPG_ERR_OOM;
    }
    Request& R = S->reqs[S->next_ticket];
    R.ticket = S->next_ticket++;
    R.P = &P;
    R.bytes = bytes;
    R.t_submit = now_ms();
    P.busy = true;
    S->queue.push_back(&R);
    *ticket = R.ticket;
    S->cv_work.notify_one();
    return HPG_OK;
}

hpg_status server_poll(hpg_ctx* ctx, long long ticket, double wait_ms, int* done, hpg_status* result,
                       double* times3) {
    Server* S = ctx->server;
    if (!S) return HPG_ERR_STATE;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return HPG_ERR_ARG;
    Request& R = it->second;
    if (wait_ms > 0 && R.state != 2) {
        const bool ok = S->cv_done.wait_for(lock, std::chrono::duration<double, std::milli>(wait_ms),
                                            [&] { return R.state == 2; });
        if (!ok) {
            if (done) *done = 0;
            return HPG_ERR_TIMEOUT;
        }
    }
    if (done) *done = R.state == 2 ? 1 : 0;
    if (result) *result = R.state == 2 ? R.result : HPG_OK;
    if (times3) {
        times3[0] = R.state >= 1 ? R.t_start - R.t_submit : now_ms() - R.t_submit;   // queued
        times3[1] = R.state == 2 ? R.t_done - R.t_start : 0.0;                          // running
        times3[2] = R.state == 2 ? R.t_done - R.t_submit : 0.0;                         // latency
    }
    return HPG_OK;
}

hpg_status server_set_policy(hpg_ctx* ctx, int policy) {
    Server* S = ctx->server;
    if (!S) return HPG_ERR_STATE;
    std::lock_guard<std::mutex> lock(S->mu);
    S->policy = policy;
    return HPG_OK;
}

hpg_status server_ticket_error(hpg_ctx* ctx, long long ticket, std::string* msg) {
    Server* S = ctx->server;
    if (!S) return HPG_ERR_STATE;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return HPG_ERR_ARG;
    *msg = it->second.state == 2 ? it->second.err : std::string();
    return HPG_OK;
}

// Called by hpg_problem_free: release the problem's budget charge.
void server_release(hpg_ctx* ctx, Problem& P) {
    Server* S = ctx->server;
    if (!S) return;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->charged.find(&P);
    if (it != S->charged.end()) {
        S->in_use -= it->second;
        S->charged.erase(it);
    }
    for (auto& kv : S->reqs)
        if (kv.second.P == &P) kv.second.P = nullptr;
    S->cv_work.notify_all();
}

size_t server_in_use(hpg_ctx* ctx) {
    Server* S = ctx->server;
    if (!S) return 0;
    std::lock_guard<std::mutex> lock(S->mu);
    return S->in_use;
}

}  // namespace hpg
