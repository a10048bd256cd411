// Allocation-free variant of the stiffness-inverse apply (A_alpha^{-1} by fast
// diagonalisation, FP64).  The two intermediate tensors of the GEMM passes live
// in a fixed file-scope device array instead of context-owned cudaMalloc
// buffers, so a call never allocates or frees device memory.
#include <cstdio>
#include <mutex>

#include "state.h"

namespace {

// Largest interior u vector (prod_j (m_j p - 1)) this entry point accepts.
constexpr size_t kNoAllocMaxInterior = 262144;

// Scratch shared by every call on a device: two tensors of kNoAllocMaxInterior
// doubles (4 MiB), resident on every GPU that loads the library until exit.
__device__ __align__(256) double g_fdm_scratch[2 * kNoAllocMaxInterior];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" hpg_status hpg_apply_stiffness_inv_noalloc(hpg_ctx* ctx, int pid, double alpha, const double* x_dev,
                                                      double* y_dev, size_t len) {
    if (!ctx || !x_dev || !y_dev || !(alpha > 0.0)) return HPG_ERR_ARG;
    auto it = ctx->problems.find(pid);
    if (it == ctx->problems.end()) return HPG_ERR_ARG;
    hpg::Problem& P = *it->second;
    if (P.busy.load()) {
        // a request-loop worker owns the problem and may release its device buffers
        ctx->err = "problem is queued or running in the request loop";
        return HPG_ERR_BUSY;
    }
    if (!P.alloc_done) {
        ctx->err = "problem operators are not on the device yet (solve or set a state first)";
        return HPG_ERR_STATE;
    }
    if (len < P.H.Nu0) return HPG_ERR_ARG;
    if (P.H.Nu0 > kNoAllocMaxInterior) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "hpg_apply_stiffness_inv_noalloc: %zu interior dofs exceed the limit of %zu",
                      (size_t)P.H.Nu0, kNoAllocMaxInterior);
        ctx->err = msg;
        return HPG_ERR_ARG;
    }
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return HPG_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return HPG_ERR_CUDA;
    void* base = nullptr;
    {
        // one-time set-up per device: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[ctx->device]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_fdm_scratch);
            if (e != cudaSuccess || !p) {
                ctx->err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return HPG_ERR_CUDA;
            }
            g_scratch_addr[ctx->device] = p;
        }
        base = g_scratch_addr[ctx->device];
    }
    double* w1 = static_cast<double*>(base);
    double* w2 = w1 + kNoAllocMaxInterior;
    const cudaError_t e = hpg::launch_fdm<double>(P.D.gd, nullptr, alpha, x_dev, y_dev, w1, w2, ctx->stream);
    if (e != cudaSuccess) {
        ctx->err = std::string("launch_fdm: ") + cudaGetErrorString(e);
        return HPG_ERR_CUDA;
    }
    return HPG_OK;
}
