// Thermoforming quasi-variational inequality (Section 6.4): the fixed point of an
// obstacle problem whose obstacle depends on a temperature T and a nonlinear heat
// equation for T, every step on the device.
//
//   (I)  given T_i, the obstacle problem u <= Phi_0 + xi T_i by hpG (the solver of this
//        library, its constraint written on the device at the latent Gauss points);
//   (II) given u_{i+1}, Newton on the T equation posed in all of U_{h,p} (no boundary
//        condition):
//          R(T) = (A + gamma M) T - (g(Phi_0 + xi T - u), phi) = 0,
//          J d  = (A + gamma M) d - (g'(s) xi d, phi),
//        each Newton system by GMRES right-preconditioned with (A + gamma M)^{-1}, applied
//        exactly by fast diagonalisation of the full-space 1D pencils (the paper factorises
//        A + gamma M by sparse Cholesky);
//   until ||u_{i+1} - u_i||_{H^1} <= tol.  g(s) = g_0 for s <= 0, g_0 (1 - s) on (0, 1),
//   0 for s >= 1; g' = -g_0 on (0, 1), 0 elsewhere.
// Integrals of the nonsmooth term use p + 2 Gauss points per direction per cell.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "state.h"

namespace hpg {

namespace {

// What the kernels need: the full U_{h,p} numbering (hats 0..m then bubbles cell-major
// per axis, x fastest), the 1D basis tables and the full 1D stencils.
struct QviGeo {
    int d, p;
    int m[kMaxDim], N1[kMaxDim];
    long long Nc, Nfull;
    int nq, nl;                 // T-step and latent points per direction per cell
    const double* Uq;           // (p+1) x nq, local functions at the T-step points
    const double* Ul;           // (p+1) x nl, at the latent points
    const double* Wref;         // nq^d weights times |J|
    const int* acnt[kMaxDim];
    const int* acol[kMaxDim];
    const double* aval[kMaxDim];
    const int* mcnt[kMaxDim];
    const int* mcol[kMaxDim];
    const double* mval[kMaxDim];
};

// full 1D index of local function a (0: left hat, 1: right hat, 2 + b: bubble b) of cell c
__device__ __forceinline__ int q_glob(int m, int p, int c, int a) {
    return a == 0 ? c : (a == 1 ? c + 1 : m + 1 + c * (p - 1) + (a - 2));
}

// one tensor pass along axis ax: out[.., r, ..] = sum_s W(r, s) in[.., s, ..] with
// W(r, s) = U[s * ld + r] (values: s a local function, r a point) or U[r * ld + s]
// (loads: r a local function, s a point); ext_in / ext_out the extents (x fastest)
__device__ void q_pass(const double* in, double* out, const double* U, int ld, bool values, const int* ext_in,
                       const int* ext_out, int d, int ax) {
    int tot = 1, sin = 1, sout = 1;
    for (int j = 0; j < d; ++j) tot *= ext_out[j];
    for (int j = 0; j < ax; ++j) { sin *= ext_in[j]; sout *= ext_out[j]; }
    const int nin = ext_in[ax], nout = ext_out[ax];
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int r = (e / sout) % nout;
        const int lo = e % sout, hi = e / (sout * nout);
        const int base = lo + hi * sin * nin;
        double acc = 0.0;
        for (int s2 = 0; s2 < nin; ++s2)
            acc += (values ? U[s2 * ld + r] : U[r * ld + s2]) * in[base + s2 * sin];
        out[e] = acc;
    }
}

// values of the full field coef at the tensor points of table U (np points per axis), per cell
__global__ void k_qvi_eval(QviGeo g, const double* __restrict__ coef, const double* __restrict__ U, int np,
                           double* __restrict__ out) {
    extern __shared__ double smq[];
    const int d = g.d, nl1 = g.p + 1;
    int mx = nl1 > np ? nl1 : np, cap = 1;
    for (int j = 0; j < d; ++j) cap *= mx;
    double* b0 = smq;
    double* b1 = smq + cap;
    const long long cell = blockIdx.x;
    int c[kMaxDim] = {0, 0, 0};
    long long e = cell;
    for (int j = 0; j < d; ++j) { c[j] = (int)(e % g.m[j]); e /= g.m[j]; }
    int nloc = 1;
    for (int j = 0; j < d; ++j) nloc *= nl1;
    for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
        long long I = 0, stride = 1;
        int rl = l;
        for (int j = 0; j < d; ++j) {
            const int a = rl % nl1;
            rl /= nl1;
            I += (long long)q_glob(g.m[j], g.p, c[j], a) * stride;
            stride *= g.N1[j];
        }
        b0[l] = coef[I];
    }
    __syncthreads();
    int ext[kMaxDim] = {1, 1, 1};
    for (int j = 0; j < d; ++j) ext[j] = nl1;
    double *in = b0, *o = b1;
    for (int ax = 0; ax < d; ++ax) {
        int eo[kMaxDim] = {ext[0], ext[1], ext[2]};
        eo[ax] = np;
        q_pass(in, o, U, np, true, ext, eo, d, ax);
        __syncthreads();
        ext[ax] = np;
        double* t = in; in = o; o = t;
    }
    int tot = 1;
    for (int j = 0; j < d; ++j) tot *= np;
    for (int l = threadIdx.x; l < tot; l += blockDim.x) out[cell * tot + l] = in[l];
}

// per cell, (v, phi_a) for every local function a from values v at the T-step points
__global__ void k_qvi_load(QviGeo g, const double* __restrict__ vals, double* __restrict__ Yc) {
    extern __shared__ double smq[];
    const int d = g.d, nl1 = g.p + 1, nq = g.nq;
    int mx = nl1 > nq ? nl1 : nq, cap = 1;
    for (int j = 0; j < d; ++j) cap *= mx;
    double* b0 = smq;
    double* b1 = smq + cap;
    const long long cell = blockIdx.x;
    int tot = 1;
    for (int j = 0; j < d; ++j) tot *= nq;
    for (int l = threadIdx.x; l < tot; l += blockDim.x) b0[l] = vals[cell * tot + l];
    __syncthreads();
    int ext[kMaxDim] = {1, 1, 1};
    for (int j = 0; j < d; ++j) ext[j] = nq;
    double *in = b0, *o = b1;
    for (int ax = 0; ax < d; ++ax) {
        int eo[kMaxDim] = {ext[0], ext[1], ext[2]};
        eo[ax] = nl1;
        q_pass(in, o, g.Uq, nq, false, ext, eo, d, ax);
        __syncthreads();
        ext[ax] = nl1;
        double* t = in; in = o; o = t;
    }
    int nloc = 1;
    for (int j = 0; j < d; ++j) nloc *= nl1;
    for (int l = threadIdx.x; l < nloc; l += blockDim.x) Yc[cell * nloc + l] = in[l];
}

// every full dof sums its cells' local loads (at most 2^d, in a fixed order)
__global__ void k_qvi_gather(QviGeo g, const double* __restrict__ Yc, double* __restrict__ out) {
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= g.Nfull) return;
    const int nl1 = g.p + 1;
    int cc[kMaxDim][2], aa[kMaxDim][2], nch[kMaxDim];
    long long e = I;
    for (int j = 0; j < g.d; ++j) {
        const int i = (int)(e % g.N1[j]);
        e /= g.N1[j];
        const int m = g.m[j];
        nch[j] = 0;
        if (i <= m) {
            if (i >= 1) { cc[j][nch[j]] = i - 1; aa[j][nch[j]] = 1; ++nch[j]; }
            if (i <= m - 1) { cc[j][nch[j]] = i; aa[j][nch[j]] = 0; ++nch[j]; }
        } else {
            const int b = i - (m + 1);
            cc[j][0] = b / (g.p - 1);
            aa[j][0] = 2 + b % (g.p - 1);
            nch[j] = 1;
        }
    }
    long long nloc = 1;
    for (int j = 0; j < g.d; ++j) nloc *= nl1;
    double acc = 0.0;
    for (int sel = 0; sel < (1 << g.d); ++sel) {
        bool ok = true;
        long long cell = 0, cs = 1, l = 0, ls = 1;
        for (int j = 0; j < g.d; ++j) {
            const int bj = (sel >> j) & 1;
            if (bj >= nch[j]) { ok = false; break; }
            cell += (long long)cc[j][bj] * cs;
            cs *= g.m[j];
            l += (long long)aa[j][bj] * ls;
            ls *= nl1;
        }
        if (ok) acc += Yc[cell * nloc + l];
    }
    out[I] = acc;
}

// y = (A + gamma M) x on the full space: A = sum_k (x)_j (j == k ? A_j : M_j), M = (x)_j M_j
__device__ __forceinline__ double q_term(const QviGeo& g, const int* idx, const bool* useA, const double* x) {
    // sum over the tensor stencil prod_j S_j[idx_j], S_j = A_j if useA[j] else M_j
    const int d = g.d;
    const int* cnt[kMaxDim];
    const int* col[kMaxDim];
    const double* val[kMaxDim];
    for (int j = 0; j < d; ++j) {
        cnt[j] = useA[j] ? g.acnt[j] : g.mcnt[j];
        col[j] = useA[j] ? g.acol[j] : g.mcol[j];
        val[j] = useA[j] ? g.aval[j] : g.mval[j];
    }
    double s = 0.0;
    const int c0 = cnt[0][idx[0]], c1 = cnt[1][idx[1]];
    const int c2 = d == 3 ? cnt[2][idx[2]] : 1;
    for (int e2 = 0; e2 < c2; ++e2) {
        long long b2 = 0;
        double v2 = 1.0;
        if (d == 3) {
            b2 = (long long)col[2][(size_t)idx[2] * kEll + e2] * g.N1[1];
            v2 = val[2][(size_t)idx[2] * kEll + e2];
        }
        double t2 = 0.0;
        for (int e1 = 0; e1 < c1; ++e1) {
            const long long base = (b2 + col[1][(size_t)idx[1] * kEll + e1]) * g.N1[0];
            double t = 0.0;
            for (int e0 = 0; e0 < c0; ++e0)
                t += val[0][(size_t)idx[0] * kEll + e0] * x[base + col[0][(size_t)idx[0] * kEll + e0]];
            t2 += val[1][(size_t)idx[1] * kEll + e1] * t;
        }
        s += v2 * t2;
    }
    return s;
}

__global__ void k_qvi_kron(QviGeo g, double gamma, const double* __restrict__ x, double* __restrict__ y) {
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= g.Nfull) return;
    int idx[kMaxDim] = {0, 0, 0};
    long long e = I;
    for (int j = 0; j < g.d; ++j) { idx[j] = (int)(e % g.N1[j]); e /= g.N1[j]; }
    double acc = 0.0;
    for (int k = 0; k < g.d; ++k) {
        bool useA[kMaxDim] = {false, false, false};
        useA[k] = true;
        acc += q_term(g, idx, useA, x);
    }
    const bool none[kMaxDim] = {false, false, false};
    acc += gamma * q_term(g, idx, none, x);
    y[I] = acc;
}

// mode 0: w = W g(s); mode 1: w = W g'(s) xi; s = Phi_0 + xi T - u at the T-step points
__global__ void k_qvi_point(QviGeo g, int mode, double g0, const double* __restrict__ Tq, const double* __restrict__ uq,
                            const double* __restrict__ Phi0, const double* __restrict__ xi, double* __restrict__ w,
                            long long n, int per) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = Phi0[i] + xi[i] * Tq[i] - uq[i];
    const double W = g.Wref[i % per];
    if (mode == 0) w[i] = W * (s <= 0.0 ? g0 : (s < 1.0 ? g0 * (1.0 - s) : 0.0));
    else w[i] = (s > 0.0 && s < 1.0) ? -W * g0 * xi[i] : 0.0;
}

__global__ void k_qvi_mul(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c,
                          long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] * b[i];
}

// phiq = Phi_0 + xi T at the latent points
__global__ void k_qvi_latent(const double* __restrict__ Tl, const double* __restrict__ Phi0, const double* __restrict__ xi,
                             double* __restrict__ phiq, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) phiq[i] = Phi0[i] + xi[i] * Tl[i];
}

// full u = interior u scattered (homogeneous Dirichlet data: boundary entries 0)
__global__ void k_qvi_int_to_full(QviGeo g, const double* __restrict__ x, double* __restrict__ u, long long n0) {
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n0) return;
    long long e = I, full = 0, stride = 1;
    for (int j = 0; j < g.d; ++j) {
        const int n1 = g.m[j] * g.p - 1;
        const int i = (int)(e % n1);
        e /= n1;
        const int gi = i < g.m[j] - 1 ? i + 1 : g.m[j] + 1 + (i - (g.m[j] - 1));
        full += (long long)gi * stride;
        stride *= g.N1[j];
    }
    u[full] = x[I];
}

inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

// device allocations of one QVI solve, released (stream-ordered) when it returns
struct Arena {
    cudaStream_t s;
    std::vector<void*> ptrs;
    bool ok = true;
    explicit Arena(cudaStream_t st) : s(st) {}
    template <typename T>
    T* get(size_t n) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), s) != cudaSuccess) { ok = false; return nullptr; }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    template <typename T>
    T* up(const T* v, size_t n) {
        T* p = get<T>(n);
        if (p && n && cudaMemcpyAsync(p, v, n * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess) ok = false;
        return p;
    }
    ~Arena() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

// local 1D functions [hatL, hatR, W_0 .. W_{p-2}] at the points y: U[a * ny + q]
void local_table(int p, const std::vector<double>& y, std::vector<double>& U) {
    const int ny = (int)y.size();
    U.assign((size_t)(p + 1) * ny, 0.0);
    std::vector<double> Pl(p + 3), dPl(p + 3);
    for (int q = 0; q < ny; ++q) {
        legendre_all(p + 1, y[q], Pl.data(), dPl.data());
        U[0 * ny + q] = 0.5 * (1.0 - y[q]);
        U[1 * ny + q] = 0.5 * (1.0 + y[q]);
        for (int b = 0; b + 2 <= p; ++b) U[(size_t)(2 + b) * ny + q] = (Pl[b] - Pl[b + 2]) / (2 * b + 3);
    }
}

// Everything one QVI solve holds on the device, with its operations.
struct QviRun {
    hpg_ctx* ctx;
    cudaStream_t s;
    QviGeo g{};
    Geo<double> gfdm{};          // the problem's FP64 view with the full-space pencils
    long long N = 0, Nq = 0, Nl = 0;
    size_t smem_q = 0, smem_l = 0;
    double gamma = 1.0, g0 = 0.2;
    int nqd = 1;
    // fields and scratch (N each unless noted)
    double *T, *uf, *up, *R, *dl, *t1, *t2, *w1, *w2, *lift;
    double *Tq, *uq, *phi0q, *xiq, *wq, *wd, *vq, *Yc;    // Nq (Yc: Nc (p+1)^d)
    double *Tl, *phi0l, *xil;                            // Nl
    double *V = nullptr, *part = nullptr, *hd = nullptr; // GMRES basis (kmax+1) N, partials, coefficients
    int kmax = 0;

    cudaError_t post() {
        note_kernel_launches(1);
        return cudaGetLastError();
    }
    cudaError_t eval(const double* coef, const double* U, int np, double* out, size_t smem) {
        k_qvi_eval<<<(unsigned)g.Nc, 128, smem, s>>>(g, coef, U, np, out);
        return post();
    }
    // out = (v, phi_i) for the weighted values v at the T-step points
    cudaError_t load(const double* v, double* out) {
        k_qvi_load<<<(unsigned)g.Nc, 128, smem_q, s>>>(g, v, Yc);
        cudaError_t e = post();
        if (e != cudaSuccess) return e;
        k_qvi_gather<<<nblk(N), 256, 0, s>>>(g, Yc, out);
        return post();
    }
    cudaError_t kron(double gm, const double* x, double* y) {
        k_qvi_kron<<<nblk(N), 256, 0, s>>>(g, gm, x, y);
        return post();
    }
    // (A + gamma M)^{-1} x by fast diagonalisation of the full-space pencils
    cudaError_t kinv(const double* x, double* y) {
        cudaError_t e = launch_fdm<double>(gfdm, nullptr, 1.0, x, y, w1, w2, s, nullptr, Bat{}, gamma);
        return e;
    }
    // sum of the partial dot products of a and b, on the host
    hpg_status dot(const double* a, const double* b, double* out) {
        int np = 0;
        cudaError_t e = launch_dot(a, b, N, part, &np, s);
        std::vector<double> h((size_t)np);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, np * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { ctx->err = std::string("QVI dot: ") + cudaGetErrorString(e); return HPG_ERR_CUDA; }
        double acc = 0.0;
        for (double v : h) acc += v;
        *out = acc;
        return HPG_OK;
    }
    // R = (A + gamma M) T - (g(Phi_0 + xi T - u), phi); leaves T at the points in Tq
    hpg_status residual(double* norm) {
        cudaError_t e = eval(T, g.Uq, g.nq, Tq, smem_q);
        if (e == cudaSuccess) {
            k_qvi_point<<<nblk(Nq), 256, 0, s>>>(g, 0, g0, Tq, uq, phi0q, xiq, wq, Nq, nqd);
            e = post();
        }
        if (e == cudaSuccess) e = load(wq, t1);
        if (e == cudaSuccess) e = kron(gamma, T, R);
        if (e == cudaSuccess) e = launch_axpby(-1.0, t1, 1.0, R, N, s);
        if (e != cudaSuccess) { ctx->err = std::string("QVI residual: ") + cudaGetErrorString(e); return HPG_ERR_CUDA; }
        double n2 = 0.0;
        hpg_status st = dot(R, R, &n2);
        *norm = std::sqrt(std::max(n2, 0.0));
        return st;
    }
    // y = J x = (A + gamma M) x - (g'(s) xi x, phi), weights W g' xi in wd
    cudaError_t jac(const double* x, double* y) {
        cudaError_t e = eval(x, g.Uq, g.nq, vq, smem_q);
        if (e != cudaSuccess) return e;
        k_qvi_mul<<<nblk(Nq), 256, 0, s>>>(wd, vq, vq, Nq);
        if ((e = post()) != cudaSuccess) return e;
        if ((e = load(vq, t2)) != cudaSuccess) return e;
        if ((e = kron(gamma, x, y)) != cudaSuccess) return e;
        return launch_axpby(-1.0, t2, 1.0, y, N, s);
    }
    // GMRES on J z = b right-preconditioned by (A + gamma M)^{-1}, classical Gram-Schmidt
    // with one re-orthogonalisation (FP64), Givens rotations on the host
    hpg_status gmres(const double* b, double* z, double rtol, int* its) {
        *its = 0;
        double beta2 = 0.0;
        hpg_status st = dot(b, b, &beta2);
        if (st != HPG_OK) return st;
        const double beta = std::sqrt(std::max(beta2, 0.0));
        cudaError_t e = cudaMemsetAsync(z, 0, N * sizeof(double), s);
        if (e != cudaSuccess || !(beta > 0.0)) return e == cudaSuccess ? HPG_OK : HPG_ERR_CUDA;
        const int m = kmax, nch = fg_chunks(N);
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1, 0.0), hp((size_t)(m + 1) * nch),
            h(m + 1);
        gv[0] = beta;
        auto fail = [&](cudaError_t ce) {
            ctx->err = std::string("QVI GMRES: ") + cudaGetErrorString(ce);
            return HPG_ERR_CUDA;
        };
        if ((e = launch_axpby(1.0 / beta, b, 0.0, V, N, s)) != cudaSuccess) return fail(e);
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* w = V + (long long)(j + 1) * N;
            if ((e = kinv(V + (long long)j * N, t1)) != cudaSuccess) return fail(e);
            if ((e = jac(t1, w)) != cudaSuccess) return fail(e);
            double* col = H.data() + (size_t)j * (m + 1);
            for (int pass = 0; pass < 2; ++pass) {
                if ((e = launch_mdot(V, N, j + 1, w, N, part, s)) != cudaSuccess) return fail(e);
                if ((e = cudaMemcpyAsync(hp.data(), part, (size_t)(j + 1) * nch * sizeof(double),
                                         cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                    return fail(e);
                if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
                for (int v = 0; v <= j; ++v) {
                    double a = 0.0;
                    for (int c = 0; c < nch; ++c) a += hp[(size_t)v * nch + c];
                    h[v] = a;
                    col[v] += a;
                }
                if ((e = cudaMemcpyAsync(hd, h.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess)
                    return fail(e);
                if ((e = launch_maxpy(w, V, N, hd, j + 1, N, -1.0, s)) != cudaSuccess) return fail(e);
            }
            double hn2 = 0.0;
            if ((st = dot(w, w, &hn2)) != HPG_OK) return st;
            const double hn = std::sqrt(std::max(hn2, 0.0));
            col[j + 1] = hn;
            if (hn > 0.0 && (e = launch_axpby(1.0 / hn, w, 0.0, w, N, s)) != cudaSuccess) return fail(e);
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
        std::vector<double> y(k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            double t = gv[i];
            for (int l = i + 1; l < k; ++l) t -= H[(size_t)l * (m + 1) + i] * y[l];
            const double dg = H[(size_t)i * (m + 1) + i];
            y[i] = dg != 0.0 ? t / dg : 0.0;
        }
        // z = K^{-1} (V y)
        if ((e = cudaMemsetAsync(t1, 0, N * sizeof(double), s)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpyAsync(hd, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return fail(e);
        if ((e = launch_maxpy(t1, V, N, hd, k, N, 1.0, s)) != cudaSuccess) return fail(e);
        if ((e = kinv(t1, z)) != cudaSuccess) return fail(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
        return HPG_OK;
    }
};

}  // namespace

void qvi_points(const HostProblem& H, int nq, std::vector<double>& pts) {
    const int d = H.d;
    std::vector<double> y, w;
    gauss_legendre(nq, y, w);
    long long per = 1;
    for (int j = 0; j < d; ++j) per *= nq;
    pts.assign((size_t)H.Nc * per * d, 0.0);
    for (size_t c = 0; c < H.Nc; ++c) {
        int cm[kMaxDim] = {0, 0, 0};
        size_t cc = c;
        for (int j = 0; j < d; ++j) { cm[j] = (int)(cc % H.m[j]); cc /= H.m[j]; }
        for (long long q = 0; q < per; ++q) {
            long long qq = q;
            for (int j = 0; j < d; ++j) {
                const int qi = (int)(qq % nq);
                qq /= nq;
                pts[((size_t)c * per + q) * d + j] = H.lo[j] + (cm[j] + 0.5 * (y[qi] + 1.0)) * H.h[j];
            }
        }
    }
}

#define QCK(...)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (__VA_ARGS__);                                                      \
        if (e_ != cudaSuccess) {                                                             \
            ctx->err = std::string("QVI: ") + #__VA_ARGS__ + ": " + cudaGetErrorString(e_);  \
            return HPG_ERR_CUDA;                                                             \
        }                                                                                    \
    } while (0)

hpg_status qvi_solve(hpg_ctx* ctx, Problem& P, const hpg_qvi_params& q, const double* phi0_lat, const double* xi_lat,
                     const double* phi0_q, const double* xi_q, hpg_qvi_stats* out) {
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = kernel_launch_count();
    HostProblem& H = P.H;
    const int d = H.d, p = H.p, nq = q.nq > 0 ? q.nq : p + 2, n = H.n;
    hpg_qvi_stats st{};
    cudaStream_t s = ctx->stream;
    // the first obstacle: Phi_0 + xi T_0 = Phi_0 at the latent points
    H.phiq.assign(phi0_lat, phi0_lat + H.Nq);
    H.has_phi = true;
    P.phi_dirty = true;
    hpg_status rs = alloc_device(ctx, P);
    if (rs != HPG_OK) return rs;
    if ((rs = upload_data(ctx, P)) != HPG_OK) return rs;
    // until the end the device constraint differs from H.phiq: a failed solve leaves the
    // next hpg_solve to upload Phi_0 again
    P.phi_dirty = true;
    DevState& D = P.D;

    Arena ar(s);
    QviRun r{};
    r.ctx = ctx;
    r.s = s;
    r.gamma = q.gamma;
    r.g0 = q.g0;
    QviGeo& g = r.g;
    g.d = d;
    g.p = p;
    g.Nc = (long long)H.Nc;
    g.Nfull = (long long)H.Nu_full;
    g.nq = nq;
    g.nl = n;
    r.N = g.Nfull;
    r.nqd = 1;
    int nld = 1, nloc1 = 1;
    for (int j = 0; j < d; ++j) { r.nqd *= nq; nld *= n; nloc1 *= p + 1; }
    r.Nq = g.Nc * r.nqd;
    r.Nl = g.Nc * nld;
    {
        size_t capq = 1, capl = 1;
        for (int j = 0; j < d; ++j) { capq *= (size_t)std::max(p + 1, nq); capl *= (size_t)std::max(p + 1, n); }
        r.smem_q = 2 * capq * sizeof(double);
        r.smem_l = 2 * capl * sizeof(double);
    }
    // tables: local functions at the T-step points and at the latent points, weights
    std::vector<double> yq, wq1, Uq, Ul;
    gauss_legendre(nq, yq, wq1);
    local_table(p, yq, Uq);
    local_table(p, H.yq, Ul);
    std::vector<double> Wref((size_t)r.nqd);
    for (int l = 0; l < r.nqd; ++l) {
        double w = H.detJ;
        int ll = l;
        for (int j = 0; j < d; ++j) { w *= wq1[ll % nq]; ll /= nq; }
        Wref[l] = w;
    }
    g.Uq = ar.up(Uq.data(), Uq.size());
    g.Ul = ar.up(Ul.data(), Ul.size());
    g.Wref = ar.up(Wref.data(), Wref.size());
    // full-space 1D stencils and pencils (A_j + shift M_j diagonalised with V_j^T M_j V_j = I)
    std::vector<double> Vj[kMaxDim], lamj[kMaxDim];
    r.gfdm = D.gd;
    for (int j = 0; j < d; ++j) {
        const Dir1D& Dj = H.dir[j];
        g.m[j] = Dj.m;
        g.N1[j] = Dj.N1;
        g.acnt[j] = ar.up(Dj.A.cnt.data(), Dj.A.cnt.size());
        g.acol[j] = ar.up(Dj.A.col.data(), Dj.A.col.size());
        g.aval[j] = ar.up(Dj.A.val.data(), Dj.A.val.size());
        g.mcnt[j] = ar.up(Dj.M.cnt.data(), Dj.M.cnt.size());
        g.mcol[j] = ar.up(Dj.M.col.data(), Dj.M.col.size());
        g.mval[j] = ar.up(Dj.M.val.data(), Dj.M.val.size());
        const int N1 = Dj.N1;
        std::vector<double> Ad((size_t)N1 * N1, 0.0), Md((size_t)N1 * N1, 0.0);
        for (int i = 0; i < N1; ++i) {
            for (int e = 0; e < Dj.A.cnt[i]; ++e)
                Ad[(size_t)i * N1 + Dj.A.col[(size_t)i * kEll + e]] += Dj.A.val[(size_t)i * kEll + e];
            for (int e = 0; e < Dj.M.cnt[i]; ++e)
                Md[(size_t)i * N1 + Dj.M.col[(size_t)i * kEll + e]] += Dj.M.val[(size_t)i * kEll + e];
        }
        pencil_eigen(N1, Ad, Md, Vj[j], lamj[j]);
        r.gfdm.n1[j] = N1;
        r.gfdm.V[j] = ar.up(Vj[j].data(), Vj[j].size());
        r.gfdm.VT[j] = nullptr;
        r.gfdm.lam[j] = ar.up(lamj[j].data(), lamj[j].size());
    }
    // data and state
    r.phi0q = ar.up(phi0_q, (size_t)r.Nq);
    r.xiq = ar.up(xi_q, (size_t)r.Nq);
    r.phi0l = ar.up(phi0_lat, (size_t)r.Nl);
    r.xil = ar.up(xi_lat, (size_t)r.Nl);
    r.lift = ar.up(H.ulift.data(), H.ulift.size());
    const long long N = r.N;
    double** vecs[] = {&r.T, &r.uf, &r.up, &r.R, &r.dl, &r.t1, &r.t2, &r.w1, &r.w2};
    for (double** v : vecs) *v = ar.get<double>((size_t)N);
    double** qv[] = {&r.Tq, &r.uq, &r.wq, &r.wd, &r.vq};
    for (double** v : qv) *v = ar.get<double>((size_t)r.Nq);
    r.Yc = ar.get<double>((size_t)g.Nc * nloc1);
    r.Tl = ar.get<double>((size_t)r.Nl);
    r.kmax = std::max(1, q.t_krylov_max);
    r.V = ar.get<double>((size_t)(r.kmax + 1) * N);
    r.part = ar.get<double>((size_t)std::max<long long>((long long)(r.kmax + 1) * fg_chunks(N), 1024));
    r.hd = ar.get<double>((size_t)r.kmax + 1);
    if (!ar.ok) { ctx->err = "QVI: device allocation or upload failed"; return HPG_ERR_OOM; }
    QCK(cudaFuncSetAttribute(k_qvi_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCellSmemMax));
    QCK(cudaFuncSetAttribute(k_qvi_load, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCellSmemMax));
    QCK(cudaMemsetAsync(r.T, 0, N * sizeof(double), s));
    QCK(cudaStreamSynchronize(s));   // host tables above are released on return

    hpg_status status = HPG_OK;
    double tres = 0.0;
    for (int it = 0; it < q.max_fp; ++it) {
        // (I) obstacle Phi_0 + xi T_i at the latent points, then (phi, zeta) and the hpG solve
        QCK(r.eval(r.T, g.Ul, n, r.Tl, r.smem_l));
        k_qvi_latent<<<nblk(r.Nl), 256, 0, s>>>(r.Tl, r.phi0l, r.xil, D.phiq, r.Nl);
        QCK(r.post());
        QCK(launch_project(D.gd, D.phiq, D.phiz, s));
        hpg_status os = solve_problem(ctx, P);
        st.newton_total += P.stats.newton_total;
        st.krylov_total += P.stats.krylov_total;
        st.newton_per_fp[it] = P.stats.newton_total;
        if (os != HPG_OK) {
            ctx->err = "QVI iteration " + std::to_string(it + 1) + ", obstacle step: " + ctx->err;
            status = os;
            st.iterations = it + 1;
            break;
        }
        // u_{i+1} in the full numbering (lifting + interior coefficients)
        QCK(launch_copy<double>(r.lift, r.uf, N, s));
        k_qvi_int_to_full<<<nblk((long long)H.Nu0), 256, 0, s>>>(g, D.x, r.uf, (long long)H.Nu0);
        QCK(r.post());
        QCK(r.eval(r.uf, g.Uq, nq, r.uq, r.smem_q));
        // (II) Newton on the T equation from T_i
        hpg_status ts = r.residual(&tres);
        if (ts != HPG_OK) return ts;
        int tn = 0;
        while (tres > q.t_tol && tn < q.t_newton_max) {
            k_qvi_point<<<nblk(r.Nq), 256, 0, s>>>(g, 1, r.g0, r.Tq, r.uq, r.phi0q, r.xiq, r.wd, r.Nq, r.nqd);
            QCK(r.post());
            int its = 0;
            if ((ts = r.gmres(r.R, r.dl, q.t_krylov_rtol, &its)) != HPG_OK) return ts;
            st.t_krylov_total += its;
            QCK(launch_axpby(-1.0, r.dl, 1.0, r.T, N, s));
            if ((ts = r.residual(&tres)) != HPG_OK) return ts;
            ++tn;
        }
        st.t_newton_total += tn;
        st.t_newton_per_fp[it] = tn;
        st.iterations = it + 1;
        if (!(tres <= q.t_tol)) {
            status = HPG_ERR_NEWTON_CAP;
            ctx->err = "QVI iteration " + std::to_string(it + 1) + ": temperature Newton stopped at ||R|| = " +
                       std::to_string(tres);
            break;
        }
        // ||u_{i+1} - u_i||_{H^1}^2 = e^T (A + M) e
        if (it > 0) {
            QCK(launch_axpby(1.0, r.uf, -1.0, r.up, N, s));   // up = u_{i+1} - u_i
            QCK(r.kron(1.0, r.up, r.t2));
            double h2 = 0.0;
            if ((ts = r.dot(r.up, r.t2, &h2)) != HPG_OK) return ts;
            st.du_h1[it] = std::sqrt(std::max(h2, 0.0));
        }
        QCK(launch_copy<double>(r.uf, r.up, N, s));
        if (it > 0 && st.du_h1[it] <= q.tol) { st.converged = 1; break; }
    }
    if (status == HPG_OK && !st.converged) {
        status = HPG_ERR_NEWTON_CAP;
        ctx->err = "QVI fixed point did not reach the H^1 tolerance in " + std::to_string(q.max_fp) + " iterations";
    }
    // keep T and the last obstacle on the host
    P.qvi_T.assign((size_t)N, 0.0);
    QCK(cudaMemcpyAsync(P.qvi_T.data(), r.T, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    QCK(cudaMemcpyAsync(H.phiq.data(), D.phiq, H.Nq * sizeof(double), cudaMemcpyDeviceToHost, s));
    QCK(cudaStreamSynchronize(s));
    P.phi_dirty = false;
    st.status = status;
    st.t_residual = tres;
    st.kernel_launches = kernel_launch_count() - launches0;
    st.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (out) *out = st;
    return status;
}

}  // namespace hpg
