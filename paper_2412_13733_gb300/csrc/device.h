// Device-side views of a problem and the kernel launchers of libhpg.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>

#include "hpg_internal.h"

namespace hpg {

// A 1D operator in padded-ELL form (kEll entries per row; cnt[r] used).
// For Gram operators the column packs (cell << 8) | k.
template <typename T>
struct Sten {
    const int* cnt;
    const int* col;
    const T* val;
    const int* lcol;   // column as a position in the row tile's column list (TileCols), or null
};

// Columns referenced by the rows of each row tile of one axis (tiles of the tiled
// u-row kernels): count[t] sorted entries at list[t * cap].  The u-row kernels stage
// the values at these columns (a box per tile) in shared memory before the gathers.
struct TileCols {
    const int* list;
    const int* count;
    int cap;
};

// Row-tile extent of the tiled u-row kernels along axis `axis` for dimension d.
int utile_extent(int d, int axis);
template <typename T>
struct Geo;
// Whether the value boxes of the tiled u-row kernels fit their shared-memory budget.
template <typename T>
bool urow_boxes_fit(const Geo<T>& g);

struct FdmTma;

// Everything a kernel needs to know about one problem, for compute type T.
template <typename T>
struct Geo {
    int d, n, ncomp, kind;
    int m[kMaxDim], n1[kMaxDim];
    long long Nu0, Nc, nloc, nb, Npsi;
    Sten<T> A[kMaxDim], M[kMaxDim];          // interior x interior
    Sten<T> B[kMaxDim], BT[kMaxDim];         // interior -> psi-1D, psi-1D -> interior
    Sten<T> Bd[kMaxDim], BdT[kMaxDim];       // derivative Gram (gradient kind)
    const T* Vq;                              // n x n : P_k(y_q)
    const T* wq;                              // n
    T detJ;
    const T* Mpsi;                            // nloc (one component)
    const T* Kpsi;                            // nloc x nloc (gradient E_beta)
    const T* C;                               // nloc x nloc (obstacle S-hat constant part)
    const T* V[kMaxDim];                      // n1 x n1 fast-diagonalisation eigenvectors
    const T* VT[kMaxDim];                     // their transposes VT[a][k] = V[k][a] (or null): the
                                              // forward passes along the outer axes read V^T K-contiguous
    const T* lam[kMaxDim];                    // n1 eigenvalues
    int gemm_cfg;                             // tile variant of the FDM passes (autotuned)
    TileCols tu[kMaxDim];                     // u columns of the A, M stencils per row tile
    TileCols tp[kMaxDim];                     // psi columns (packed) of the B, Bd stencils
    int staged;                               // 1: the u-row kernels stage value boxes in shared memory
    const int* perm0;                         // n1[0] rows of axis 0 in the order the unstaged u-row
                                              // tiles take them (sorted by stencil counts), or null
    const FdmTma* tma;                        // host view of the TMA/tcgen05 fast diagonalisation (FP32), or null
};

// Lockstep group of same-shape problems (identical mesh, degree, kind and operator
// constants): one launch serves every problem of the group.  Each problem keeps its
// per-problem buffers (state, data, Krylov basis, factors) in one slab laid out
// identically for all of them, so problem pb's copy of a buffer is problem 0's
// pointer moved by delta[pb] bytes; the constant operators (stencils, eigenvectors,
// quadrature) are read from problem 0.  The launch gives the problem index its own
// grid coordinate; `act` (device, np flags, may be null) masks problems out of a
// launch.  Bat{} (np = 1, no delta) is a single problem: every kernel then does
// exactly what it does without batching.
struct Bat {
    const long long* delta = nullptr;   // device, np byte offsets (delta[0] = 0)
    const int* act = nullptr;           // device, np flags (1: problem takes part)
    const double* par = nullptr;        // device, np x kBatPar per-problem scalars (see BatPar)
    int np = 1;
};
// per-problem scalars a batched launch reads from Bat::par instead of an argument
enum BatPar { kParLam = 0, kParRtol = 1, kParAlpha = 2, kBatPar = 4 };

#ifdef __CUDACC__
// problem index of this block (the launch's problem grid coordinate) -> byte offset;
// returns false when the problem is masked out (the whole block returns)
__device__ __forceinline__ bool bat_enter(const Bat& bt, int pb, long long* off) {
    if (bt.act && !bt.act[pb]) return false;
    *off = bt.delta ? bt.delta[pb] : 0LL;
    return true;
}
template <typename P>
__device__ __forceinline__ P* bsh(P* p, long long off) {
    return p ? reinterpret_cast<P*>(reinterpret_cast<char*>(const_cast<void*>(static_cast<const void*>(p))) + off)
             : p;
}
#endif

// Number of values stored per Gauss point by the evaluation kernel:
// obstacle: 1 (w |J| exp(-psi)); gradient: packed symmetric d x d Jacobian * w|J|.
inline int gauss_stride(int kind, int d) { return kind == HPG_GRADIENT ? d * (d + 1) / 2 : 1; }

// Device-side loop control for kernels replayed inside a captured GMRES chunk:
// `skip` (non-null) makes the kernel return when *skip != 0; `jptr` offsets an
// input (precond) or output (cell operator) by (*jptr [+1]) * jstride.
struct IterCtl {
    const int* skip = nullptr;
    const int* jptr = nullptr;
    long long jstride = 0;
};

// ------------------------------------------------------------ launchers
// Each launcher enqueues on `s` and returns the CUDA error of the launch.

// Latent nonlinearity at Gauss points: gw (FP64, Nc*nloc*gstride), gwf (FP32
// copy, may be null), eg = projection onto zeta (FP64, Npsi), flag |= 1 on
// psi < -700 (obstacle) or non-finite values.
cudaError_t launch_eval(const Geo<double>& g, const double* psi, const double* phiq, double* gw, float* gwf,
                        double* eg, int* flag, cudaStream_t s, const Bat& bt = Bat{});

// phiz = (phi, zeta) from phi at the latent Gauss points (obstacle kinds).
cudaError_t launch_project(const Geo<double>& g, const double* phiq, double* phiz, cudaStream_t s);
// Number of kernels launched (or replayed in graphs) by this library from the calling
// host thread since it started.
long long kernel_launch_count();
// Add n kernels launched by another translation unit of the library to that count.
void note_kernel_launches(long long n);
void add_kernel_launches(long long n);

// F_u = alpha A u + alpha rA + B (psi - psi_prev) - alpha bf;  F_psi = B^T u + rB + sgn*eg - phiz.
// Writes F (Nu0 + Npsi) and block partial sums of squares into part (see n_res_partials).
cudaError_t launch_residual(const Geo<double>& g, const double* u, const double* psi, const double* psi_prev,
                            const double* eg, const double* rA, const double* rB, const double* bf,
                            const double* phiz, double alpha, double* F, double* part, cudaStream_t s,
                            const Bat& bt = Bat{});
int n_res_partials(const Geo<double>& g);
int n_res_partials_for(int d, const int* n1, long long Npsi);

// Deterministic reduction of `count` partials into out[0] (one block).
cudaError_t launch_reduce_sum(const double* part, int count, double* out, cudaStream_t s, const Bat& bt = Bat{});

// Assemble -S-hat cell blocks, Cholesky, invert: Sinv (Nc x nb x nb, precision T)
// holds (-S-hat)^{-1}.  If `dump` is non-null the assembled -S-hat blocks are written there.
// gwork: global workspace of factor_workspace_elems() elements (null when that is 0).
template <typename T>
cudaError_t launch_factor(const Geo<T>& g, const T* gw, double alpha, double beta, T* Sinv, double* dump,
                          int* flag, T* gwork, cudaStream_t s, const Bat& bt = Bat{});
size_t factor_smem_bytes(int nb, int elem);
size_t factor_workspace_elems(int n, int d, int nb, int nc, long long Nc, int elem);

// z = -Sinv v (per cell), in/out precision mixing: v (Tin), z (Tout).
template <typename T, typename Tin, typename Tout>
cudaError_t launch_precond(const Geo<T>& g, const T* Sinv, const Tin* v, Tout* z, cudaStream_t s,
                           IterCtl ctl = IterCtl{}, const Bat& bt = Bat{});

// y = B z  (psi -> interior u);  Tin/Tout storage, T compute.
template <typename T, typename Tin, typename Tout>
cudaError_t launch_bapply(const Geo<T>& g, const Tin* z, Tout* y, cudaStream_t s, const int* skip = nullptr,
                          const Bat& bt = Bat{});

// y = B^T x (interior u -> psi).
template <typename T, typename Tin, typename Tout>
cudaError_t launch_btapply(const Geo<T>& g, const Tin* x, Tout* y, cudaStream_t s, const Bat& bt = Bat{});

// y = A_alpha^{-1} x (interior) by fast diagonalisation; work1/work2 scratch of Nu0.  With
// shift s > 0 (and alpha 1): y = (A + s M)^{-1} x for the pencil of g's eigenpairs.
// alpha is read from alpha_dev when non-null (graph replay), else alpha.
template <typename T>
cudaError_t launch_fdm(const Geo<T>& g, const double* alpha_dev, double alpha, const T* x, T* y, T* work1,
                       T* work2, cudaStream_t s, const int* skip = nullptr, const Bat& bt = Bat{}, double shift = 0.0);

// The fast diagonalisation on TMA-fed tcgen05 passes (FP32 in, 3xTF32 products, FP32
// accumulation): the tensors between passes live in a workspace in sliced form
// [k/4][rows][k%4], rows padded to the 128-row tile and slices to the 4-slice stage, as
// TF32-exact high parts and FP32 remainders; np problems (a lockstep group) share the
// pass matrices.  Host view: device pointers and sizes.
struct FdmTma {
    bool ready = false;
    int d = 0, np = 0;
    int n1[kMaxDim] = {1, 1, 1};
    long long R[kMaxDim] = {}, Rp[kMaxDim] = {};   // rows of the pass along axis j, padded
    int C[kMaxDim] = {}, Cp[kMaxDim] = {};         // 4-float slices of axis j, padded
    long long wsz = 0;                             // floats per workspace buffer
    float* ws = nullptr;                           // np x [buffer 0 hi, lo, buffer 1 hi, lo]
    const void* mA = nullptr;                      // device CUtensorMap [np][d][2 buffers][hi, lo]
    const void* mB = nullptr;                      // device CUtensorMap [variant][d][fwd, bwd][hi, lo]
    const float* lam[kMaxDim] = {};
};
// Number of TMA variants (N tiles of 64, 128, 256 and 32 columns).
int fdm_tma_variants();
// y = A_alpha^{-1} x (or (A + shift M)^{-1} x) for every problem of bt; x, y natural FP32.
cudaError_t launch_fdm_tma(const FdmTma& t, int variant, const double* alpha_dev, double alpha, const float* x,
                           float* y, cudaStream_t s, const int* skip, const Bat& bt, double shift);
// Build t for np problems of H's shape: workspace and maps through `alloc` (device bytes),
// the pass matrices from `consts` when given (a group reuses problem 0's), else uploaded.
// False (with the reason) when a tensor map cannot be made.
bool fdm_tma_setup(FdmTma& t, const HostProblem& H, const float* const* lam, int np,
                   const std::function<void*(size_t)>& alloc, cudaStream_t s, const FdmTma* consts,
                   std::string* why);

// w = -(D z + E z + B^T t)  (per cell), D from gw.  z, t in T; w in Tout.
template <typename T, typename Tout>
cudaError_t launch_schur_rest(const Geo<T>& g, const T* gw, double beta, const T* z, const T* t, Tout* w,
                              cudaStream_t s, IterCtl ctl = IterCtl{}, const Bat& bt = Bat{});

// FP64 matrix-free Newton apply y = G x (eq. pG-matrix), one fused launch.
cudaError_t launch_newton_apply(const Geo<double>& g, const double* gw, double alpha, double beta,
                                const double* x, double* y, cudaStream_t s, const Bat& bt = Bat{});


// ---- iterative A_alpha^{-1}: preconditioned CG on the stiffness matrix
// Block-Jacobi preconditioner over the entities of the hierarchical basis (see
// AinvPrecond): geometry of the blocks as the kernels need it.
struct PcgGeo {
    int d, nbub;
    int m[kMaxDim], n1[kMaxDim], nv[kMaxDim];
    int bsize[8];
    long long eoff[9];       // first entity of type t (types 1 .. 2^d - 1); eoff[2^d] = all
    long long boff[8];
    int bmax;
    const double* Binv;
    // overlapping two-level variant (one block per cell, classes by boundary ends)
    int cmax;
    int csize[64];
    long long coff[64];
    const double* Cinv;
    double* Y;               // per-cell block solutions, cmax per cell
    // overlapping variant with vertex-star patches (tensor boxes, local fast diagonalisation)
    int ns[kMaxDim];         // box extent per axis
    int np_[kMaxDim];        // patches per axis (interior vertices, or 1 on a one-cell axis)
    const double* Vs[kMaxDim];
    const double* lams[kMaxDim];
    double* Ys;              // per-patch solutions, ns0 ns1 ns2 per patch
};
// z = alpha^{-1} B_e^{-1} r on the dofs of every edge/face/interior entity e
cudaError_t launch_ainv_blocks(const PcgGeo& pg, double alpha, const double* r, double* z, cudaStream_t s);
// overlapping cell patches: Y_c = B_c^{-1} r|_c per cell, then z = alpha^{-1} sum_c R_c^T Y_c
// (+ zc at the vertex dofs), each dof summing its cells in a fixed order
cudaError_t launch_cells_solve(const PcgGeo& pg, long long ncells, const double* r, cudaStream_t s);
cudaError_t launch_cells_gather(const PcgGeo& pg, double alpha, const double* zc, double* z, long long n,
                                cudaStream_t s);
// vertex-star patches: Ys_v = A_v^{-1} r|_v per patch by fast diagonalisation of the box,
// then z = alpha^{-1} sum_v R_v^T Ys_v (+ zc at the vertex dofs), fixed order per dof
cudaError_t launch_stars_solve(const PcgGeo& pg, const double* r, cudaStream_t s);
cudaError_t launch_stars_gather(const PcgGeo& pg, double alpha, const double* zc, double* z, long long n,
                                cudaStream_t s);
// rc = r at the vertex (all-hat) dofs; z at the vertex dofs = zc
cudaError_t launch_vertex_gather(const PcgGeo& pg, const double* r, double* rc, long long nc, cudaStream_t s);
cudaError_t launch_vertex_scatter(const PcgGeo& pg, const double* zc, double* z, long long nc, cudaStream_t s);
// y = alpha A x (interior u, FP64, matrix-free)
cudaError_t launch_aapply(const Geo<double>& g, double alpha, const double* x, double* y, cudaStream_t s);
// partial dot products of a and b into part (count through nparts)
cudaError_t launch_dot(const double* a, const double* b, long long n, double* part, int* nparts, cudaStream_t s);

// ---- vector helpers (FP64 unless typed)
template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* x, Tout* y, long long n, cudaStream_t s, const Bat& bt = Bat{});
// y = a*x + b*y
cudaError_t launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s,
                         const Bat& bt = Bat{});
// y = x - b*z  (elementwise, z of precision T)
template <typename T>
cudaError_t launch_sub_scaled(const double* x, double b, const T* z, double* y, long long n, cudaStream_t s,
                              const Bat& bt = Bat{});
// trial state: xt = x - lam * dx (lam per problem from Bat::par when given)
cudaError_t launch_trial(const double* x, const double* dx, double lam, double* xt, long long n, cudaStream_t s,
                         const Bat& bt = Bat{});
// partial sums of squares of x into part (returns number of partials through nparts)
cudaError_t launch_sumsq(const double* x, long long n, double* part, int* nparts, cudaStream_t s,
                         const Bat& bt = Bat{});
// y = x (x null: y = 0), n elements
template <typename T>
cudaError_t launch_copy(const T* x, T* y, long long n, cudaStream_t s, const Bat& bt = Bat{});
// *dst = Bat::par[pb][slot] for every problem of the batch
cudaError_t launch_scatter_par(double* dst, int slot, cudaStream_t s, const Bat& bt);
// status words of every problem of the batch into out (device): out[pb*nd + k] = d[k],
// out[np*nd + pb*ni + k] = iv[k] (as doubles)
cudaError_t launch_gather_status(const double* d, int nd, const int* iv, int ni, double* out, cudaStream_t s,
                                 const Bat& bt);

// ---- GMRES (right-preconditioned, unrestarted), all state on the device.
constexpr int kMaxKrylov = 1000;   // upper bound of hpg_params.krylov_max
struct GmresDev {
    double* Vb;       // (kmax+1) x N basis storage: doubles (FP64 solves) or, in the same
                      // allocation, floats (FP32 inner solves); see gmres_basis
    double* H;        // kmax columns of (kmax+1)
    double* cs;       // kmax
    double* sn;       // kmax
    double* gv;       // kmax+1
    double* part_dots;  // dot-product partials, gmres_dot_blocks(N) x (kmax+2)
    double* part_norm;  // norm partials, >= max(gmres_upd_blocks(N), 1024)
    double* scal;     // [0] beta0, [1] resid estimate, [2] tol*beta0, [3] h_{j+1,j}, [4] ||w1||^2
    int* iflag;       // [0] stop flag, [1] completed iterations, [2] breakdown, [3] cap reached,
                      // [4] iteration cap of the current run (<= kmax)
    int* jdev;        // current iteration index
    double* hsum;     // final dot sums of the current pass, kmax+2
    unsigned int* counter;   // last-block counters of the dot kernel, one per vector group
    unsigned int* counter2;
    int* reo;         // 1: the current Arnoldi step takes a second Gram-Schmidt pass
    int* force;       // nonzero: every step takes the second pass (timing of the full step)
    double* y;        // kmax coefficients (also CGS scratch)
    int kmax;
    long long N;
};
// The basis viewed in its element type VT (double or float).
template <typename VT>
inline VT* gmres_basis(const GmresDev& G) { return reinterpret_cast<VT*>(G.Vb); }
int gmres_dot_blocks(long long N);
// Flexible GMRES on G: chunk partials of the dots V_v . w (v < nv, vectors ld apart),
// part[v * fg_chunks(N) + c]; and w += sgn * sum_v h[v] V_v (h on the device).
int fg_chunks(long long N);
cudaError_t launch_mdot(const double* V, long long ld, int nv, const double* w, long long N, double* part,
                        cudaStream_t s);
cudaError_t launch_maxpy(double* w, const double* V, long long ld, const double* h, int nv, long long N, double sgn,
                         cudaStream_t s);
int gmres_dot_groups(int kmax);
int gmres_upd_blocks(long long N);
// The GMRES launchers take the basis element type VT (double or float).
// r0 = b: beta0 = ||b||, V_0 = b / beta0, g = beta0 e_1, tol*beta0 stored, j = 0.
template <typename VT>
cudaError_t gmres_start(GmresDev& G, const double* b, double rtol, cudaStream_t s, int cap = 0,
                        const Bat& bt = Bat{});
// After w (= S Shat^{-1} V_j) has been written into V_{j+1}: CGS2 orthogonalise,
// normalise, Givens update, convergence test, j += 1.  No-op once stopped.
template <typename VT>
cudaError_t gmres_arnoldi(GmresDev& G, cudaStream_t s, const Bat& bt = Bat{});
// Timing aid: set j (and clear the stop flags), then one Arnoldi step.
template <typename VT>
cudaError_t gmres_timed_step(GmresDev& G, int j, cudaStream_t s);
// Set the WHILE condition of a device-side GMRES loop to "not stopped".
cudaError_t launch_gm_setcond(cudaGraphConditionalHandle h, const int* iflag, cudaStream_t s);
// the same for a batch: loop while any problem of the batch has not stopped
cudaError_t launch_gm_setcond_batch(cudaGraphConditionalHandle h, const int* iflag, cudaStream_t s, const Bat& bt);
// set the stop flag of the GMRES of every problem the mask selects
cudaError_t launch_gm_stop(int* iflag, cudaStream_t s, const Bat& bt);
// Solve H y = g for the completed iterations and form x = sum_i y_i V_i (FP64 sums).
template <typename VT>
cudaError_t gmres_finish(GmresDev& G, double* x, cudaStream_t s, const Bat& bt = Bat{});
// Number of FDM GEMM tile variants for elements of `elem` bytes.
int fdm_tile_count(int elem);
// K split of variant idx (variants with the same split give the same bits); 0: tensor cores
int fdm_tile_ks(int elem, int idx);
// FMA throughput of the SIMT pipe for elements of `elem` bytes (4: FP32, 8: FP64),
// measured with independent FMA chains on every SM (best of three timed launches on s).
cudaError_t measure_fma_peak(int elem, int sm_count, cudaStream_t s, double* tflops);
// Opt-in shared-memory limits of the large-smem kernels (call once per device).
void configure_kernels();

}  // namespace hpg
