// Internal declarations of libhpg (host setup, device buffers, kernel launchers).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "hpg.h"

namespace hpg {

constexpr int kMaxDim = 3;
constexpr int kMaxN = 32;       // coefficients per direction per cell (n = p-1 or p)
// largest dynamic shared memory a per-cell kernel of the path may ask for (bytes)
constexpr size_t kCellSmemMax = 200 * 1024;
constexpr int kEll = 8;         // padded width of the 1D stencils

// ---------------------------------------------------------------- host math
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// P_0..P_kmax and their derivatives at y
void legendre_all(int kmax, double y, double* P, double* dP);
// Cholesky A = L L^T (row-major, lower triangle written); false if not SPD
bool cholesky(int n, std::vector<double>& A);
// Symmetric eigen-decomposition (Householder tridiagonalisation + implicit QL).
// On return w holds eigenvalues ascending and Z (row-major, column j = vector j).
bool symmetric_eigen(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& Z);

// Padded-ELL sparse operator: row r has cnt[r] <= kEll entries (col, val).
struct Ell {
    int rows = 0;
    std::vector<int> cnt, col;
    std::vector<double> val;
    void init(int r) { rows = r; cnt.assign(r, 0); col.assign((size_t)r * kEll, 0); val.assign((size_t)r * kEll, 0.0); }
    void add(int r, int c, double v);
};

// 1D operators of one direction (uniform mesh of m cells of width h, degree p).
struct Dir1D {
    int m = 0, p = 0, n = 0;    // n = latent coefficients per cell
    int N1 = 0, n1 = 0;         // full and interior 1D u counts
    double lo = 0, h = 0;
    // Full 1D matrices over the N1 global dofs (closed forms, Section 3)
    Ell A, M;                   // (v_i', v_j'), (v_i, v_j)            N1 x N1
    Ell B, Bd;                  // (v_i, zeta_k), (v_i', zeta_k)       N1 x (m n)
    // Interior-only versions used by the device (columns in interior numbering)
    Ell Ai, Mi;                 // n1 x n1
    Ell Bi, Bdi;                // n1 x (m n)
    Ell BTi, BdTi;              // (m n) x n1
    // Fast diagonalisation: A_int V = M_int V diag(lam), V^T M_int V = I
    std::vector<double> V, lam; // V row-major n1 x n1
    int glob_of_int(int i) const;   // interior index -> global 1D index
    int int_of_glob(int g) const;   // global -> interior (-1 for boundary)
};

// Preconditioner of the stiffness matrix A for the iterative (inexact) A_alpha^{-1}:
// block Jacobi over the hierarchical basis split by entity -- the vertex (all-hat)
// functions form one block, the coarse Q1 stiffness, solved exactly by fast
// diagonalisation of the 1D hat pencils; every edge, face and cell interior carries the
// block of its bubble functions, solved with a dense inverse.  On a uniform mesh all
// entities of one type (which axes carry bubbles) share one block.
struct AinvPrecond {
    bool built = false;
    int nv[kMaxDim] = {1, 1, 1};                 // interior vertices per axis (m_j - 1)
    std::vector<double> Vc[kMaxDim], lamc[kMaxDim];
    int bsize[8] = {};                           // block size of type t (bubble-axis mask t)
    long long nent[8] = {};                      // entities of type t
    long long boff[8] = {};                      // offset of type t's inverse block in Binv
    std::vector<double> Binv;                    // the inverse blocks, row-major, by type
    // two-level overlapping variant: one block per cell holding all the cell's interior
    // dofs (principal submatrix of A); cells fall in classes by which of their ends are
    // on the boundary along each axis (code 0: both, 1: left, 2: right, 3: none)
    bool cells_built = false;
    int cmax = 0;                                // largest cell block
    int csize[64] = {};                          // block size of class k (-1: class absent)
    long long coff[64] = {};                     // offset of class k's inverse block in Cinv
    std::vector<double> Cinv;
    // two-level overlapping variant with one patch per interior vertex: the interior of
    // the vertex's star of cells, a tensor-product box per axis [bubbles of the left cell,
    // the vertex's hat, bubbles of the right cell] (just the cell's bubbles on an axis with
    // one cell), solved exactly by fast diagonalisation of the 1D star pencils
    bool stars_built = false;
    int ns[kMaxDim] = {1, 1, 1};                 // star box extent per axis
    std::vector<double> Vs[kMaxDim], lams[kMaxDim];
};

// Everything the device path needs, computed on the host at setup.
struct HostProblem {
    int d = 2, p = 2, n = 1, kind = 0, ncomp = 1;
    int m[kMaxDim] = {1, 1, 1};
    double lo[kMaxDim] = {0, 0, 0}, hi[kMaxDim] = {1, 1, 1}, h[kMaxDim] = {1, 1, 1};
    Dir1D dir[kMaxDim];
    size_t Nu_full = 0, Nu0 = 0, Nc = 0, nloc = 0, nb = 0, Npsi = 0, Nq = 0;
    double detJ = 1.0;
    // reference quadrature of the latent rule (q = n Gauss points)
    std::vector<double> yq, wq;          // n
    std::vector<double> Vq;              // n x n, Vq[i*n + k] = P_k(y_i)
    std::vector<double> Mpsi_loc;        // nloc: diagonal Psi mass of one cell (per component)
    std::vector<double> Kpsi_loc;        // nloc x nloc broken H^1 seminorm of one cell (gradient E_beta)
    std::vector<double> Cblk;            // nloc x nloc: B-hat^T A-hat_1^{-1} B-hat (obstacle)
    // data
    double sign = 1.0;                   // -1 for lower obstacles
    std::vector<double> bf;              // (f, v) over interior dofs  (sign applied)
    std::vector<double> phiq;            // phi at the latent Gauss points (sign applied)
    std::vector<double> phiz;            // (phi, zeta) (obstacle)
    std::vector<double> ulift;           // full u with boundary lifting (sign applied)
    std::vector<double> rA;              // A_{0g} u_g (interior rows)
    std::vector<double> rB;              // B_g^T u_g (psi rows)
    bool has_phi = false;
    std::vector<double> alphas;
    AinvPrecond ap;
};

void build_dir1d(Dir1D& D, int m, int p, int n, double lo, double hi);
void pencil_eigen(int N, const std::vector<double>& Ad, const std::vector<double>& Md, std::vector<double>& V,
                  std::vector<double>& lam);
void build_problem_constants(HostProblem& P);
// Quadrature points of the latent rule, Nq x d, cell-major, x fastest.
void latent_points(const HostProblem& P, std::vector<double>& pts);
void compute_rhs(HostProblem& P, hpg_field_fn f, void* user, bool is_const, double c);
void compute_phi(HostProblem& P, const double* phi_q);
void compute_lifting(HostProblem& P, hpg_field_fn g, void* user);
double eval_u_point(const HostProblem& P, const std::vector<double>& ufull, const double* x);
// Build P.ap (coarse pencils and entity blocks of the stiffness preconditioner).
void build_ainv_precond(HostProblem& P);
// Build the cell-patch blocks of P.ap (the overlapping two-level variant).
void build_ainv_cells(HostProblem& P);
// Build the vertex-star pencils of P.ap (the overlapping variant with star patches).
void build_ainv_stars(HostProblem& P);
// e^T (M_1 (x) ... (x) M_d) e for a full u-coefficient vector e: the squared L2(Omega)
// norm of the field, with the exact 1D mass matrices of Section 3.
double mass_norm2(const HostProblem& P, const std::vector<double>& e);

}  // namespace hpg
