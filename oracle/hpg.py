"""hpG obstacle solver: LVPP subproblems (eq. pG) solved by Newton with a
sparse direct solve of the Newton matrix G (eq. pG-matrix) at every step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discrete subproblem for alpha = alpha_k, given psi_prev = psi_{k-1}
(eq. pG, Section 4.1), unknowns: interior u coefficients and psi:

    F_u   = alpha A u + B (psi - psi_prev) - alpha (f, v)          (interior rows)
    F_psi = B^T u + (exp(-psi), zeta) - (phi, zeta)

where u is the full coefficient vector (its boundary entries are the fixed
Dirichlet lifting, so the lifting terms are the boundary columns of A and B).
The Newton matrix of eq. (pG-matrix) is

    G = [[alpha A_00, B_0], [B_0^T, -D_psi - E_beta]],
    [D_psi]_ij = (zeta_i, exp(-psi) zeta_j),  E_beta = beta M_Psi,

with E_beta added to the Jacobian only (Section 4.1): the fixed point does not
depend on beta.  Each Newton step solves G delta = F and sets x <- x - lambda delta.

Readings where the paper is silent:
  * line search: lambda = 1, halved while ||F(x - lambda delta)||_2 >
    (1 - 1e-4 lambda) ||F(x)||_2, at most 10 halvings (then the step is
    accepted and flagged);
  * Newton stops when ||[F_u; F_psi]||_2 <= tol (absolute, default 1e-10),
    cap 50 per proximal step;
  * each subproblem is warm-started from the previous (u, psi); psi_0 = 0;
  * alpha_k = min(alpha_1 2^{(k-1)/2}, cap) (the sqrt(2)-growth rule of
    Section 6.1 written in closed form), stopping once alpha_k = alpha_{k-1};
  * if any Gauss value psi(x_q) < -700 the exponential would overflow; the
    solve stops with a non-finite flag;
  * lower obstacles u >= phi (not treated in the paper, which has u <= phi)
    are solved as -u <= -phi with f, g negated; u is negated back.
"""
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .space import TensorSpace


def block_diagonal(blocks):
    """Sparse block-diagonal matrix from dense blocks (Nc, b, b)."""
    nc = blocks.shape[0]
    return sp.csr_matrix(sp.bsr_matrix((blocks, np.arange(nc), np.arange(nc + 1)),
                                       shape=(nc * blocks.shape[1], nc * blocks.shape[2])))


def sparse_direct_solve(G, F):
    """Sparse LU (SuperLU) of G with a symmetric minimum-degree ordering and no pivoting.

    G is symmetric quasi-definite (alpha A_00 SPD, -D - E negative definite),
    so every symmetric permutation of it has an LDL^T factorisation and
    diagonal pivots are safe.
    """
    lu = spla.splu(sp.csc_matrix(G), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    return lu.solve(F)


def eliminated_direct_solve(alphaA00, B0, C_blocks, F, G=None, refine=8):
    """The same linear system G delta = F, by exact block elimination of psi.

    G = [[alpha A_00, B_0], [B_0^T, -C]] with C = D_psi + E_beta block-diagonal
    over the cells and SPD.  The second block row gives
    delta_psi = C^{-1} (B_0^T delta_u - F_psi); substituted into the first,
    (alpha A_00 + B_0 C^{-1} B_0^T) delta_u = F_u + B_0 C^{-1} F_psi, whose
    matrix is SPD and is factorised by the same sparse LU (symmetric
    minimum-degree ordering, diagonal pivots).  Up to rounding the result is
    that of ``sparse_direct_solve(G, F)``; the elimination order only moves the
    fill-in to where it fits in host memory for the 3D workloads (the direct
    factorisation of G for 8^3 hexes at p = 6 does not fit in 62 GB).

    Where the constraint is active exp(-psi) is tiny, C^{-1} is huge and the
    eliminated matrix is badly scaled, so the solve alone can lose digits; with G
    given, the result is refined against G itself (r = F - G delta, delta += the
    same solve of r) until ||r|| <= 1e-14 ||F|| or `refine` passes -- iterative
    refinement in FP64 of a direct method, which converges to the solution of
    G delta = F whenever the factorisation is a contraction for G.
    """
    nu = B0.shape[0]
    Cinv = block_diagonal(np.linalg.inv(C_blocks))
    K = sp.csc_matrix(alphaA00 + B0 @ Cinv @ B0.T)
    lu = spla.splu(K, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0, options=dict(SymmetricMode=True))
    def once(R):
        Ru, Rpsi = R[:nu], R[nu:]
        du = lu.solve(Ru + B0 @ (Cinv @ Rpsi))
        dpsi = Cinv @ (B0.T @ du - Rpsi)
        return np.concatenate([du, dpsi])

    delta = once(F)
    if G is not None:
        nF = np.linalg.norm(F)
        for _ in range(refine):
            R = F - G @ delta
            if np.linalg.norm(R) <= 1e-14 * nF:
                break
            delta = delta + once(R)
    return delta


def alpha_schedule(alpha1, cap, growth_log2=0.5, max_steps=1000):
    """alpha_k = min(alpha_1 * 2^{growth_log2 (k-1)}, cap), stop once alpha_k == alpha_{k-1}."""
    out = []
    k = 1
    while k <= max_steps:
        a = min(alpha1 * 2.0 ** (growth_log2 * (k - 1)), cap)
        out.append(a)
        if len(out) >= 2 and out[-1] == out[-2]:
            break
        k += 1
    return out


def _as_field(v):
    if callable(v):
        return v
    c = float(v)
    return lambda X: np.full(np.asarray(X).shape[0], c)


class ObstacleOracle:
    """Plain FP64 hpG for u <= phi (or u >= phi with ``lower=True``)."""

    def __init__(self, breakpoints, p, f, phi, g=None, beta=0.0, lower=False, linear="direct"):
        """``linear``: "direct" (sparse LU of G) or "eliminate_psi" (the same
        system by block elimination of psi, see ``eliminated_direct_solve``)."""
        if linear not in ("direct", "eliminate_psi"):
            raise ValueError("linear must be 'direct' or 'eliminate_psi'")
        self.linear = linear
        self.sp = TensorSpace(breakpoints, p, kind="obstacle")
        self.beta = float(beta)
        self.lower = bool(lower)
        s = -1.0 if lower else 1.0
        fF, phiF = _as_field(f), _as_field(phi)
        self.f = lambda X: s * fF(X)
        self.phi = lambda X: s * phiF(X)
        self.g = None if g is None else (lambda X: s * _as_field(g)(X))
        S = self.sp
        self.interior = S.interior
        self.A = S.A
        self.B = S.B
        self.A00 = sp.csr_matrix(S.A[S.interior][:, S.interior])
        self.B0 = sp.csr_matrix(S.B[S.interior])
        self.bf = S.f_load(self.f)
        self.phiz = S.phi_zeta(self.phi)
        self.ulift = S.lifting(self.g)
        self.Mpsi = sp.csr_matrix(S.Mpsi)

    # ------------------------------------------------------------ pieces
    def gauss_values(self, psi):
        """psi at the q^d Gauss points of every cell: (Nc, q^d)."""
        S = self.sp
        return psi.reshape(S.Nc, S.nloc) @ S.Vd.T

    def gauss_weights(self, psi):
        """g_q = w_q |J_K| exp(-psi(x_q)); raises FloatingPointError if psi_q < -700."""
        pq = self.gauss_values(psi)
        if np.any(pq < -700.0) or not np.all(np.isfinite(pq)):
            raise FloatingPointError("exp(-psi) overflow: psi < -700 at a Gauss point")
        return self.sp.wJ * np.exp(-pq)

    def residual(self, u, psi, psi_prev, alpha):
        """[F_u (interior rows); F_psi] of eq. (pG) for full u."""
        S = self.sp
        Fu = alpha * (self.A @ u) + self.B @ (psi - psi_prev) - alpha * self.bf
        eg = (self.gauss_weights(psi) @ S.Vd).ravel()
        Fpsi = self.B.T @ u + eg - self.phiz
        return np.concatenate([Fu[S.interior], Fpsi])

    def D_blocks(self, psi):
        """Cell blocks of D_psi: (Nc, n^d, n^d), D_K = V^T diag(g_q) V."""
        S = self.sp
        gw = self.gauss_weights(psi)
        return np.einsum("qi,cq,qj->cij", S.Vd, gw, S.Vd)

    def D_matrix(self, psi):
        return block_diagonal(self.D_blocks(psi))

    def jacobian(self, psi, alpha, beta=None):
        beta = self.beta if beta is None else beta
        D = self.D_matrix(psi)
        E = beta * self.Mpsi
        return sp.bmat([[alpha * self.A00, self.B0], [self.B0.T, -D - E]], format="csc")

    def newton_step(self, psi, alpha, F):
        """delta with G(psi, alpha) delta = F (eq. pG-matrix), solved exactly."""
        if self.linear == "direct":
            return sparse_direct_solve(self.jacobian(psi, alpha), F)
        S = self.sp
        mloc = self.Mpsi.diagonal().reshape(S.Nc, S.nloc)
        C = self.D_blocks(psi) + self.beta * np.einsum("ci,ij->cij", mloc, np.eye(S.nloc))
        return eliminated_direct_solve(alpha * self.A00, self.B0, C, F, G=self.jacobian(psi, alpha))

    def split(self, x):
        ni = len(self.interior)
        return x[:ni], x[ni:]

    def initial_state(self):
        u = self.ulift.copy()
        psi = np.zeros(self.sp.Npsi)
        return u, psi

    # ------------------------------------------------------------ Newton
    def newton(self, u, psi, psi_prev, alpha, tol=1e-10, max_it=50, ls_max=10, log=None):
        """Solve one subproblem.  Returns (u, psi, iterations, info)."""
        u = u.copy()
        psi = psi.copy()
        F = self.residual(u, psi, psi_prev, alpha)
        nF = np.linalg.norm(F)
        hist = [nF]
        it = 0
        ls_fail = 0
        t_solve = 0.0
        while nF > tol and it < max_it:
            t0 = time.perf_counter()
            delta = self.newton_step(psi, alpha, F)
            t_solve += time.perf_counter() - t0
            du, dpsi = self.split(delta)
            lam = 1.0
            for halving in range(ls_max + 1):
                ut = u.copy()
                ut[self.interior] -= lam * du
                pt = psi - lam * dpsi
                try:
                    Ft = self.residual(ut, pt, psi_prev, alpha)
                    nFt = np.linalg.norm(Ft)
                except FloatingPointError:
                    nFt = np.inf
                if nFt <= (1.0 - 1e-4 * lam) * nF:
                    break
                if halving == ls_max:
                    ls_fail += 1
                    if not np.isfinite(nFt):
                        raise FloatingPointError("line search ended on a non-finite residual")
                    break
                lam *= 0.5
            u, psi, F, nF = ut, pt, Ft, nFt
            it += 1
            hist.append(nF)
            if log:
                log(f"alpha={alpha:.6g} it={it} |F|={nF:.3e} lambda={lam}")
        info = dict(converged=nF <= tol, residual=nF, history=hist, ls_fail=ls_fail,
                    t_linear=t_solve)
        return u, psi, it, info

    def solve(self, alphas, tol=1e-10, max_it=50, log=None):
        """Full hpG proximal loop.  Returns dict with u (external sign), psi, counts."""
        u, psi = self.initial_state()
        psi_prev = psi.copy()
        counts, infos = [], []
        for a in alphas:
            u, psi, it, info = self.newton(u, psi, psi_prev, a, tol=tol, max_it=max_it, log=log)
            counts.append(it)
            infos.append(info)
            if not info["converged"]:
                break
            psi_prev = psi.copy()
        s = -1.0 if self.lower else 1.0
        return dict(u=s * u, psi=psi, newton=counts, infos=infos,
                    converged=all(i["converged"] for i in infos) and len(counts) == len(alphas))
