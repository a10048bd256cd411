"""hpG for the gradient-type constraint |grad u| <= phi (eq. pG:gradient, Section 4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

u has partial degree p (continuous); psi in Psi^d has partial degree p-1
(n = p Legendre functions per direction) with d components, stored
[cell][component][n^d].  With G(psi) = phi psi (1 + |psi|^2)^{-1/2}:

    F_u   = alpha A u + B (psi - psi_prev) - alpha (f, v),   B_ij = (grad v_i, zeta_j)
    F_psi = B^T u - (G(psi), zeta)

Newton matrix (eq. pG-matrix, not relabelled in Section 4.2):
    [[alpha A_00, B_0], [B_0^T, -D_psi - E_beta]],
    D_psi = (zeta_i, J(psi) zeta_j),  J = phi (s I - psi psi^T) s^{-3/2},  s = 1 + |psi|^2.

Readings: the Gauss rule has q = n = p points per direction (as for the
obstacle case); E_beta = beta (grad_h zeta_i, grad_h zeta_j) per component on
the Psi^d basis itself (the printed definition indexes it by Phi, which has
no d-vector Legendre counterpart of the same size).  Newton, line search,
tolerances and the alpha loop are those of ``hpg.ObstacleOracle``.
"""
import time

import numpy as np
import scipy.sparse as sp

from .space import TensorSpace
from .hpg import sparse_direct_solve, block_diagonal, _as_field


class GradientOracle:
    def __init__(self, breakpoints, p, f, phi, beta=0.0):
        self.sp = TensorSpace(breakpoints, p, kind="gradient")
        self.beta = float(beta)
        S = self.sp
        self.f = _as_field(f)
        self.phi = _as_field(phi)
        self.interior = S.interior
        self.A = S.A
        self.B = S.B
        self.A00 = sp.csr_matrix(S.A[S.interior][:, S.interior])
        self.B0 = sp.csr_matrix(S.B[S.interior])
        self.bf = S.f_load(self.f)
        self.phiq = self.phi(S.cell_points.reshape(-1, S.d)).reshape(S.Nc, -1)   # (Nc, q^d)
        self.Kpsi = sp.csr_matrix(S.Kpsi)

    def gauss_values(self, psi):
        """(Nc, d, q^d) Gauss values of each component."""
        S = self.sp
        return np.einsum("ckj,qj->ckq", psi.reshape(S.Nc, S.d, S.nloc), S.Vd)

    def residual(self, u, psi, psi_prev, alpha):
        S = self.sp
        Fu = alpha * (self.A @ u) + self.B @ (psi - psi_prev) - alpha * self.bf
        pq = self.gauss_values(psi)
        s = 1.0 + np.sum(pq * pq, axis=1)                      # (Nc, q^d)
        Gq = self.phiq[:, None, :] * pq / np.sqrt(s)[:, None, :]
        proj = np.einsum("cq,ckq,qj->ckj", S.wJ, Gq, S.Vd).ravel()
        Fpsi = self.B.T @ u - proj
        return np.concatenate([Fu[S.interior], Fpsi])

    def D_blocks(self, psi):
        """(Nc, d n^d, d n^d) cell blocks of D_psi, component-major inside a cell."""
        S = self.sp
        d, nl = S.d, S.nloc
        pq = self.gauss_values(psi)
        s = 1.0 + np.sum(pq * pq, axis=1)
        out = np.zeros((S.Nc, d * nl, d * nl))
        for a in range(d):
            for b in range(d):
                Jab = self.phiq * ((s if a == b else 0.0) - pq[:, a, :] * pq[:, b, :]) / s ** 1.5
                out[:, a * nl:(a + 1) * nl, b * nl:(b + 1) * nl] = np.einsum(
                    "qi,cq,qj->cij", S.Vd, S.wJ * Jab, S.Vd)
        return out

    def jacobian(self, psi, alpha, beta=None):
        beta = self.beta if beta is None else beta
        D = block_diagonal(self.D_blocks(psi))
        return sp.bmat([[alpha * self.A00, self.B0], [self.B0.T, -D - beta * self.Kpsi]], format="csc")

    def initial_state(self):
        return np.zeros(self.sp.Nu), np.zeros(self.sp.Npsi)

    def newton(self, u, psi, psi_prev, alpha, tol=1e-10, max_it=50, ls_max=10, log=None):
        u, psi = u.copy(), psi.copy()
        F = self.residual(u, psi, psi_prev, alpha)
        nF = np.linalg.norm(F)
        hist, it, ls_fail = [nF], 0, 0
        ni = len(self.interior)
        while nF > tol and it < max_it:
            delta = sparse_direct_solve(self.jacobian(psi, alpha), F)
            du, dpsi = delta[:ni], delta[ni:]
            lam = 1.0
            for halving in range(ls_max + 1):
                ut = u.copy()
                ut[self.interior] -= lam * du
                pt = psi - lam * dpsi
                Ft = self.residual(ut, pt, psi_prev, alpha)
                nFt = np.linalg.norm(Ft)
                if nFt <= (1.0 - 1e-4 * lam) * nF:
                    break
                if halving == ls_max:
                    ls_fail += 1
                    break
                lam *= 0.5
            u, psi, F, nF = ut, pt, Ft, nFt
            it += 1
            hist.append(nF)
            if log:
                log(f"alpha={alpha:.6g} it={it} |F|={nF:.3e} lambda={lam}")
        return u, psi, it, dict(converged=nF <= tol, residual=nF, history=hist, ls_fail=ls_fail)

    def solve(self, alphas, tol=1e-10, max_it=50, log=None):
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
        return dict(u=u, psi=psi, newton=counts, infos=infos,
                    converged=all(i["converged"] for i in infos) and len(counts) == len(alphas))

    def grad_magnitude_at(self, u, X):
        """|grad u_h| at points X by central differences of the FE function (diagnostic)."""
        S = self.sp
        eps = 1e-6
        g2 = 0.0
        for j in range(S.d):
            e = np.zeros(S.d)
            e[j] = eps
            g2 = g2 + ((S.evaluate(u, X + e) - S.evaluate(u, X - e)) / (2 * eps)) ** 2
        return np.sqrt(g2)
