"""Schur complement S and its block-diagonal approximation S-hat (Sections 4.4-4.6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

eq. (schur4):  S = -(D_psi + E_beta + B^T A_alpha^{-1} B).
eq. (schur-preconditioner) (obstacle):
    S-hat = -D_psi - E_beta - B-hat^T A-hat_alpha^{-1} B-hat,
    [A-hat_alpha]_ij = alpha (grad_h eta_i, grad_h eta_j),  B-hat_ij = (eta_i, zeta_j),
  with eta the tensor-product spectral-Galerkin functions Y_a of each cell.
  Reading: the index range of Phi_{h,p} is not printed; it is taken to be
  Y_0..Y_{p-2} per direction, i.e. the bubbles of U_{h,p} rescaled (the hats
  are removed), which makes B-hat square (n^d x n^d per cell).
eq. (schur-preconditioner:gradient):  S-hat = -D_psi - E_beta.
eq. (schur2): y = b_psi - B^T A^{-1} b_u, delta_psi = S^{-1} y,
              delta_u = A^{-1}(b_u - B delta_psi).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis1d as b1
from .space import kron_dense


def spectral_cell_matrices(h, p):
    """1D reference-mapped cell matrices of Y_0..Y_{p-2} and P_0..P_{p-2}.

    Returns (KY, MY, BY): (Y_a', Y_b')_K, (Y_a, Y_b)_K, (Y_a, P_k)_K, each (p-1) x (p-1).
    """
    y, w = b1.gauss(b1.QUAD_REF)
    nb = p - 1
    Y = np.array([b1.spectral(a, y) for a in range(nb)])
    dY = np.array([b1.spectral_deriv(a, y) for a in range(nb)])
    P = b1.local_psi_values(nb, y)
    J = 0.5 * h
    KY = (dY * w) @ dY.T / J
    MY = (Y * w) @ Y.T * J
    BY = (Y * w) @ P.T * J
    return KY, MY, BY


def shat_constant_block(hs, p):
    """C_K = B-hat^T A-hat_1^{-1} B-hat for a cell with side lengths hs (n^d x n^d)."""
    d = len(hs)
    mats = [spectral_cell_matrices(h, p) for h in hs]
    Ahat = 0.0
    for k in range(d):
        Ahat = Ahat + kron_dense([mats[j][0] if j == k else mats[j][1] for j in range(d)])
    Bhat = kron_dense([mats[j][2] for j in range(d)])
    return Bhat.T @ np.linalg.solve(Ahat, Bhat), Ahat, Bhat


class SchurOracle:
    """S, S-hat and the sequential Schur solve for an ``ObstacleOracle``."""

    def __init__(self, orc):
        self.o = orc
        S = orc.sp
        self.sp = S
        hs = [ms.h[0] for ms in S.meshes]
        for ms in S.meshes:
            assert np.allclose(ms.h, ms.h[0]), "uniform meshes only"
        self.C, self.Ahat, self.Bhat = shat_constant_block(hs, S.p)
        self.Mdiag = orc.Mpsi.diagonal().reshape(S.Nc, S.nloc)
        self.lu_A = spla.splu(sp.csc_matrix(orc.A00))

    def Ainv(self, x, alpha):
        return self.lu_A.solve(x) / alpha

    def shat_blocks(self, psi, alpha, beta=None):
        """Cell blocks of S-hat (negative definite), (Nc, n^d, n^d)."""
        beta = self.o.beta if beta is None else beta
        D = self.o.D_blocks(psi)
        M = np.einsum("ci,ij->cij", self.Mdiag, np.eye(self.sp.nloc))
        return -(D + beta * M + self.C[None, :, :] / alpha)

    def apply_S(self, x, psi, alpha, beta=None):
        beta = self.o.beta if beta is None else beta
        D = self.o.D_matrix(psi)
        t = self.Ainv(self.o.B0 @ x, alpha)
        return -(D @ x + beta * (self.o.Mpsi @ x) + self.o.B0.T @ t)

    def apply_shat_inv(self, x, psi, alpha, beta=None):
        blocks = self.shat_blocks(psi, alpha, beta)
        xs = x.reshape(self.sp.Nc, self.sp.nloc)
        return np.linalg.solve(blocks, xs[..., None])[..., 0].ravel()

    def dense_S(self, psi, alpha, beta=None):
        n = self.sp.Npsi
        return np.column_stack([self.apply_S(e, psi, alpha, beta) for e in np.eye(n)])

    def schur_solve(self, bu, bpsi, psi, alpha, beta=None):
        """eq. (schur2) with exact A^{-1} and exact (dense) S^{-1}; small problems only."""
        y = bpsi - self.o.B0.T @ self.Ainv(bu, alpha)
        dpsi = np.linalg.solve(self.dense_S(psi, alpha, beta), y)
        du = self.Ainv(bu - self.o.B0 @ dpsi, alpha)
        return du, dpsi
