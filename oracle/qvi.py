"""Thermoforming quasi-variational inequality by the fixed point of Section 6.4.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The QVI couples the membrane u (an obstacle problem whose obstacle depends on the
solution) with the mould temperature T:

    u <= Phi_0 + xi T,  (grad u, grad (v - u)) >= (f, v - u)  for all admissible v,
    (grad T, grad q) + gamma (T, q) = (g(Phi_0 + xi T - u), q)  for all q in H^1,

with g(s) = g_0 for s <= 0, g_0 (1 - s) for 0 < s < 1, 0 for s >= 1 (the paper's g
has g_0 = 1/5).  The fixed point of Section 6.4, from T_0 = 0:

  (I)  given T_i, solve the obstacle problem with phi = Phi_0 + xi T_i by hpG (the
       ObstacleOracle, a fresh proximal loop from psi_0 = 0);
  (II) given u_{i+1}, solve the nonlinear T equation by Newton's method, each
       system (A + gamma M - K) delta = R solved directly (SuperLU), with
       K_ij = (g'(s) xi phi_j, phi_i); R the residual below;

until ||u_i - u_{i-1}||_{H^1} <= tol.  T lives in the full U_{h,p} (no boundary
condition: the T equation is posed in H^1); A and M are the full stiffness and
mass matrices (hats and bubbles, boundary dofs included).

Readings where the paper is silent:
  * the quadrature of the nonsmooth term (g(.), q): p + 2 Gauss points per direction
    per cell;
  * the obstacle at the latent Gauss points is Phi_0 + xi T evaluated there (the
    constraint enters eq. (pG) only through (phi, zeta) on that rule);
  * Newton on T stops at ||R||_2 <= 1e-11 (absolute), from the previous T;
  * g'(s) is -g_0 on (0, 1) and 0 elsewhere (at the two kinks the one-sided value 0).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis1d as b1
from .hpg import ObstacleOracle, _as_field


def g_fun(s, g0):
    return np.where(s <= 0.0, g0, np.where(s < 1.0, g0 * (1.0 - s), 0.0))


def g_deriv(s, g0):
    return np.where((s > 0.0) & (s < 1.0), -g0, 0.0)


class QVIOracle:
    """Plain FP64 fixed point of the thermoforming QVI (Section 6.4)."""

    def __init__(self, breakpoints, p, f, Phi0, xi, gamma=1.0, g0=0.2, beta=1e-6, nq=None):
        self.Phi0 = _as_field(Phi0)
        self.xi = _as_field(xi)
        self.gamma = float(gamma)
        self.g0 = float(g0)
        # the obstacle oracle; its constraint is replaced at every fixed-point step
        self.obs = ObstacleOracle(breakpoints, p, f, lambda X: np.zeros(np.atleast_2d(X).shape[0]), None,
                                  beta=beta)
        S = self.obs.sp
        self.sp = S
        self.d, self.p = S.d, S.p
        self.Afull = sp.csr_matrix(S.A)
        self.Mfull = sp.csr_matrix(S.M)
        # quadrature of the T equation: nq Gauss points per direction per cell
        self.nq = nq or (self.p + 2)
        yq, wq = b1.gauss(self.nq)
        self.Uq = b1.local_u_values(self.p, yq)                 # (p+1, nq)
        self.cells = []
        for c in range(S.Nc):
            cidx = S.cell_multi(c)
            coords, det, l2g = [], 1.0, []
            for j in range(self.d):
                ms = S.meshes[j]
                coords.append(ms.to_physical(cidx[j], yq))
                det *= 0.5 * ms.h[cidx[j]]
                l2g.append(ms.local_to_global(cidx[j]))
            G = np.meshgrid(*coords, indexing="ij")
            X = np.stack([gg.ravel() for gg in G], axis=1)
            W = det
            for j in range(self.d):
                shape = [1] * self.d
                shape[j] = self.nq
                W = W * wq.reshape(shape)
            gl = S._global_grid(l2g)
            self.cells.append(dict(gl=gl, W=W, Phi0=self.Phi0(X).reshape([self.nq] * self.d),
                                   xi=self.xi(X).reshape([self.nq] * self.d)))
        # the latent Gauss points of the obstacle solve (q = n per direction per cell)
        Xl = S.cell_points.reshape(-1, self.d)
        self.Phi0_lat = self.Phi0(Xl).reshape(S.Nc, -1)
        self.xi_lat = self.xi(Xl).reshape(S.Nc, -1)
        yl, _ = b1.gauss(S.n)
        self.Ul = b1.local_u_values(self.p, yl)                 # (p+1, n)

    # ------------------------------------------------------------ fields
    def _at(self, ufull, U, c):
        """Values of the U_{h,p} field ufull at the tensor points of table U in cell c."""
        T = ufull[self.cells[c]["gl"]]
        for j in range(self.d):
            T = np.tensordot(U, T, axes=([0], [j]))
            T = np.moveaxis(T, 0, j)
        return T

    def _load(self, vals):
        """(v, phi_i) for the quadrature values vals[c] (weights included by the caller)."""
        out = np.zeros(self.sp.Nu)
        for c, cd in enumerate(self.cells):
            T = vals[c]
            for j in range(self.d):
                T = np.tensordot(self.Uq, T, axes=([1], [j]))
                T = np.moveaxis(T, 0, j)
            np.add.at(out, cd["gl"].ravel(), T.ravel())
        return out

    def latent_obstacle(self, T):
        """Phi_0 + xi T at the latent Gauss points, (Nc, n^d), x index fastest."""
        out = np.zeros_like(self.Phi0_lat)
        for c in range(self.sp.Nc):
            v = self._at(T, self.Ul, c)                          # indexed [i_0, i_1, ...]
            out[c] = self.Phi0_lat[c] + self.xi_lat[c] * v.ravel(order="F")
        return out

    # ------------------------------------------------------------ T step
    def T_residual(self, T, u):
        vals = []
        for c, cd in enumerate(self.cells):
            s = cd["Phi0"] + cd["xi"] * self._at(T, self.Uq, c) - self._at(u, self.Uq, c)
            vals.append(cd["W"] * g_fun(s, self.g0))
        return self.Afull @ T + self.gamma * (self.Mfull @ T) - self._load(vals)

    def T_jacobian(self, T, u):
        rows, cols, data = [], [], []
        npl = (self.p + 1) ** self.d
        for c, cd in enumerate(self.cells):
            s = cd["Phi0"] + cd["xi"] * self._at(T, self.Uq, c) - self._at(u, self.Uq, c)
            w = cd["W"] * g_deriv(s, self.g0) * cd["xi"]            # (nq,)*d
            # K_loc[a, b] = sum_q w_q phi_a(x_q) phi_b(x_q), phi tensor products of Uq rows
            Kloc = self._local_mass(w)
            gl = cd["gl"].ravel()
            rows.append(np.repeat(gl, npl))
            cols.append(np.tile(gl, npl))
            data.append(Kloc.ravel())
        K = sp.csr_matrix((np.concatenate(data), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.sp.Nu, self.sp.Nu))
        return (self.Afull + self.gamma * self.Mfull - K).tocsc()

    def _local_mass(self, w):
        """sum_q w_q phi_a(x_q) phi_b(x_q) over the tensor local basis, indexed like cd['gl'].ravel()."""
        d, U = self.d, self.Uq
        if d == 2:
            return np.einsum("iq,jr,qr,kq,lr->ijkl", U, U, w, U, U).reshape((self.p + 1) ** 2, -1)
        return np.einsum("iq,jr,ks,qrs,lq,mr,ns->ijklmn", U, U, U, w, U, U, U).reshape((self.p + 1) ** 3, -1)

    def T_newton(self, u, T0, tol=1e-11, max_it=50):
        T = T0.copy()
        R = self.T_residual(T, u)
        it = 0
        while np.linalg.norm(R) > tol and it < max_it:
            T = T - spla.spsolve(self.T_jacobian(T, u), R)
            R = self.T_residual(T, u)
            it += 1
        return T, it, np.linalg.norm(R)

    # ------------------------------------------------------------ fixed point
    def h1_norm(self, v):
        return float(np.sqrt(max(v @ (self.Afull @ v + self.Mfull @ v), 0.0)))

    def solve(self, alphas, tol=3e-3, max_fp=30, newton_tol=1e-10):
        S = self.sp
        T = np.zeros(S.Nu)
        u_prev = None
        hist = []
        for i in range(max_fp):
            phi_q = self.latent_obstacle(T)
            self.obs.phiz = S.project_gauss(phi_q).ravel()
            r = self.obs.solve(alphas, tol=newton_tol)
            if not r["converged"]:
                raise RuntimeError("obstacle step did not converge")
            u = r["u"]
            T, t_it, t_res = self.T_newton(u, T)
            dn = None if u_prev is None else self.h1_norm(u - u_prev)
            hist.append(dict(newton=r["newton"], t_newton=t_it, t_res=t_res, du_h1=dn))
            u_prev = u
            if dn is not None and dn <= tol:
                break
        return dict(u=u, T=T, iterations=len(hist), history=hist)
