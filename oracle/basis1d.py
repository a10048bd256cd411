"""1D hierarchical p-FEM bases and 1D global matrices (Section 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Reference cell K = [-1, 1].  A physical cell [x_c, x_{c+1}] of width h is
mapped by x = x_c + (y + 1) h / 2, so dx = (h/2) dy and d/dx = (2/h) d/dy.

Functions (Section 3):
  * Legendre P_k            -- basis of the discontinuous space Psi_{h,p}.
  * hats (1 -/+ y)/2        -- the piecewise-linear H_i of U_{h,p}.
  * bubbles W_n, eq. (Wn):  W_n(y) = (1 - y^2) P_n^{(1,1)}(y) / (2(n+1)),
                            n = 0..p-2  (so that d/dy W_n = -P_{n+1}).
  * spectral Galerkin Y_n = P_n - P_{n+2}.

All integrals below use a 64-point Gauss--Legendre rule applied to
``scipy.special`` evaluations; nothing uses the closed forms of the
integrals (those are what the tests check).

Global 1D numbering of U_{h,p} on m cells: hats 0..m first, then bubbles
cell-major, bubble b of cell c at index m + 1 + c (p - 1) + b.  The Dirichlet
(boundary) dofs are the hats 0 and m; the remaining n1 = m p - 1 are interior.
Global 1D numbering of Psi: cell c, Legendre degree k at c n + k.
"""
import numpy as np
from scipy.special import eval_legendre, eval_jacobi, roots_legendre
import scipy.sparse as sp

QUAD_REF = 64


def gauss(npts):
    """Gauss--Legendre nodes and weights on [-1, 1] (scipy)."""
    y, w = roots_legendre(npts)
    return np.asarray(y, dtype=np.float64), np.asarray(w, dtype=np.float64)


def legendre(k, y):
    return eval_legendre(k, y)


def legendre_deriv(k, y):
    """d/dy P_k = (k + 1)/2 P_{k-1}^{(1,1)} (Jacobi derivative identity)."""
    if k == 0:
        return np.zeros_like(np.asarray(y, dtype=np.float64))
    return 0.5 * (k + 1) * eval_jacobi(k - 1, 1, 1, y)


def bubble(nb, y):
    """W_n of eq. (Wn)."""
    y = np.asarray(y, dtype=np.float64)
    return (1.0 - y * y) * eval_jacobi(nb, 1, 1, y) / (2.0 * (nb + 1))


def bubble_deriv(nb, y):
    """d/dy W_n from the product rule and d/dy P_n^{(1,1)} = (n+3)/2 P_{n-1}^{(2,2)}."""
    y = np.asarray(y, dtype=np.float64)
    jac = eval_jacobi(nb, 1, 1, y)
    djac = 0.5 * (nb + 3) * eval_jacobi(nb - 1, 2, 2, y) if nb >= 1 else 0.0 * y
    return (-2.0 * y * jac + (1.0 - y * y) * djac) / (2.0 * (nb + 1))


def spectral(nb, y):
    """Y_n = P_n - P_{n+2} (Section 3)."""
    return eval_legendre(nb, y) - eval_legendre(nb + 2, y)


def spectral_deriv(nb, y):
    return legendre_deriv(nb, y) - legendre_deriv(nb + 2, y)


def local_u_values(p, y):
    """Values of the p+1 local U-functions [hatL, hatR, W_0..W_{p-2}] at y: (p+1, len(y))."""
    y = np.asarray(y, dtype=np.float64)
    rows = [0.5 * (1.0 - y), 0.5 * (1.0 + y)]
    rows += [bubble(b, y) for b in range(p - 1)]
    return np.array(rows)


def local_u_derivs(p, y):
    """d/dy of the local U-functions: (p+1, len(y))."""
    y = np.asarray(y, dtype=np.float64)
    rows = [-0.5 * np.ones_like(y), 0.5 * np.ones_like(y)]
    rows += [bubble_deriv(b, y) for b in range(p - 1)]
    return np.array(rows)


def local_psi_values(n, y):
    """Values of P_0..P_{n-1} at y: (n, len(y))."""
    return np.array([legendre(k, y) for k in range(n)])


def local_psi_derivs(n, y):
    return np.array([legendre_deriv(k, y) for k in range(n)])


class Mesh1D:
    """Breakpoints a = x_0 < ... < x_m = b with uniform partial degree p."""

    def __init__(self, breakpoints, p):
        self.x = np.asarray(breakpoints, dtype=np.float64)
        self.m = len(self.x) - 1
        self.p = int(p)
        assert self.m >= 1 and self.p >= 1
        self.h = np.diff(self.x)
        self.N1 = self.m * self.p + 1

    def local_to_global(self, c):
        """Global indices of the local U-functions [hatL, hatR, W_0..W_{p-2}] of cell c."""
        m, p = self.m, self.p
        return np.array([c, c + 1] + [m + 1 + c * (p - 1) + b for b in range(p - 1)])

    def interior(self):
        """Interior (non-Dirichlet) 1D dofs in global order."""
        return np.array([i for i in range(self.N1) if i not in (0, self.m)])

    def boundary(self):
        return np.array([0, self.m])

    def to_physical(self, c, y):
        return self.x[c] + 0.5 * (np.asarray(y) + 1.0) * self.h[c]


def assemble_1d(mesh, n_psi):
    """1D global matrices over U_{h,p} (all N1 dofs) and Psi (m * n_psi dofs).

    Returns dict with sparse CSR matrices
      A  : (v_i', v_j')            stiffness, N1 x N1
      M  : (v_i, v_j)              mass,      N1 x N1
      B  : (v_i, zeta_k)           Gram U x Psi, N1 x (m n_psi)
      Bd : (v_i', zeta_k)          Gram of derivatives (gradient-type B), N1 x (m n_psi)
      Mpsi : (zeta_k, zeta_l)      Psi mass (diagonal by the Lemma), (m n_psi)^2
      Kpsi : (zeta_k', zeta_l')    broken H^1 seminorm on Psi (cellwise), (m n_psi)^2
    """
    yq, wq = gauss(QUAD_REF)
    p, m = mesh.p, mesh.m
    U = local_u_values(p, yq)
    dU = local_u_derivs(p, yq)
    P = local_psi_values(n_psi, yq)
    dP = local_psi_derivs(n_psi, yq)
    A = sp.lil_matrix((mesh.N1, mesh.N1))
    M = sp.lil_matrix((mesh.N1, mesh.N1))
    B = sp.lil_matrix((mesh.N1, m * n_psi))
    Bd = sp.lil_matrix((mesh.N1, m * n_psi))
    Mpsi = sp.lil_matrix((m * n_psi, m * n_psi))
    Kpsi = sp.lil_matrix((m * n_psi, m * n_psi))
    for c in range(m):
        h = mesh.h[c]
        J = 0.5 * h
        Kloc = (dU * wq) @ dU.T / J            # (2/h) int dU dU dy
        Mloc = (U * wq) @ U.T * J
        Bloc = (U * wq) @ P.T * J
        Bdloc = (dU * wq) @ P.T                 # int (dv/dy) zeta dy
        Mp = (P * wq) @ P.T * J
        Kp = (dP * wq) @ dP.T / J
        g = mesh.local_to_global(c)
        cols = c * n_psi + np.arange(n_psi)
        for a in range(p + 1):
            for b in range(p + 1):
                A[g[a], g[b]] += Kloc[a, b]
                M[g[a], g[b]] += Mloc[a, b]
            for k in range(n_psi):
                B[g[a], cols[k]] += Bloc[a, k]
                Bd[g[a], cols[k]] += Bdloc[a, k]
        for k in range(n_psi):
            for l in range(n_psi):
                Mpsi[cols[k], cols[l]] += Mp[k, l]
                Kpsi[cols[k], cols[l]] += Kp[k, l]
    return dict(A=A.tocsr(), M=M.tocsr(), B=B.tocsr(), Bd=Bd.tocsr(),
                Mpsi=Mpsi.tocsr(), Kpsi=Kpsi.tocsr())


def lifting_operator_1d(mesh, npts_cell=None):
    """1D Dirichlet lifting rule Pi as a linear map from samples to coefficients.

    Reading (the paper's examples all have homogeneous data): hats take the
    value of g at their vertex; on each cell the bubbles take the
    H^1_0-seminorm projection of r = g - (linear interpolant of g).  Because
    (W_a', W_b') = 2/(2b+3) delta_ab on the reference cell, that projection is
    diagonal: c_b = ((2b+3)/2) int r(y) P_{b+1}'(y) dy (integrated by parts
    from -((2b+3)/2) int r' P_{b+1}), evaluated with a (2p+2)-point Gauss rule.

    Returns (pts, Pi) where ``pts`` are the physical sample points (vertices
    first, then each cell's Gauss points) and ``Pi`` is (N1 x len(pts)).
    """
    p, m = mesh.p, mesh.m
    nq = npts_cell or (2 * p + 2)
    yq, wq = gauss(nq)
    pts = list(mesh.x)
    Pi = np.zeros((mesh.N1, m + 1 + m * nq))
    for j in range(m + 1):
        Pi[j, j] = 1.0
    for c in range(m):
        base = m + 1 + c * nq
        pts += list(mesh.to_physical(c, yq))
        for b in range(p - 1):
            row = m + 1 + c * (p - 1) + b
            wt = 0.5 * (2 * b + 3) * wq * legendre_deriv(b + 1, yq)
            # r(y_q) = g(y_q) - g(x_c)(1-y)/2 - g(x_{c+1})(1+y)/2
            Pi[row, base:base + nq] += wt
            Pi[row, c] -= np.sum(wt * 0.5 * (1.0 - yq))
            Pi[row, c + 1] -= np.sum(wt * 0.5 * (1.0 + yq))
    return np.array(pts), Pi


def evaluate_1d(mesh, coeffs, x):
    """Evaluate a U_{h,p} function with global coefficients at physical points x."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    c = np.clip(np.searchsorted(mesh.x, x, side="right") - 1, 0, mesh.m - 1)
    for cell in range(mesh.m):
        sel = c == cell
        if not np.any(sel):
            continue
        y = 2.0 * (x[sel] - mesh.x[cell]) / mesh.h[cell] - 1.0
        vals = local_u_values(mesh.p, y)
        out[sel] = coeffs[mesh.local_to_global(cell)] @ vals
    return out
