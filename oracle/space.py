"""Tensor-product spaces U_{h,p} x Psi_{h,p} on quad/hex meshes (Sections 3-4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Orderings (shared *by specification* with the C ABI, not by code):
  * u: full tensor product of the 1D global numbering (hats 0..m, then
    bubbles cell-major), x index fastest.  Interior (unknown) dofs are those
    whose every 1D index is interior; they keep their relative global order.
  * psi: cell-major.  Cell c = c_x + m_x c_y (+ m_x m_y c_z); inside a cell the
    n^d Legendre coefficients are lexicographic with the x degree fastest.
    For the vector-valued (gradient-type) latent variable the layout is
    [cell][component][n^d].

Quadrature of the latent nonlinearity (Section 5, "Quadrature"): the paper
interpolates exp(-psi) (and exp(-psi) zeta_j) onto the Legendre basis at
unstated nodes.  Reading used here: the nodes are the q = n Gauss--Legendre
points per direction of each cell.  With those nodes the interpolatory rule
is identical to Gauss quadrature with q = n points (V^T W V = M because the
n-point rule integrates degree 2n - 1 exactly), so
    (exp(-psi), zeta_i)_K       = sum_q w_q |J_K| exp(-psi(x_q)) zeta_i(x_q)
    (zeta_i, exp(-psi) zeta_j)_K = sum_q w_q |J_K| exp(-psi(x_q)) zeta_i zeta_j
The data term (phi, zeta) uses the same rule; (f, v) uses p+2 Gauss points.
"""
import numpy as np
import scipy.sparse as sp

from . import basis1d as b1


def kron_list(mats):
    """kron(mats[d-1], ..., mats[0]) so that direction 0 (x) is the fastest index."""
    out = None
    for M in mats:
        out = M if out is None else sp.kron(M, out, format="csr")
    return sp.csr_matrix(out)


def kron_dense(mats):
    out = None
    for M in mats:
        out = M if out is None else np.kron(M, out)
    return out


class TensorSpace:
    """U_{h,p} (continuous, degree p) x Psi (discontinuous Legendre, n per direction).

    ``kind`` = "obstacle": n = p - 1 (psi of degree p-2, Section 4.1);
               "gradient": n = p     (psi of degree p-1, Section 4.2), d components.
    """

    def __init__(self, breakpoints, p, kind="obstacle"):
        self.d = len(breakpoints)
        self.p = int(p)
        self.kind = kind
        self.n = self.p - 1 if kind == "obstacle" else self.p
        if kind == "obstacle":
            assert self.p >= 2, "obstacle pairing needs p >= 2 (Section 4.1)"
        self.meshes = [b1.Mesh1D(bp, p) for bp in breakpoints]
        self.m = [ms.m for ms in self.meshes]
        self.N1 = [ms.N1 for ms in self.meshes]
        self.Nu = int(np.prod(self.N1))
        self.Nc = int(np.prod(self.m))
        self.ncomp = 1 if kind == "obstacle" else self.d
        self.nloc = self.n ** self.d
        self.Npsi = self.Nc * self.ncomp * self.nloc
        self.mats1d = [b1.assemble_1d(ms, self.n) for ms in self.meshes]
        self._build_indices()
        self._build_operators()
        self._build_quadrature()

    # ------------------------------------------------------------------ indices
    def _build_indices(self):
        # full index = i_0 + N1_0 (i_1 + N1_1 i_2)
        interior_1d = [ms.interior() for ms in self.meshes]
        mask = np.ones(self.Nu, dtype=bool)
        idx = np.arange(self.Nu)
        rem = idx.copy()
        for j in range(self.d):
            ij = rem % self.N1[j]
            rem //= self.N1[j]
            mask &= np.isin(ij, interior_1d[j])
        self.interior = idx[mask]
        self.boundary = idx[~mask]
        # psi permutation: Kronecker order -> cell-major
        n, d = self.n, self.d
        npsi1 = [mj * n for mj in self.m]
        nkron = int(np.prod(npsi1))
        J = np.arange(nkron)
        rem = J.copy()
        cell = np.zeros(nkron, dtype=np.int64)
        loc = np.zeros(nkron, dtype=np.int64)
        cstride, kstride = 1, 1
        for j in range(d):
            jj = rem % npsi1[j]
            rem //= npsi1[j]
            cj, kj = jj // n, jj % n
            cell += cj * cstride
            loc += kj * kstride
            cstride *= self.m[j]
            kstride *= n
        self.kron_to_cell = cell * self.nloc + loc     # cell-major index of Kronecker index J

    def perm_cols(self, Bkron):
        """Reorder columns of a (rows x psi-Kronecker) matrix into cell-major order."""
        P = sp.csr_matrix((np.ones(len(self.kron_to_cell)),
                           (np.arange(len(self.kron_to_cell)), self.kron_to_cell)),
                          shape=(len(self.kron_to_cell), self.Nc * self.nloc))
        return sp.csr_matrix(Bkron @ P)

    # ---------------------------------------------------------------- operators
    def _build_operators(self):
        d = self.d
        A1 = [mt["A"] for mt in self.mats1d]
        M1 = [mt["M"] for mt in self.mats1d]
        B1 = [mt["B"] for mt in self.mats1d]
        Bd1 = [mt["Bd"] for mt in self.mats1d]
        self.A = sum(kron_list([A1[j] if j == k else M1[j] for j in range(d)]) for k in range(d))
        self.M = kron_list(M1)
        if self.kind == "obstacle":
            self.B = self.perm_cols(kron_list(B1))
        else:
            comps = [self.perm_cols(kron_list([Bd1[j] if j == k else B1[j] for j in range(d)]))
                     for k in range(d)]
            # [cell][component][n^d]: interleave the component blocks cell by cell
            blocks = []
            for c in range(self.Nc):
                for k in range(d):
                    blocks.append(comps[k][:, c * self.nloc:(c + 1) * self.nloc])
            self.B = sp.hstack(blocks, format="csr")
        # Psi mass and broken H^1 seminorm, cell-major, per component
        Mp1 = [mt["Mpsi"] for mt in self.mats1d]
        Kp1 = [mt["Kpsi"] for mt in self.mats1d]
        Mk = kron_list(Mp1)
        Kk = sum(kron_list([Kp1[j] if j == k else Mp1[j] for j in range(d)]) for k in range(d))
        P = self.perm_cols(sp.identity(Mk.shape[0], format="csr"))
        Mcell = sp.csr_matrix(P.T @ Mk @ P)
        Kcell = sp.csr_matrix(P.T @ Kk @ P)
        if self.ncomp == 1:
            self.Mpsi, self.Kpsi = Mcell, Kcell
        else:
            self.Mpsi = self._expand_components(Mcell)
            self.Kpsi = self._expand_components(Kcell)

    def _expand_components(self, Mcell):
        """Block-diagonal per component in the [cell][component][n^d] layout."""
        nl, nc = self.nloc, self.ncomp
        blocks = []
        for c in range(self.Nc):
            blk = Mcell[c * nl:(c + 1) * nl, c * nl:(c + 1) * nl]
            for _ in range(nc):
                blocks.append(blk)
        return sp.block_diag(blocks, format="csr")

    # --------------------------------------------------------------- quadrature
    def _build_quadrature(self):
        n = self.n
        yq, wq = b1.gauss(n)
        V1 = b1.local_psi_values(n, yq).T          # (q, n): P_k(y_q)
        self.q = n
        self.Vd = kron_dense([V1] * self.d)         # (q^d, n^d)
        self.wref = kron_dense([wq[:, None]] * self.d).ravel()   # (q^d,)
        self.cell_detJ = np.zeros(self.Nc)
        self.cell_points = np.zeros((self.Nc, n ** self.d, self.d))
        for c in range(self.Nc):
            cidx = self.cell_multi(c)
            det = 1.0
            coords = []
            for j in range(self.d):
                ms = self.meshes[j]
                det *= 0.5 * ms.h[cidx[j]]
                coords.append(ms.to_physical(cidx[j], yq))
            self.cell_detJ[c] = det
            G = np.meshgrid(*coords, indexing="ij")      # G[j][i_0, i_1, ...]
            # flatten with x fastest: transpose axes so that axis 0 is slowest
            pts = np.stack([g.transpose(tuple(range(self.d))[::-1]).ravel() for g in G], axis=1)
            self.cell_points[c] = pts
        self.wJ = self.cell_detJ[:, None] * self.wref[None, :]    # (Nc, q^d)

    def cell_multi(self, c):
        out = []
        for j in range(self.d):
            out.append(c % self.m[j])
            c //= self.m[j]
        return out

    # ------------------------------------------------------------- data terms
    def project_gauss(self, vals):
        """Cellwise V^T (w |J| vals): (Nc, q^d) -> cell-major (Nc n^d) vector."""
        return (self.wJ * vals) @ self.Vd

    def phi_zeta(self, phi):
        """(phi, zeta) by the q = n Gauss rule; phi(X) takes an (N, d) array."""
        vals = phi(self.cell_points.reshape(-1, self.d)).reshape(self.Nc, -1)
        return self.project_gauss(vals).ravel()

    def f_load(self, f):
        """(f, v_i) for every full u dof, with p+2 Gauss points per direction per cell."""
        nq = self.p + 2
        yq, wq = b1.gauss(nq)
        Uq = b1.local_u_values(self.p, yq)          # (p+1, nq)
        out = np.zeros(self.Nu)
        for c in range(self.Nc):
            cidx = self.cell_multi(c)
            coords, det, l2g = [], 1.0, []
            for j in range(self.d):
                ms = self.meshes[j]
                coords.append(ms.to_physical(cidx[j], yq))
                det *= 0.5 * ms.h[cidx[j]]
                l2g.append(ms.local_to_global(cidx[j]))
            G = np.meshgrid(*coords, indexing="ij")
            X = np.stack([g.ravel() for g in G], axis=1)          # C order: axis 0 slowest?
            fv = np.asarray(f(X), dtype=np.float64).reshape([nq] * self.d)  # indexed [i_0, i_1, ...]
            T = fv * det
            # contract each direction j with (Uq * wq)
            for j in range(self.d):
                T = np.tensordot(Uq * wq, T, axes=([1], [j]))     # new axis 0 = local fn of dir j
                T = np.moveaxis(T, 0, j)
            # T[a_0, a_1, ...] -> global
            gl = np.zeros_like(T, dtype=np.int64)
            mesh_idx = np.meshgrid(*l2g, indexing="ij")
            stride = 1
            for j in range(self.d):
                gl += mesh_idx[j] * stride
                stride *= self.N1[j]
            np.add.at(out, gl.ravel(), T.ravel())
        return out

    def lifting(self, g):
        """Full u vector whose boundary entries realise the Dirichlet datum g.

        Rule (reading; the paper's examples are homogeneous): the tensor
        product of the 1D operator Pi of ``basis1d.lifting_operator_1d``
        applied to samples of g; only the boundary entries are kept.  On a
        boundary face the 1D Pi of the normal direction selects the vertex
        value, so the coefficient depends on g restricted to the face only.
        """
        u = np.zeros(self.Nu)
        if g is None:
            return u
        ops = [b1.lifting_operator_1d(ms) for ms in self.meshes]
        pts = [o[0] for o in ops]
        G = np.meshgrid(*pts, indexing="ij")
        X = np.stack([gg.ravel() for gg in G], axis=1)
        S = np.asarray(g(X), dtype=np.float64).reshape([len(p_) for p_ in pts])
        T = S
        for j in range(self.d):
            T = np.tensordot(ops[j][1], T, axes=([1], [j]))
            T = np.moveaxis(T, 0, j)
        # T indexed [i_0, i_1, ...]; full index has i_0 fastest -> ravel in Fortran order
        coef = T.ravel(order="F")
        u[self.boundary] = coef[self.boundary]
        return u

    # -------------------------------------------------------------- evaluation
    def evaluate(self, ufull, X):
        """u_h at physical points X (N, d)."""
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        N = X.shape[0]
        cells, ys = [], []
        for j in range(self.d):
            ms = self.meshes[j]
            c = np.clip(np.searchsorted(ms.x, X[:, j], side="right") - 1, 0, ms.m - 1)
            cells.append(c)
            ys.append(2.0 * (X[:, j] - ms.x[c]) / ms.h[c] - 1.0)
        out = np.zeros(N)
        for i in range(N):
            vals = [b1.local_u_values(self.p, np.array([ys[j][i]]))[:, 0] for j in range(self.d)]
            l2g = [self.meshes[j].local_to_global(cells[j][i]) for j in range(self.d)]
            T = ufull[self._global_grid(l2g)]
            for j in range(self.d):
                T = np.tensordot(vals[j], T, axes=([0], [0]))
            out[i] = T
        return out

    def _global_grid(self, l2g):
        mesh_idx = np.meshgrid(*l2g, indexing="ij")
        gl = np.zeros_like(mesh_idx[0])
        stride = 1
        for j in range(self.d):
            gl = gl + mesh_idx[j] * stride
            stride *= self.N1[j]
        return gl

    def l2_error(self, ufull, uexact, extra=3):
        """(||u_h - u*||_{L2}, ||u*||_{L2}) with (p + extra) Gauss points per direction per cell."""
        nq = self.p + extra
        yq, wq = b1.gauss(nq)
        Uq = b1.local_u_values(self.p, yq)
        err2, ref2 = 0.0, 0.0
        for c in range(self.Nc):
            cidx = self.cell_multi(c)
            coords, det, l2g = [], 1.0, []
            for j in range(self.d):
                ms = self.meshes[j]
                coords.append(ms.to_physical(cidx[j], yq))
                det *= 0.5 * ms.h[cidx[j]]
                l2g.append(ms.local_to_global(cidx[j]))
            T = ufull[self._global_grid(l2g)]
            for j in range(self.d):
                T = np.tensordot(Uq, T, axes=([0], [j]))
                T = np.moveaxis(T, 0, j)
            G = np.meshgrid(*coords, indexing="ij")
            X = np.stack([gg.ravel() for gg in G], axis=1)
            ue = np.asarray(uexact(X)).reshape([nq] * self.d)
            W = det
            for j in range(self.d):
                shape = [1] * self.d
                shape[j] = nq
                W = W * wq.reshape(shape)
            err2 += np.sum(W * (T - ue) ** 2)
            ref2 += np.sum(W * ue ** 2)
        return np.sqrt(err2), np.sqrt(ref2)
