"""Pins of the oracle's tensor-product operators, loads, lifting and quadrature.

* Manufactured solution: with psi fixed the u-equation is Galerkin Poisson,
  which reproduces any u* in U_{h,p} exactly (to round-off).  This pins A,
  the load (f, v), the Dirichlet lifting and the orderings in 2D and 3D.
* Constant psi = c: D_psi = exp(-c) M_Psi and (exp(-psi), zeta) = exp(-c)|K| delta_{k0}.
* Gauss rule with q = n points: V^T W V = M_Psi (the quadrature reading).
* B = Kronecker product of 1D Gram matrices, checked entry-wise against a
  direct tensor quadrature of (v_i, zeta_j) on random entries.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import basis1d as b1
from oracle.space import TensorSpace


def _poly_field(d, p, seed):
    rng = np.random.default_rng(seed)
    C = rng.normal(size=[p + 1] * d)

    def u(X):
        X = np.atleast_2d(X)
        out = np.zeros(X.shape[0])
        for idx in np.ndindex(*C.shape):
            term = C[idx] * np.ones(X.shape[0])
            for j in range(d):
                term = term * X[:, j] ** idx[j]
            out += term
        return out

    def lap(X):
        X = np.atleast_2d(X)
        out = np.zeros(X.shape[0])
        for idx in np.ndindex(*C.shape):
            for k in range(d):
                if idx[k] < 2:
                    continue
                term = C[idx] * idx[k] * (idx[k] - 1) * np.ones(X.shape[0])
                for j in range(d):
                    e = idx[j] - 2 if j == k else idx[j]
                    term = term * X[:, j] ** e
                out += term
        return out

    return u, lambda X: -lap(X)


@pytest.mark.parametrize("d,m,p", [(2, 3, 4), (2, 2, 6), (3, 2, 3)])
def test_manufactured_poisson_exact(d, m, p):
    bps = [np.sort(np.concatenate([[0.0, 1.0], np.random.default_rng(j).uniform(0.1, 0.9, m - 1)]))
           for j in range(d)]
    S = TensorSpace(bps, p)
    ustar, f = _poly_field(d, p, seed=7)
    ul = S.lifting(ustar)
    bf = S.f_load(f)
    I = S.interior
    A00 = S.A[I][:, I]
    rhs = bf[I] - S.A[I] @ ul
    u = ul.copy()
    u[I] = spla.spsolve(A00.tocsc(), rhs)
    X = np.random.default_rng(3).uniform(0, 1, size=(25, d))
    assert np.max(np.abs(S.evaluate(u, X) - ustar(X))) < 1e-9 * max(1.0, np.abs(ustar(X)).max())


def test_constant_psi_gives_scaled_mass():
    S = TensorSpace([np.linspace(0, 2, 4), np.linspace(-1, 1, 3)], 5)
    c = 0.37
    psi = np.zeros(S.Npsi)
    psi.reshape(S.Nc, S.nloc)[:, 0] = c                      # P_0 coefficient = constant c
    pq = psi.reshape(S.Nc, S.nloc) @ S.Vd.T
    assert np.allclose(pq, c)
    gw = S.wJ * np.exp(-pq)
    D = np.einsum("qi,cq,qj->cij", S.Vd, gw, S.Vd)
    Mblocks = np.array([S.Mpsi[k * S.nloc:(k + 1) * S.nloc, k * S.nloc:(k + 1) * S.nloc].toarray()
                        for k in range(S.Nc)])
    assert np.allclose(D, np.exp(-c) * Mblocks, atol=1e-14)
    eg = gw @ S.Vd
    assert np.allclose(eg[:, 0], np.exp(-c) * 4 * S.cell_detJ)   # |K| = 2^d det J
    assert np.allclose(eg[:, 1:], 0.0, atol=1e-14)


def test_gauss_n_points_reproduce_psi_mass():
    # V^T W V = M exactly with n points (degree 2n-2 integrands), Section 5 quadrature reading
    for n in range(1, 11):
        y, w = b1.gauss(n)
        V = b1.local_psi_values(n, y).T
        assert np.allclose(V.T @ (w[:, None] * V), np.diag([2.0 / (2 * k + 1) for k in range(n)]), atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_B_matches_direct_tensor_quadrature(d):
    m, p = 2, 4
    S = TensorSpace([np.linspace(0, 1, m + 1)] * d, p)
    rng = np.random.default_rng(11)
    yq, wq = b1.gauss(20)
    for _ in range(12):
        c = int(rng.integers(S.Nc))
        k = [int(v) for v in rng.integers(0, S.n, size=d)]
        cm = S.cell_multi(c)
        # pick a u dof that touches this cell
        l2g = [S.meshes[j].local_to_global(cm[j]) for j in range(d)]
        a = [int(rng.integers(0, p + 1)) for _ in range(d)]
        gi = sum(l2g[j][a[j]] * int(np.prod(S.N1[:j])) for j in range(d))
        val = 1.0
        for j in range(d):
            h = S.meshes[j].h[cm[j]]
            val *= 0.5 * h * np.sum(wq * b1.local_u_values(p, yq)[a[j]] * b1.legendre(k[j], yq))
        col = c * S.nloc + sum(k[j] * S.n ** j for j in range(d))
        assert abs(S.B[gi, col] - val) < 1e-13
