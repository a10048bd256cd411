"""Pins of the oracle's 1D bases and matrices against closed forms (Section 3).

The oracle computes every 1D integral by 64-point Gauss quadrature of
scipy.special evaluations; these tests check the results against closed
forms derived by hand from the definitions, so a wrong sign, index or
normalisation in the oracle fails here.
"""
import numpy as np
import pytest

from oracle import basis1d as b1
from oracle import schur as osch

Y = np.linspace(-1.0, 1.0, 41)


def test_gauss_rule_exactness():
    # n-point Gauss integrates degree 2n-1 exactly, and not degree 2n
    for n in range(1, 12):
        y, w = b1.gauss(n)
        for deg in range(2 * n):
            exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
            assert abs(np.sum(w * y ** deg) - exact) < 1e-13
        assert abs(np.sum(w * y ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-8


def test_bubble_derivative_is_minus_legendre():
    # eq. (Wn): normalisation chosen so that d/dx W_n = -P_{n+1}
    for nb in range(0, 15):
        assert np.allclose(b1.bubble_deriv(nb, Y), -b1.legendre(nb + 1, Y), atol=1e-12)
        assert abs(b1.bubble(nb, np.array([1.0]))[0]) < 1e-14
        assert abs(b1.bubble(nb, np.array([-1.0]))[0]) < 1e-14


def test_spectral_galerkin_is_rescaled_bubble():
    # Section 3: Y_n = (2n+3) W_n and Y_n(+-1) = 0
    for nb in range(0, 15):
        assert np.allclose(b1.spectral(nb, Y), (2 * nb + 3) * b1.bubble(nb, Y), atol=1e-12)


def test_legendre_orthogonality():
    y, w = b1.gauss(40)
    P = b1.local_psi_values(12, y)
    G = (P * w) @ P.T
    assert np.allclose(G, np.diag([2.0 / (2 * k + 1) for k in range(12)]), atol=1e-14)


@pytest.mark.parametrize("bp,p", [(np.linspace(0, 1, 4), 5), (np.array([-2.0, -0.5, 0.25, 1.0, 3.0]), 6)])
def test_1d_matrices_closed_forms(bp, p):
    mesh = b1.Mesh1D(bp, p)
    n = p - 1
    mt = b1.assemble_1d(mesh, n)
    A, M, B, Mp = (mt[k].toarray() for k in ("A", "M", "B", "Mpsi"))
    m = mesh.m
    A_ref = np.zeros_like(A)
    M_ref = np.zeros_like(M)
    B_ref = np.zeros_like(B)
    for c in range(m):
        h = mesh.h[c]
        g = mesh.local_to_global(c)
        hl, hr = g[0], g[1]
        # hats: (1/h)[[1,-1],[-1,1]] stiffness, (h/6)[[2,1],[1,2]] mass
        A_ref[np.ix_([hl, hr], [hl, hr])] += np.array([[1, -1], [-1, 1]]) / h
        M_ref[np.ix_([hl, hr], [hl, hr])] += np.array([[2, 1], [1, 2]]) * h / 6
        for a in range(p - 1):
            ia = g[2 + a]
            A_ref[ia, ia] += (2.0 / h) * 2.0 / (2 * a + 3)
            for b in range(p - 1):
                ib = g[2 + b]
                yab = 0.0
                if a == b:
                    yab = 2.0 / (2 * a + 1) + 2.0 / (2 * a + 5)
                elif b == a + 2:
                    yab = -2.0 / (2 * a + 5)
                elif a == b + 2:
                    yab = -2.0 / (2 * b + 5)
                M_ref[ia, ib] += 0.5 * h * yab / ((2 * a + 3) * (2 * b + 3))
            # hat-bubble mass: only W_0 (h/6, h/6) and W_1 (-h/30, +h/30)
            if a == 0:
                for hh in (hl, hr):
                    M_ref[hh, ia] += h / 6
                    M_ref[ia, hh] += h / 6
            if a == 1:
                M_ref[hl, ia] += -h / 30
                M_ref[ia, hl] += -h / 30
                M_ref[hr, ia] += h / 30
                M_ref[ia, hr] += h / 30
            # Gram (W_a, P_k): (h/2)/(2a+3) [2/(2a+1) d_{ka} - 2/(2a+5) d_{k,a+2}]
            for k in range(n):
                v = 0.0
                if k == a:
                    v = 2.0 / (2 * a + 1)
                elif k == a + 2:
                    v = -2.0 / (2 * a + 5)
                B_ref[ia, c * n + k] += 0.5 * h * v / (2 * a + 3)
        # hats against Legendre: only P_0 (h/2) and P_1 (-/+ h/6)
        B_ref[hl, c * n + 0] += h / 2
        B_ref[hr, c * n + 0] += h / 2
        if n > 1:
            B_ref[hl, c * n + 1] += -h / 6
            B_ref[hr, c * n + 1] += h / 6
    assert np.allclose(A, A_ref, atol=1e-13)
    assert np.allclose(M, M_ref, atol=1e-13)
    assert np.allclose(B, B_ref, atol=1e-13)
    # Lemma (diagonal mass matrix): (zeta_k, zeta_l) = |K| delta_kl / (2k+1), k the degree
    Mp_ref = np.diag(np.concatenate([[mesh.h[c] / (2 * k + 1) for k in range(n)] for c in range(m)]))
    assert np.allclose(Mp, Mp_ref, atol=1e-14)
    # exact sparsity: no entries beyond the closed forms
    for X, R in ((A, A_ref), (M, M_ref), (B, B_ref)):
        tol = 1e-11 * np.abs(R).max()
        assert np.all((np.abs(X) > tol) == (np.abs(R) > tol))


def test_sparsity_counts():
    # nnz of A, M, B grow as O(p/h) in 1D (Section 4.3)
    for m, p in [(3, 4), (8, 7), (16, 9)]:
        mesh = b1.Mesh1D(np.linspace(0, 1, m + 1), p)
        mt = b1.assemble_1d(mesh, p - 1)
        nnz = lambda X: int(np.sum(np.abs(X.toarray()) > 1e-11 * np.abs(X).max()))
        assert nnz(mt["A"]) == (3 * (m + 1) - 2) + m * (p - 1)
        # M: hat tridiagonal + 2 hats x {W_0, W_1} x 2 + bubbles (diag + |a-b| = 2 pairs)
        assert nnz(mt["M"]) == (3 * (m + 1) - 2) + m * (2 * 2 * min(2, p - 1)) + m * ((p - 1) + 2 * max(0, p - 3))
        # B: hats x {P_0, P_1}, bubbles x {P_a, P_{a+2}}
        n = p - 1
        assert nnz(mt["B"]) == m * (2 * min(2, n)) + m * sum(1 + (a + 2 < n) for a in range(p - 1))


def test_spectral_galerkin_cell_matrices():
    # (Y_a', Y_b')_K = (2/h) 2 (2a+3) delta_ab ; (Y_a, Y_b)_K non-zero only for |a-b| in {0,2}
    h, p = 0.3, 9
    KY, MY, BY = osch.spectral_cell_matrices(h, p)
    assert np.allclose(KY, np.diag([(2.0 / h) * 2.0 * (2 * a + 3) for a in range(p - 1)]), atol=1e-11)
    i, j = np.nonzero(np.abs(MY) > 1e-11 * np.abs(MY).max())
    assert set(np.abs(i - j).tolist()) == {0, 2}


def _spectral_closed_forms(h, p):
    """(Y_a', Y_b')_K, (Y_a, Y_b)_K, (Y_a, P_k)_K on a cell of width h, from
    Y_a = P_a - P_{a+2} and (P_a, P_b) = 2 delta_ab / (2a+1) on (-1, 1), scaled
    by dx = (h/2) dy and d/dx = (2/h) d/dy."""
    nb = p - 1
    KY = np.zeros((nb, nb))
    MY = np.zeros((nb, nb))
    BY = np.zeros((nb, nb))
    for a in range(nb):
        KY[a, a] = (2.0 / h) * 2.0 * (2 * a + 3)
        MY[a, a] = (h / 2.0) * (2.0 / (2 * a + 1) + 2.0 / (2 * a + 5))
        if a + 2 < nb:
            MY[a, a + 2] = MY[a + 2, a] = -(h / 2.0) * 2.0 / (2 * a + 5)
        BY[a, a] = (h / 2.0) * 2.0 / (2 * a + 1)
        if a + 2 < nb:
            BY[a, a + 2] = -(h / 2.0) * 2.0 / (2 * a + 5)
    return KY, MY, BY


def test_spectral_cell_matrices_closed_forms():
    # every entry of the three 1D cell matrices, on cells of several widths
    for h, p in [(0.3, 9), (1.7, 5), (2.0, 2)]:
        got = osch.spectral_cell_matrices(h, p)
        want = _spectral_closed_forms(h, p)
        for g, w in zip(got, want):
            assert np.allclose(g, w, atol=1e-12 * max(1.0, np.abs(w).max()), rtol=0)


@pytest.mark.parametrize("hs,p", [([0.3, 0.7], 5), ([0.25, 0.5], 8), ([0.4, 0.2, 0.9], 4)])
def test_shat_constant_block_against_closed_forms(hs, p):
    # C_K = B-hat^T A-hat_1^{-1} B-hat of eq. (schur-preconditioner) on one cell, built
    # entry by entry (x index fastest) from the closed forms, then one dense solve
    d, nb = len(hs), p - 1
    mats = [_spectral_closed_forms(h, p) for h in hs]
    idx = np.array(np.unravel_index(np.arange(nb ** d), (nb,) * d, order="F")).T   # x fastest
    N = nb ** d
    Ahat = np.zeros((N, N))
    Bhat = np.zeros((N, N))
    for I in range(N):
        for J in range(N):
            a, b = idx[I], idx[J]
            Bhat[I, J] = np.prod([mats[j][2][a[j], b[j]] for j in range(d)])
            for k in range(d):
                Ahat[I, J] += np.prod([mats[j][0 if j == k else 1][a[j], b[j]] for j in range(d)])
    C_want = Bhat.T @ np.linalg.solve(Ahat, Bhat)
    C_got, _, _ = osch.shat_constant_block(hs, p)
    assert np.allclose(C_got, C_want, atol=1e-12 * np.abs(C_want).max(), rtol=0)


def test_shat_parity_blocks_2d():
    # Section 4.5: A-hat has 4 blocks per 2D cell (parities of the two degrees)
    import scipy.sparse.csgraph as csg
    for p in (4, 5, 8):
        _, Ahat, _ = osch.shat_constant_block([0.5, 0.5], p)
        ncomp, _ = csg.connected_components(np.abs(Ahat) > 1e-11 * np.abs(Ahat).max(), directed=False)
        assert ncomp == 4
        _, Ahat3, _ = osch.shat_constant_block([0.5, 0.5, 0.5], p)
        ncomp3, _ = csg.connected_components(np.abs(Ahat3) > 1e-11 * np.abs(Ahat3).max(), directed=False)
        assert ncomp3 == 8


def test_lifting_reproduces_polynomials_1d():
    mesh = b1.Mesh1D(np.array([0.0, 0.3, 0.7, 1.2]), 5)
    pts, Pi = b1.lifting_operator_1d(mesh)
    coef = np.random.default_rng(1).normal(size=6)
    poly = lambda x: np.polyval(coef, x)            # degree 5 = p
    c = Pi @ poly(pts)
    xs = np.linspace(0, 1.2, 37)
    assert np.allclose(b1.evaluate_1d(mesh, c, xs), poly(xs), atol=1e-12)
