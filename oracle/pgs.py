"""Projected Gauss--Seidel for the classical low-order obstacle discretisation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A brute-force cross-check that is independent of the hierarchical basis:
the 5-point finite-difference Laplacian on a uniform N x N grid of a
rectangle, nodal constraint u >= phi (lower) or u <= phi (upper), Dirichlet
data g, solved by red-black projected successive over-relaxation until the
update stalls.  It solves a *different* discretisation (p = 1, nodal
constraint), so it only shares the continuous limit with hpG.
"""
import numpy as np


def pgs_obstacle(lo, hi, N, f, phi, g, lower=True, omega=1.9, tol=1e-13, max_sweeps=200000):
    x = np.linspace(lo, hi, N + 1)
    h = x[1] - x[0]
    X, Yg = np.meshgrid(x, x, indexing="ij")
    P = np.stack([X.ravel(), Yg.ravel()], axis=1)
    F = f(P).reshape(X.shape)
    Phi = phi(P).reshape(X.shape)
    U = np.zeros_like(X)
    G = g(P).reshape(X.shape)
    U[0, :], U[-1, :], U[:, 0], U[:, -1] = G[0, :], G[-1, :], G[:, 0], G[:, -1]
    inner = np.zeros_like(X, dtype=bool)
    inner[1:-1, 1:-1] = True
    I, J = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    colors = [inner & ((I + J) % 2 == c) for c in (0, 1)]
    U[inner] = np.maximum(U[inner], Phi[inner]) if lower else np.minimum(U[inner], Phi[inner])
    for sweep in range(max_sweeps):
        change = 0.0
        for mask in colors:
            nb = np.zeros_like(U)
            nb[1:-1, 1:-1] = U[:-2, 1:-1] + U[2:, 1:-1] + U[1:-1, :-2] + U[1:-1, 2:]
            gs = 0.25 * (nb + h * h * F)
            new = U + omega * (gs - U)
            new = np.maximum(new, Phi) if lower else np.minimum(new, Phi)
            change = max(change, float(np.max(np.abs(new[mask] - U[mask]))))
            U[mask] = new[mask]
        if change < tol:
            break
    return x, U, sweep + 1
