"""Pins of the oracle's nonlinear solve (eq. pG, eq. pG:gradient, eq. pG-matrix).

* Taylor test: the sparse Newton matrix is the derivative of the residual
  (||F(x + eps h) - F(x) - eps J h|| = O(eps^2)), obstacle and gradient.
* Brute force: the obstacle and gradient subproblems are saddle points of
  convex-concave functions; eliminating u gives a concave dual in psi whose
  maximiser (L-BFGS, no Newton, no G) must equal the Newton fixed point.
* eq. (schur2) with exact inner solves equals the direct solve of G.
* Feasibility by construction (eq. pG: u = phi - exp(-psi)) and the discrete
  invariant B^T u + (exp(-psi), zeta) = (phi, zeta) at convergence.
* alpha-schedule counts and mesh-independent Newton counts (Section 6.2:
  the Newton count does not depend on h and p).
* Closed form (radial obstacle): driving alpha higher, hpG approaches the
  closed-form solution, more closely on finer meshes; projected
  Gauss--Seidel on a p = 1 grid approaches the same solution.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse.linalg as spla

from paper_2412_13733_gb300 import workloads as W
from oracle.hpg import ObstacleOracle, alpha_schedule
from oracle.gradient import GradientOracle
from oracle.schur import SchurOracle
from oracle.pgs import pgs_obstacle


def _radial(m, p, beta=0.0):
    return ObstacleOracle([W.uniform(-2, 2, m)] * 2, p, W.zero_field, W.radial_phi, W.radial_exact,
                          beta=beta, lower=True)


def _taylor_slopes(F, J, x, h):
    r = []
    F0 = F(x)
    Jh = J @ h
    for eps in [1e-2, 5e-3, 2.5e-3, 1.25e-3]:
        r.append(np.linalg.norm(F(x + eps * h) - F0 - eps * Jh))
    r = np.array(r)
    return np.log(r[:-1] / r[1:]) / np.log(2.0)


@pytest.mark.parametrize("bps,p", [([np.linspace(0, 1, 3), np.linspace(0, 1, 4)], 4),
                                   ([np.linspace(0, 1, 3), np.linspace(0, 1, 2), np.linspace(0, 1, 3)], 3)])
def test_taylor_obstacle(bps, p):
    o = ObstacleOracle(bps, p, W.const_field(3.0), lambda X: 0.3 + 0.1 * X[:, 0], None, beta=0.0)
    rng = np.random.default_rng(0)
    ni = len(o.interior)
    u0 = o.ulift.copy()
    u0[o.interior] = 0.1 * rng.normal(size=ni)
    psi = 0.3 * rng.normal(size=o.sp.Npsi)
    psi_prev = 0.2 * rng.normal(size=o.sp.Npsi)
    alpha = 0.7

    def F(x):
        u = o.ulift.copy()
        u[o.interior] = x[:ni]
        return o.residual(u, x[ni:], psi_prev, alpha)

    x = np.concatenate([u0[o.interior], psi])
    J = o.jacobian(psi, alpha, beta=0.0)
    s = _taylor_slopes(F, J, x, rng.normal(size=x.size))
    assert np.all(s > 1.9), s


@pytest.mark.parametrize("bps,p", [([np.linspace(0, 1, 3)] * 2, 3),
                                   ([np.linspace(0, 1, 3), np.linspace(0, 1, 2), np.linspace(0, 1, 2)], 2)])
def test_taylor_gradient(bps, p):
    """2D and 3D (three psi components, the derivative Gram on each axis)."""
    o = GradientOracle(bps, p, W.const_field(8.0), W.torsion_phi, beta=0.0)
    rng = np.random.default_rng(1)
    ni = len(o.interior)
    psi = 0.5 * rng.normal(size=o.sp.Npsi)
    psi_prev = 0.2 * rng.normal(size=o.sp.Npsi)
    alpha = 0.3

    def F(x):
        u = np.zeros(o.sp.Nu)
        u[o.interior] = x[:ni]
        return o.residual(u, x[ni:], psi_prev, alpha)

    x = np.concatenate([0.1 * rng.normal(size=ni), psi])
    J = o.jacobian(psi, alpha, beta=0.0)
    s = _taylor_slopes(F, J, x, rng.normal(size=x.size))
    assert np.all(s > 1.9), s


@pytest.mark.parametrize("dim", [2, 3])
def test_subproblem_matches_dual_maximisation(dim):
    if dim == 2:
        o = _radial(2, 3, beta=1e-4)
    else:
        o = ObstacleOracle([np.linspace(0, 1, 3), np.linspace(0, 1, 2), np.linspace(0, 1, 3)], 3,
                           W.const_field(40.0), lambda X: 0.05 + 0.02 * X[:, 0], None, beta=1e-4)
    rng = np.random.default_rng(5)
    psi_prev = 0.3 * rng.normal(size=o.sp.Npsi)
    alpha = 0.05
    u0, psi0 = o.initial_state()
    u, psi, it, info = o.newton(u0, psi_prev.copy(), psi_prev, alpha, tol=1e-13)
    assert info["converged"]
    I = o.interior
    bnd = o.sp.boundary
    A00 = o.A00.tocsc()
    lu = spla.splu(A00)
    ug = o.ulift
    Ag = o.A[I][:, bnd] @ ug[bnd]
    Bg = o.B[bnd].T @ ug[bnd]
    S = o.sp

    def negdual(ps):
        r = alpha * Ag + o.B0 @ (ps - psi_prev) - alpha * o.bf[I]
        z = lu.solve(r)
        pq = ps.reshape(S.Nc, S.nloc) @ S.Vd.T
        e = S.wJ * np.exp(-pq)
        val = -0.5 / alpha * r @ z + (Bg - o.phiz) @ ps - e.sum()
        grad = -o.B0.T @ z / alpha + (Bg - o.phiz) + (e @ S.Vd).ravel()
        return -val, -grad

    res = so.minimize(negdual, psi_prev.copy(), jac=True, method="L-BFGS-B",
                      options=dict(gtol=1e-13, ftol=1e-16, maxiter=20000, maxcor=50))
    assert np.max(np.abs(res.x - psi)) < 1e-6 * max(1.0, np.abs(psi).max())


def test_gradient_subproblem_matches_dual_maximisation():
    """Gradient kind: the subproblem is the saddle point of
    alpha (a(u,u)/2 - (f,u)) + u^T B (psi - psi_prev) - H(psi), H(psi) = sum_q w_q |J| phi_q
    sqrt(1 + |psi_q|^2), whose psi-gradient is the projection of G(psi) in F_psi.  Eliminating u
    leaves the concave dual -r^T A^{-1} r / (2 alpha) - H(psi), r = alpha (f, v) - B (psi - psi_prev);
    its maximiser (L-BFGS, no Newton, no G) must equal the Newton fixed point."""
    o = GradientOracle([np.linspace(0, 1, 3)] * 2, 3, W.const_field(8.0), W.torsion_phi, beta=0.0)
    S = o.sp
    rng = np.random.default_rng(6)
    psi_prev = 0.3 * rng.normal(size=S.Npsi)
    alpha = 0.2
    u0, _ = o.initial_state()
    u, psi, it, info = o.newton(u0, psi_prev.copy(), psi_prev, alpha, tol=1e-13)
    assert info["converged"]
    I = o.interior
    lu = spla.splu(o.A00.tocsc())
    bf = o.bf[I]

    def negdual(ps):
        r = alpha * bf - o.B0 @ (ps - psi_prev)
        z = lu.solve(r)
        pq = o.gauss_values(ps)                              # (Nc, d, q)
        sq = np.sqrt(1.0 + np.sum(pq * pq, axis=1))          # (Nc, q)
        H = np.sum(S.wJ * o.phiq * sq)
        val = -0.5 / alpha * r @ z - H
        gH = np.einsum("cq,ckq,qj->ckj", S.wJ * o.phiq / sq, pq, S.Vd).ravel()
        grad = o.B0.T @ z / alpha - gH
        return -val, -grad

    res = so.minimize(negdual, psi_prev.copy(), jac=True, method="L-BFGS-B",
                      options=dict(gtol=1e-13, ftol=1e-16, maxiter=20000, maxcor=50))
    assert np.max(np.abs(res.x - psi)) < 1e-6 * max(1.0, np.abs(psi).max())
    # and u is the minimiser in u for that psi
    uu = lu.solve(alpha * bf - o.B0 @ (psi - psi_prev)) / alpha
    assert np.max(np.abs(uu - u[I])) < 1e-8 * max(1.0, np.abs(u[I]).max())


def test_schur_sequence_equals_direct_solve():
    o = _radial(3, 4, beta=1e-4)
    sch = SchurOracle(o)
    rng = np.random.default_rng(2)
    psi = 0.5 * rng.normal(size=o.sp.Npsi)
    alpha = 0.1
    G = o.jacobian(psi, alpha)
    ni = len(o.interior)
    b = rng.normal(size=G.shape[0])
    x = spla.spsolve(G, b)
    du, dpsi = sch.schur_solve(b[:ni], b[ni:], psi, alpha)
    assert np.allclose(np.concatenate([du, dpsi]), x, atol=1e-10 * np.abs(x).max())
    # S-hat blocks are symmetric negative definite
    blocks = sch.shat_blocks(psi, alpha)
    assert np.allclose(blocks, np.transpose(blocks, (0, 2, 1)), atol=1e-13)
    assert np.all(np.linalg.eigvalsh(blocks) < 0)


def test_feasibility_and_invariant():
    o = _radial(4, 4, beta=1e-4)
    w = W.workload("radial4")
    r = o.solve(w["alphas"])
    assert r["converged"]
    u = -r["u"]                                   # solved as -u <= -phi
    Fpsi = o.residual(u, r["psi"], r["psi"], w["alphas"][-1])[len(o.interior):]
    assert np.linalg.norm(Fpsi) < 1e-10
    # feasible reconstruction u~ = phi - exp(-psi) <= phi pointwise (any psi)
    pq = o.gauss_values(r["psi"])
    phiq = o.phi(o.sp.cell_points.reshape(-1, 2)).reshape(pq.shape)
    assert np.all(phiq - np.exp(-pq) < phiq)


def test_alpha_schedule_counts():
    assert len(alpha_schedule(2.0 ** -7, 2.0 ** -3)) == 10     # Sections 6.1-6.2
    assert len(alpha_schedule(2.0 ** -2, 2.0)) == 8            # Section 6.5 (paper prints "six")
    assert len(alpha_schedule(2.0 ** -7, 4.0)) == 20           # Section 6.3
    assert alpha_schedule(2.0 ** -7, 2.0 ** -3) == W.alpha_list(2.0 ** -7, 2.0 ** -3)


def test_newton_counts_mesh_independent():
    w = W.workload("radial4")
    totals = []
    for m, p in [(4, 4), (8, 4), (4, 7)]:
        r = _radial(m, p, beta=1e-4).solve(w["alphas"])
        assert r["converged"]
        totals.append(sum(r["newton"]))
    assert max(totals) - min(totals) <= 2, totals


@pytest.mark.slow
def test_closed_form_approached():
    alphas = alpha_schedule(2.0 ** -7, 2.0)
    errs = []
    for m, p in [(4, 4), (8, 4)]:
        o = _radial(m, p, beta=1e-4)
        r = o.solve(alphas)
        assert r["converged"]
        e, ref = o.sp.l2_error(r["u"], W.radial_exact)
        errs.append(e / ref)
    assert errs[1] < 0.5 * errs[0] and errs[1] < 1e-2, errs
    # p = 1 projected Gauss-Seidel on the same problem also approaches it
    x, U, _ = pgs_obstacle(-2.0, 2.0, 64, W.zero_field, W.radial_phi, W.radial_exact, lower=True)
    X, Y = np.meshgrid(x, x, indexing="ij")
    ex = W.radial_exact(np.stack([X.ravel(), Y.ravel()], 1)).reshape(X.shape)
    assert np.max(np.abs(U - ex)) < 2e-2


@pytest.mark.parametrize("dim", [2, 3])
def test_psi_elimination_equals_direct_solve(dim):
    """The block elimination of psi (used for the 3D workload, whose direct
    factorisation of G does not fit in host memory) solves the same system:
    its delta satisfies G delta = F to round-off and equals SuperLU on G, and a
    whole proximal loop run with it gives the same Newton counts and u."""
    bps = [np.linspace(0, 1, 3), np.linspace(0, 1, 4), np.linspace(0, 1, 3)][:dim]
    p = 4 if dim == 2 else 3
    args = (bps, p, W.const_field(20.0), lambda X: 0.2 + 0.1 * X[:, 0], None)
    o = ObstacleOracle(*args, beta=1e-3)
    oe = ObstacleOracle(*args, beta=1e-3, linear="eliminate_psi")
    rng = np.random.default_rng(5)
    psi = 0.4 * rng.normal(size=o.sp.Npsi)
    psi.reshape(o.sp.Nc, o.sp.nloc)[::2, 0] += 25.0   # strongly active cells: exp(-psi) ~ 1e-11
    alpha = 0.3
    G = o.jacobian(psi, alpha)
    F = rng.normal(size=G.shape[0])
    d_direct = o.newton_step(psi, alpha, F)
    d_elim = oe.newton_step(psi, alpha, F)
    assert np.linalg.norm(G @ d_elim - F) < 1e-13 * np.linalg.norm(F)
    assert np.max(np.abs(d_elim - d_direct)) < 1e-10 * np.abs(d_direct).max()
    alphas = alpha_schedule(2.0 ** -2, 1.0)
    r1 = o.solve(alphas)
    r2 = oe.solve(alphas)
    assert r1["converged"] and r2["converged"]
    assert r1["newton"] == r2["newton"]
    assert np.max(np.abs(r1["u"] - r2["u"])) < 1e-10 * np.abs(r1["u"]).max()
