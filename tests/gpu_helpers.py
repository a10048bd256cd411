"""Shared helpers of the GPU parity tests: build the same problem for the CUDA
path (through the C ABI) and for the CPU oracle from one workload description."""
import numpy as np

from paper_2412_13733_gb300 import workloads as W


def case(name):
    """Small problems that span several cells, ragged tails and every kind."""
    if name == "radial_3x3_p5":
        w = W.workload("radial4")
        w.update(breakpoints=[W.uniform(-2, 2, 3)] * 2, p=5, m=3)
        return w
    if name == "radial4":
        return W.workload("radial4")
    if name == "aniso_upper":
        return dict(name=name, kind="obstacle", lower=False, dim=2,
                    breakpoints=[W.uniform(0.0, 2.0, 5), W.uniform(-0.5, 0.5, 3)], p=4,
                    f=W.const_field(7.0), f_const=7.0, phi=lambda X: 0.2 + 0.1 * np.sin(3 * X[:, 0]) * X[:, 1],
                    g=None, alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10)
    if name == "p2":
        return dict(name=name, kind="obstacle", lower=False, dim=2, breakpoints=[W.uniform(0, 1, 6)] * 2, p=2,
                    f=W.const_field(20.0), f_const=20.0, phi=lambda X: 0.05 + 0.0 * X[:, 0], g=None,
                    alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10)
    if name == "single_cell":
        return dict(name=name, kind="obstacle", lower=False, dim=2, breakpoints=[W.uniform(0, 1, 1)] * 2, p=6,
                    f=W.const_field(30.0), f_const=30.0, phi=lambda X: 0.1 + 0.05 * X[:, 0], g=None,
                    alphas=W.alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10)
    if name == "sine3d_small":
        return W.workload("sine3d_small")
    if name == "sine3d_3x2x2":
        w = W.workload("sine3d_small")
        w.update(breakpoints=[W.uniform(0, 1, 3), W.uniform(0, 1, 2), W.uniform(0, 1, 2)], p=3)
        return w
    if name == "torsion_small":
        return W.workload("torsion_small")
    if name == "torsion_3x3_p3":
        w = W.workload("torsion_small")
        w.update(breakpoints=[W.uniform(0, 1, 3)] * 2, p=3)
        return w
    if name == "grad3d_2x3x2_p3":
        # gradient constraint in 3D: three psi components, derivative Grams on every axis
        w = W.workload("torsion_small")
        w.update(name=name, dim=3, breakpoints=[W.uniform(0, 1, 2), W.uniform(0, 1, 3), W.uniform(0, 1, 2)], p=3)
        return w
    if name == "radial_2x2_p16":
        # high degree: 15 x 15 latent coefficients per cell (nb = 225, block factorisation)
        w = W.workload("radial4")
        w.update(name=name, breakpoints=[W.uniform(-2, 2, 2)] * 2, p=16, m=2)
        return w
    if name == "torsion_2x2_p12":
        w = W.workload("torsion_small")
        w.update(name=name, breakpoints=[W.uniform(0, 1, 2)] * 2, p=12)
        return w
    if name == "sine3d_1x1x2_p9":
        w = W.workload("sine3d_small")
        w.update(name=name, breakpoints=[W.uniform(0, 1, 1), W.uniform(0, 1, 1), W.uniform(0, 1, 2)], p=9)
        return w
    if name.startswith("box3d_"):
        w = W.workload(name)
        w["tol"] = 1e-10          # parity gates at the usual Newton tolerance
        return w
    raise KeyError(name)


def oracle_for(w):
    from oracle.hpg import ObstacleOracle
    from oracle.gradient import GradientOracle
    if w["kind"] == "gradient":
        return GradientOracle(w["breakpoints"], w["p"], w["f"], w["phi"], beta=w["beta"])
    return ObstacleOracle(w["breakpoints"], w["p"], w["f"], w["phi"], w.get("g"), beta=w["beta"],
                          lower=w.get("lower", False))


def random_state(o, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    u, _ = o.initial_state()
    u = u.copy()
    u[o.interior] = 0.1 * rng.normal(size=len(o.interior))
    psi = scale * rng.normal(size=o.sp.Npsi)
    psi_prev = 0.5 * scale * rng.normal(size=o.sp.Npsi)
    return u, psi, psi_prev


def mass_norm(o, v):
    """L2 norm of the U_{h,p} function with full coefficients v."""
    return float(np.sqrt(max(v @ (o.sp.M @ v), 0.0)))


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_entry(a, b):
    """The larger of the relative l2 error and the largest entry error over the largest
    entry: an error that sits in a few entries (a boundary row, a ragged tile) must also stay
    below the tolerance."""
    a = np.asarray(a)
    b = np.asarray(b)
    mx = float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if b.size else 0.0
    return max(rel(a, b), mx)
