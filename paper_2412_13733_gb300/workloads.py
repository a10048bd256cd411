"""Seeded synthetic workloads (problem data only; none of the method's arithmetic).

Both the CUDA path and the CPU oracle read their inputs from here, so that
each side sees the same f, phi, g, mesh, degree and alpha_k schedule.

Workloads (the paper measures on analytic PDE data; these are stand-ins of
the same kind and sizes):
  * ``radial``     -- 2D radially symmetric lower obstacle on (-2, 2)^2:
                      -Laplace(u) = 0, u >= phi, phi = sqrt(1 - r^2) for
                      r <= 0.9 else -1, Dirichlet data = the closed-form
                      solution.  4x4 cells p=4 (small) and 32x32 cells p=8.
  * ``sine3d``     -- 3D obstacle on (0,1)^3, f = 100, u = 0 on the boundary,
                      phi = 0.2 + 0.1 sin(2 pi x) sin(2 pi y) sin(2 pi z),
                      8x8x8 hexes, p = 6.
  * ``torsion``    -- 2D gradient constraint |grad u| <= phi on (0,1)^2,
                      f = 8, phi = 0.5 + 0.25 x_1, 16x16 cells, p = 10.
  * ``requests``   -- stream of seeded 2D obstacle requests on (0,1)^2
                      (f ~ U[1,50], phi = 0.3 + Gaussian bumps, m in 4..32,
                      p in 2..10) with Poisson arrival times.

Closed form of the radial obstacle (not in the paper; derived): outside the
contact disk u is radial and harmonic and vanishes at r = 2, so
u = -a ln(r/2).  C^1 contact with sqrt(1 - r^2) at r* gives
a = r*^2 / sqrt(1 - r*^2) and r*^2 (1 - ln(r*/2)) = 1, whose root in (0, 1)
is r* = 0.6979651482...
"""
import math

import numpy as np


# ----------------------------------------------------------------- radial
def _radial_rstar():
    lo, hi = 0.3, 0.99
    fn = lambda r: r * r * (1.0 - math.log(r / 2.0)) - 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if fn(lo) * fn(mid) <= 0.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


RADIAL_RSTAR = _radial_rstar()
RADIAL_A = RADIAL_RSTAR ** 2 / math.sqrt(1.0 - RADIAL_RSTAR ** 2)


def radial_phi(X):
    X = np.atleast_2d(X)
    r2 = X[:, 0] ** 2 + X[:, 1] ** 2
    out = np.full(X.shape[0], -1.0)
    inside = r2 <= 0.81
    out[inside] = np.sqrt(1.0 - r2[inside])
    return out


def radial_exact(X):
    X = np.atleast_2d(X)
    r = np.sqrt(X[:, 0] ** 2 + X[:, 1] ** 2)
    out = np.empty(X.shape[0])
    c = r <= RADIAL_RSTAR
    out[c] = np.sqrt(1.0 - r[c] ** 2)
    out[~c] = -RADIAL_A * np.log(r[~c] / 2.0)
    return out


def zero_field(X):
    return np.zeros(np.atleast_2d(X).shape[0])


def const_field(c):
    return lambda X: np.full(np.atleast_2d(X).shape[0], float(c))


def sine3d_phi(X):
    X = np.atleast_2d(X)
    return 0.2 + 0.1 * np.sin(2 * np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1]) * np.sin(2 * np.pi * X[:, 2])


def oscillatory_phi(X):
    from scipy.special import j0
    X = np.atleast_2d(X)
    return (1.0 + j0(20.0 * X[:, 0])) * (1.0 + j0(20.0 * X[:, 1]))


def torsion_phi(X):
    X = np.atleast_2d(X)
    return 0.5 + 0.25 * X[:, 0]


def thermoforming_phi0(X):
    """Original mould of Section 6.4 on (0,1)^d: 11/10 - 2 max_j |x_j - 1/2| + prod_j cos(8 pi x_j) / 10."""
    X = np.atleast_2d(X)
    return 1.1 - 2.0 * np.max(np.abs(X - 0.5), axis=1) + np.prod(np.cos(8 * np.pi * X), axis=1) / 10.0


def thermoforming_xi(X):
    """xi = prod_j sin(pi x_j) (Section 6.4)."""
    X = np.atleast_2d(X)
    return np.prod(np.sin(np.pi * X), axis=1)


def alpha_list(alpha1, cap):
    """alpha_1, sqrt(2) growth, capped; stops once alpha repeats (Sections 6.1, 6.3, 6.5)."""
    out = []
    k = 1
    while True:
        a = min(alpha1 * 2.0 ** (0.5 * (k - 1)), cap)
        out.append(a)
        if len(out) >= 2 and out[-1] == out[-2]:
            return out
        k += 1


def uniform(lo, hi, m):
    return np.linspace(lo, hi, m + 1)


def workload(name):
    """Problem description dict for a named workload."""
    if name in ("radial4", "radial32"):
        m, p = (4, 4) if name == "radial4" else (32, 8)
        return dict(name=name, kind="obstacle", lower=True, dim=2,
                    breakpoints=[uniform(-2.0, 2.0, m)] * 2, m=m, p=p,
                    f=zero_field, f_const=0.0, phi=radial_phi, g=radial_exact,
                    alphas=alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-10,
                    exact=radial_exact)
    if name in ("sine3d", "sine3d_small"):
        m, p = (8, 6) if name == "sine3d" else (2, 4)
        return dict(name=name, kind="obstacle", lower=False, dim=3,
                    breakpoints=[uniform(0.0, 1.0, m)] * 3, m=m, p=p,
                    f=const_field(100.0), f_const=100.0, phi=sine3d_phi, g=None,
                    alphas=alpha_list(2.0 ** -2, 2.0), beta=1e-5, tol=1e-10, exact=None)
    if name in ("torsion", "torsion_small"):
        m, p = (16, 10) if name == "torsion" else (4, 4)
        return dict(name=name, kind="gradient", lower=False, dim=2,
                    breakpoints=[uniform(0.0, 1.0, m)] * 2, m=m, p=p,
                    f=const_field(8.0), f_const=8.0, phi=torsion_phi, g=None,
                    alphas=alpha_list(2.0 ** -7, 4.0), beta=1e-14, tol=1e-10, exact=None)
    if name.startswith("oscillatory_p"):
        # Section 6.2's 2D example: (0,1)^2, 10 x 10 cells, f = 100,
        # phi = (1 + J_0(20 x)) (1 + J_0(20 y)), alpha_1 = 2^-7 growing by sqrt(2) to 2^-3,
        # beta = 1e-4 (the value of its Krylov runs); name "oscillatory_p{p}" picks the degree
        p = int(name[len("oscillatory_p"):])
        return dict(name=name, kind="obstacle", lower=False, dim=2,
                    breakpoints=[uniform(0.0, 1.0, 10)] * 2, m=10, p=p,
                    f=const_field(100.0), f_const=100.0, phi=oscillatory_phi, g=None,
                    alphas=alpha_list(2.0 ** -7, 2.0 ** -3), beta=1e-4, tol=1e-6, exact=None)
    if name.startswith("thermoforming_p"):
        # Section 6.4's QVI: (0,1)^2, 4 x 4 cells, f = 100, gamma = 1, g0 = 1/5,
        # alpha_1 = 2^-6 growing by 4 until alpha = 1, beta = 1e-6, H^1 tolerance 3e-3;
        # name "thermoforming_p{p}" picks the degree ("..._m{m}" the cells per side)
        parts = name[len("thermoforming_p"):].split("_m")
        p = int(parts[0])
        m = int(parts[1]) if len(parts) > 1 else 4
        return dict(name=name, kind="obstacle", lower=False, dim=2,
                    breakpoints=[uniform(0.0, 1.0, m)] * 2, m=m, p=p,
                    f=const_field(100.0), f_const=100.0, phi=thermoforming_phi0, g=None,
                    Phi0=thermoforming_phi0, xi=thermoforming_xi, gamma=1.0, g0=0.2,
                    alphas=[2.0 ** -6, 2.0 ** -4, 2.0 ** -2, 1.0], beta=1e-6, tol=1e-10, qvi_tol=3e-3, exact=None)
    if name.startswith("box3d_"):
        # Section 6.5's 3D solver study: (0,1)^3, f = 40, phi = 1, alpha_1 = 2^-2, cap 2,
        # beta = 1e-5; name "box3d_p{p}_m{m}" picks the degree and cells per side
        p, m = (int(t[1:]) for t in name.split("_")[1:3])
        return dict(name=name, kind="obstacle", lower=False, dim=3,
                    breakpoints=[uniform(0.0, 1.0, m)] * 3, m=m, p=p,
                    f=const_field(40.0), f_const=40.0, phi=const_field(1.0), g=None,
                    alphas=alpha_list(2.0 ** -2, 2.0), beta=1e-5, tol=1e-6, exact=None)
    raise KeyError(name)


# ----------------------------------------------------------------- requests
REQUEST_SEED = 20241213


def _bumps_phi(centres, amps, widths):
    def phi(X):
        X = np.atleast_2d(X)
        out = np.full(X.shape[0], 0.3)
        for c, a, w in zip(centres, amps, widths):
            d2 = (X[:, 0] - c[0]) ** 2 + (X[:, 1] - c[1]) ** 2
            out += a * np.exp(-d2 / (2.0 * w * w))
        return out
    return phi


def requests(count=512, seed=REQUEST_SEED, m_range=(4, 32), p_range=(2, 10)):
    """Seeded 2D obstacle requests on (0,1)^2 (u = 0 on the boundary).

    phi = 0.3 + sum_j a_j exp(-|x - c_j|^2 / (2 w_j^2)), 1..4 bumps with
    c_j ~ U[0,1]^2, a_j ~ U[-0.2, 0.2], w_j ~ U[0.05, 0.2]; bumps are redrawn
    from the same stream until min phi >= 0.05 on a 257^2 sample grid (phi
    must be non-negative on the boundary for the subproblems to be feasible).
    """
    rng = np.random.default_rng(seed)
    g = np.linspace(0.0, 1.0, 257)
    GX, GY = np.meshgrid(g, g, indexing="ij")
    grid = np.stack([GX.ravel(), GY.ravel()], axis=1)
    out = []
    for i in range(count):
        f = float(rng.uniform(1.0, 50.0))
        k = int(rng.integers(1, 5))
        while True:
            c = rng.uniform(0.0, 1.0, size=(k, 2))
            a = rng.uniform(-0.2, 0.2, size=k)
            w = rng.uniform(0.05, 0.2, size=k)
            phi = _bumps_phi(c, a, w)
            if phi(grid).min() >= 0.05:
                break
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        out.append(dict(name=f"req{i}", kind="obstacle", lower=False, dim=2,
                        breakpoints=[uniform(0.0, 1.0, m)] * 2, m=m, p=p,
                        f=const_field(f), f_const=f, phi=phi, g=None,
                        bumps=(c, a, w), alphas=alpha_list(2.0 ** -7, 2.0 ** -3),
                        beta=1e-4, tol=1e-10, exact=None))
    return out


def arrivals(count, rate, seed=REQUEST_SEED + 1):
    """Poisson arrival times (seconds) at the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
