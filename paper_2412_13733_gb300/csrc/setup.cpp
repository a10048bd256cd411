// Host-side setup of libhpg: 1D hierarchical bases (Section 3), their matrices
// in closed form, the fast-diagonalisation eigenpairs of the 1D stiffness/mass
// pencil, the constant part of the S-hat cell blocks (Section 4.5), data loads
// and the Dirichlet lifting.  Everything here runs once per problem.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "hpg_internal.h"

namespace hpg {

void Ell::add(int r, int c, double v) {
    if (v == 0.0) return;
    for (int e = 0; e < cnt[r]; ++e)
        if (col[(size_t)r * kEll + e] == c) { val[(size_t)r * kEll + e] += v; return; }
    if (cnt[r] >= kEll) throw std::runtime_error("stencil wider than kEll");
    col[(size_t)r * kEll + cnt[r]] = c;
    val[(size_t)r * kEll + cnt[r]] = v;
    cnt[r]++;
}

// ------------------------------------------------------------ Gauss, Legendre
void legendre_all(int kmax, double y, double* P, double* dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (kmax >= 1) { P[1] = y; dP[1] = 1.0; }
    for (int k = 1; k < kmax; ++k) {
        P[k + 1] = ((2.0 * k + 1.0) * y * P[k] - k * P[k - 1]) / (k + 1.0);
        dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
    }
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    std::vector<double> P(n + 1), dP(n + 1);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            legendre_all(n, z, P.data(), dP.data());
            double dz = P[n] / dP[n];
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        legendre_all(n, z, P.data(), dP.data());
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP[n] * dP[n]);
    }
}

// ------------------------------------------------------------ dense algebra
bool cholesky(int n, std::vector<double>& A) {
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        double ljj = std::sqrt(s);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / ljj;
        }
        for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = 0.0;
    }
    return true;
}

// Householder reduction to tridiagonal form followed by the implicit QL
// iteration with Wilkinson-type shifts; eigenvectors accumulated in Z.  The QL
// sweep is the textbook method of Bowdler, Martin, Reinsch and Wilkinson, "The QR
// and QL algorithms for symmetric matrices", Numer. Math. 11 (1968) 293-306
// (procedure tql2 of the Handbook for Automatic Computation, Vol. II), whose
// step order it keeps: shift from the leading 2x2 block, chase of the bulge by
// plane rotations, deflation when an off-diagonal entry falls below round-off.
bool symmetric_eigen(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& Z) {
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    auto z = [&](int i, int j) -> double& { return Z[(size_t)i * n + j]; };
    std::vector<double> v(n), q(n);
    for (int k = 0; k + 2 < n; ++k) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += a(i, k) * a(i, k);
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        double x0 = a(k + 1, k);
        double r = x0 >= 0 ? -alpha : alpha;        // new subdiagonal entry
        // v = x - r e1
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        for (int i = k + 1; i < n; ++i) v[i] = a(i, k);
        v[k + 1] -= r;
        double vtv = 0.0;
        for (int i = k + 1; i < n; ++i) vtv += v[i] * v[i];
        if (vtv == 0.0) continue;
        double tau = 2.0 / vtv;
        // q = tau A v - (tau^2/2)(v^T A v) v  over the trailing block
        for (int i = k + 1; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
            q[i] = tau * s;
        }
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) K += v[i] * q[i];
        K *= 0.5 * tau;
        for (int i = k + 1; i < n; ++i) q[i] -= K * v[i];
        for (int i = k + 1; i < n; ++i)
            for (int j = k + 1; j < n; ++j) a(i, j) -= v[i] * q[j] + q[i] * v[j];
        a(k + 1, k) = r;
        a(k, k + 1) = r;
        for (int i = k + 2; i < n; ++i) { a(i, k) = 0.0; a(k, i) = 0.0; }
        // Z <- Z H
        for (int row = 0; row < n; ++row) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += z(row, j) * v[j];
            s *= tau;
            for (int j = k + 1; j < n; ++j) z(row, j) -= s * v[j];
        }
    }
    std::vector<double> d(n), e(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
    const double eps = 2.2e-16;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            int mm = l;
            for (; mm < n - 1; ++mm) {
                double dd = std::fabs(d[mm]) + std::fabs(d[mm + 1]);
                if (std::fabs(e[mm]) <= eps * dd) break;
            }
            if (mm == l) break;
            if (++iter > 200) return false;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = mm - 1;
            bool underflow = false;
            for (; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) { d[i + 1] -= p; e[mm] = 0.0; underflow = true; break; }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                for (int k = 0; k < n; ++k) {
                    double t = z(k, i + 1);
                    z(k, i + 1) = s * z(k, i) + c * t;
                    z(k, i) = c * z(k, i) - s * t;
                }
            }
            if (underflow) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    // sort ascending
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
    w.assign(n, 0.0);
    std::vector<double> Zs((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        w[j] = d[idx[j]];
        for (int i = 0; i < n; ++i) Zs[(size_t)i * n + j] = Z[(size_t)i * n + idx[j]];
    }
    Z.swap(Zs);
    return true;
}

// ------------------------------------------------------------ 1D operators
int Dir1D::glob_of_int(int i) const { return i < m - 1 ? i + 1 : i + 2; }
int Dir1D::int_of_glob(int g) const {
    if (g == 0 || g == m) return -1;
    return g < m ? g - 1 : g - 2;
}

// Closed forms on a cell of width h (Section 3; W_a = (P_a - P_{a+2})/(2a+3)):
//   hats:      stiffness (1/h)[[1,-1],[-1,1]], mass (h/6)[[2,1],[1,2]]
//   bubbles:   (W_a', W_b') = (2/h) 2/(2a+3) d_ab, hat-bubble stiffness 0
//              (W_a, W_b) = (h/2) Y_ab / ((2a+3)(2b+3)), Y_ab = (P_a-P_{a+2}, P_b-P_{b+2})_ref
//              (hat, W_0) = h/6, (hatL, W_1) = -h/30, (hatR, W_1) = +h/30
//   Gram:      (W_a, P_k) = (h/2)/(2a+3) [2/(2a+1) d_ka - 2/(2a+5) d_k,a+2]
//              (hatL, P_0) = (hatR, P_0) = h/2, (hatL, P_1) = -h/6, (hatR, P_1) = h/6
//   Gram of derivatives: (hatL', P_k) = -d_k0, (hatR', P_k) = d_k0, (W_a', P_k) = -2/(2a+3) d_k,a+1
static double yab_ref(int a, int b) {
    if (a == b) return 2.0 / (2 * a + 1) + 2.0 / (2 * a + 5);
    if (b == a + 2) return -2.0 / (2 * a + 5);
    if (a == b + 2) return -2.0 / (2 * b + 5);
    return 0.0;
}

static void build_dir1d_uncached(Dir1D& D, int m, int p, int n, double lo, double hi);

// The 1D operators (and their fast-diagonalisation eigenpairs, the costly part)
// depend only on (m, p, n, lo, hi); many problems share them, so keep a cache.
// Generalised symmetric eigenpairs of a 1D pencil (A, M), M SPD, dense row-major N x N:
// M = L L^T, L^{-1} A L^{-T} = Q diag(lam) Q^T, V = L^{-T} Q, so V^T M V = I and
// V^T A V = diag(lam) (V row-major, column j = vector j).
void pencil_eigen(int N, const std::vector<double>& Ad, const std::vector<double>& Md, std::vector<double>& V,
                  std::vector<double>& lam) {
    std::vector<double> L = Md;
    if (!cholesky(N, L)) throw std::runtime_error("1D mass matrix not SPD");
    // C = L^{-1} A L^{-T}: first X = L^{-1} A (forward substitution on columns), then C = X L^{-T}
    std::vector<double> X = Ad;
    for (int col = 0; col < N; ++col)
        for (int i = 0; i < N; ++i) {
            double s = X[(size_t)i * N + col];
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * N + k] * X[(size_t)k * N + col];
            X[(size_t)i * N + col] = s / L[(size_t)i * N + i];
        }
    std::vector<double> C((size_t)N * N);
    for (int row = 0; row < N; ++row)
        for (int i = 0; i < N; ++i) {
            double s = X[(size_t)row * N + i];
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * N + k] * C[(size_t)row * N + k];
            C[(size_t)row * N + i] = s / L[(size_t)i * N + i];
        }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < i; ++j) {
            double s = 0.5 * (C[(size_t)i * N + j] + C[(size_t)j * N + i]);
            C[(size_t)i * N + j] = C[(size_t)j * N + i] = s;
        }
    std::vector<double> Q;
    if (!symmetric_eigen(N, C, lam, Q)) throw std::runtime_error("eigen-decomposition failed");
    // V = L^{-T} Q: back substitution per column
    V.assign((size_t)N * N, 0.0);
    for (int col = 0; col < N; ++col)
        for (int i = N - 1; i >= 0; --i) {
            double s = Q[(size_t)i * N + col];
            for (int k = i + 1; k < N; ++k) s -= L[(size_t)k * N + i] * V[(size_t)k * N + col];
            V[(size_t)i * N + col] = s / L[(size_t)i * N + i];
        }
}

void build_dir1d(Dir1D& D, int m, int p, int n, double lo, double hi) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, double, double>, Dir1D> cache;
    const auto key = std::make_tuple(m, p, n, lo, hi);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) { D = it->second; return; }
    }
    build_dir1d_uncached(D, m, p, n, lo, hi);
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() > 512) cache.clear();
    cache.emplace(key, D);
}

static void build_dir1d_uncached(Dir1D& D, int m, int p, int n, double lo, double hi) {
    D.m = m; D.p = p; D.n = n;
    D.N1 = m * p + 1;
    D.n1 = m * p - 1;
    D.lo = lo;
    D.h = (hi - lo) / m;
    const double h = D.h;
    const int nb = p - 1;
    D.A.init(D.N1); D.M.init(D.N1); D.B.init(D.N1); D.Bd.init(D.N1);
    for (int c = 0; c < m; ++c) {
        int hl = c, hr = c + 1;
        auto bub = [&](int b) { return m + 1 + c * nb + b; };
        D.A.add(hl, hl, 1.0 / h); D.A.add(hr, hr, 1.0 / h);
        D.A.add(hl, hr, -1.0 / h); D.A.add(hr, hl, -1.0 / h);
        D.M.add(hl, hl, h / 3); D.M.add(hr, hr, h / 3);
        D.M.add(hl, hr, h / 6); D.M.add(hr, hl, h / 6);
        for (int a = 0; a < nb; ++a) {
            D.A.add(bub(a), bub(a), (2.0 / h) * 2.0 / (2 * a + 3));
            for (int b = std::max(0, a - 2); b <= std::min(nb - 1, a + 2); ++b) {
                double y = yab_ref(a, b);
                if (y != 0.0) D.M.add(bub(a), bub(b), 0.5 * h * y / ((2 * a + 3) * (2 * b + 3)));
            }
        }
        if (nb >= 1) {
            for (int hh : {hl, hr}) { D.M.add(hh, bub(0), h / 6); D.M.add(bub(0), hh, h / 6); }
        }
        if (nb >= 2) {
            D.M.add(hl, bub(1), -h / 30); D.M.add(bub(1), hl, -h / 30);
            D.M.add(hr, bub(1), h / 30); D.M.add(bub(1), hr, h / 30);
        }
        // Gram with the latent Legendre basis P_0..P_{n-1} of this cell
        for (int k = 0; k < n; ++k) {
            int col = c * n + k;
            if (k == 0) {
                D.B.add(hl, col, h / 2); D.B.add(hr, col, h / 2);
                D.Bd.add(hl, col, -1.0); D.Bd.add(hr, col, 1.0);
            }
            if (k == 1) { D.B.add(hl, col, -h / 6); D.B.add(hr, col, h / 6); }
            for (int a = 0; a < nb; ++a) {
                double v = 0.0;
                if (k == a) v = 2.0 / (2 * a + 1);
                else if (k == a + 2) v = -2.0 / (2 * a + 5);
                if (v != 0.0) D.B.add(bub(a), col, 0.5 * h * v / (2 * a + 3));
                if (k == a + 1) D.Bd.add(bub(a), col, -2.0 / (2 * a + 3));
            }
        }
    }
    // interior restrictions and transposes
    D.Ai.init(D.n1); D.Mi.init(D.n1); D.Bi.init(D.n1); D.Bdi.init(D.n1);
    D.BTi.init(m * n); D.BdTi.init(m * n);
    for (int i = 0; i < D.n1; ++i) {
        int g = D.glob_of_int(i);
        for (int e = 0; e < D.A.cnt[g]; ++e) {
            int j = D.int_of_glob(D.A.col[(size_t)g * kEll + e]);
            if (j >= 0) D.Ai.add(i, j, D.A.val[(size_t)g * kEll + e]);
        }
        for (int e = 0; e < D.M.cnt[g]; ++e) {
            int j = D.int_of_glob(D.M.col[(size_t)g * kEll + e]);
            if (j >= 0) D.Mi.add(i, j, D.M.val[(size_t)g * kEll + e]);
        }
        for (int e = 0; e < D.B.cnt[g]; ++e) {
            D.Bi.add(i, D.B.col[(size_t)g * kEll + e], D.B.val[(size_t)g * kEll + e]);
            D.BTi.add(D.B.col[(size_t)g * kEll + e], i, D.B.val[(size_t)g * kEll + e]);
        }
        for (int e = 0; e < D.Bd.cnt[g]; ++e) {
            D.Bdi.add(i, D.Bd.col[(size_t)g * kEll + e], D.Bd.val[(size_t)g * kEll + e]);
            D.BdTi.add(D.Bd.col[(size_t)g * kEll + e], i, D.Bd.val[(size_t)g * kEll + e]);
        }
    }
    // Fast diagonalisation of the interior pencil (A_i, M_i): M = L L^T,
    // L^{-1} A L^{-T} = Q diag(lam) Q^T, V = L^{-T} Q  (so V^T M V = I, V^T A V = diag(lam))
    const int N = D.n1;
    std::vector<double> Md((size_t)N * N, 0.0), Ad((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i) {
        for (int e = 0; e < D.Mi.cnt[i]; ++e) Md[(size_t)i * N + D.Mi.col[(size_t)i * kEll + e]] += D.Mi.val[(size_t)i * kEll + e];
        for (int e = 0; e < D.Ai.cnt[i]; ++e) Ad[(size_t)i * N + D.Ai.col[(size_t)i * kEll + e]] += D.Ai.val[(size_t)i * kEll + e];
    }
    pencil_eigen(N, Ad, Md, D.V, D.lam);
    // self-check: V^T A V = diag(lam), V^T M V = I
    double err = 0.0, scale = 1.0;
    for (double l : D.lam) scale = std::max(scale, std::fabs(l));
    std::vector<double> AV((size_t)N * N, 0.0), MV((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double sa = 0.0, sm = 0.0;
            for (int e = 0; e < D.Ai.cnt[i]; ++e) sa += D.Ai.val[(size_t)i * kEll + e] * D.V[(size_t)D.Ai.col[(size_t)i * kEll + e] * N + j];
            for (int e = 0; e < D.Mi.cnt[i]; ++e) sm += D.Mi.val[(size_t)i * kEll + e] * D.V[(size_t)D.Mi.col[(size_t)i * kEll + e] * N + j];
            AV[(size_t)i * N + j] = sa;
            MV[(size_t)i * N + j] = sm;
        }
    for (int a = 0; a < N; a += std::max(1, N / 17))
        for (int b = 0; b < N; b += std::max(1, N / 13)) {
            double sa = 0.0, sm = 0.0;
            for (int i = 0; i < N; ++i) {
                sa += D.V[(size_t)i * N + a] * AV[(size_t)i * N + b];
                sm += D.V[(size_t)i * N + a] * MV[(size_t)i * N + b];
            }
            err = std::max(err, std::fabs(sa - (a == b ? D.lam[a] : 0.0)) / scale);
            err = std::max(err, std::fabs(sm - (a == b ? 1.0 : 0.0)));
        }
    if (!(err < 1e-9)) throw std::runtime_error("fast-diagonalisation self-check failed");
}

// ------------------------------------------------------------ problem constants
static void kron_into(const std::vector<std::vector<double>>& mats, int n, int d, std::vector<double>& out) {
    // out[(i_0 + n i_1 + ..), (j_0 + n j_1 + ..)] = prod_k mats[k][i_k * n + j_k]
    size_t N = 1;
    for (int k = 0; k < d; ++k) N *= n;
    out.assign(N * N, 0.0);
    for (size_t I = 0; I < N; ++I)
        for (size_t J = 0; J < N; ++J) {
            size_t ii = I, jj = J;
            double v = 1.0;
            for (int k = 0; k < d; ++k) {
                v *= mats[k][(ii % n) * n + (jj % n)];
                ii /= n;
                jj /= n;
            }
            out[I * N + J] = v;
        }
}

void build_problem_constants(HostProblem& P) {
    const int d = P.d, n = P.n;
    P.ncomp = (P.kind == HPG_GRADIENT) ? d : 1;
    P.Nu_full = P.Nu0 = P.Nc = P.nloc = 1;
    P.detJ = 1.0;
    for (int j = 0; j < d; ++j) {
        build_dir1d(P.dir[j], P.m[j], P.p, n, P.lo[j], P.hi[j]);
        P.h[j] = P.dir[j].h;
        P.Nu_full *= P.dir[j].N1;
        P.Nu0 *= P.dir[j].n1;
        P.Nc *= P.m[j];
        P.nloc *= n;
        P.detJ *= 0.5 * P.h[j];
    }
    P.nb = P.nloc * P.ncomp;
    P.Npsi = P.Nc * P.nb;
    P.Nq = P.Nc * P.nloc;
    gauss_legendre(n, P.yq, P.wq);
    P.Vq.assign((size_t)n * n, 0.0);
    std::vector<double> Pl(n + 3), dPl(n + 3);
    for (int i = 0; i < n; ++i) {
        legendre_all(n + 2, P.yq[i], Pl.data(), dPl.data());
        for (int k = 0; k < n; ++k) P.Vq[(size_t)i * n + k] = Pl[k];
    }
    // Psi mass of a cell (Lemma: diagonal |K_j| / (2k+1) per direction) and broken
    // H^1 seminorm (P_k', P_l')_ref = min(k,l)(min(k,l)+1) when k = l mod 2, times 2/h.
    P.Mpsi_loc.assign(P.nloc, 1.0);
    for (size_t I = 0; I < P.nloc; ++I) {
        size_t ii = I;
        for (int k = 0; k < d; ++k) {
            int kk = (int)(ii % n);
            ii /= n;
            P.Mpsi_loc[I] *= P.h[k] / (2.0 * kk + 1.0);
        }
    }
    if (P.kind == HPG_GRADIENT) {
        P.Kpsi_loc.assign(P.nloc * P.nloc, 0.0);
        for (int dir = 0; dir < d; ++dir) {
            std::vector<std::vector<double>> mats(d, std::vector<double>((size_t)n * n, 0.0));
            for (int k = 0; k < d; ++k)
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) {
                        double v = 0.0;
                        if (k == dir) {
                            int mn = std::min(a, b);
                            if ((a - b) % 2 == 0) v = (2.0 / P.h[k]) * mn * (mn + 1.0);
                        } else if (a == b) {
                            v = P.h[k] / (2.0 * a + 1.0);
                        }
                        mats[k][(size_t)a * n + b] = v;
                    }
            std::vector<double> Kd;
            kron_into(mats, n, d, Kd);
            for (size_t i = 0; i < Kd.size(); ++i) P.Kpsi_loc[i] += Kd[i];
        }
    } else {
        // C_K = B-hat^T A-hat_1^{-1} B-hat, eq. (schur-preconditioner), with the
        // spectral-Galerkin functions Y_0..Y_{p-2} of the cell:
        //   (Y_a', Y_b')_K = (2/h) 2 (2a+3) d_ab,  (Y_a, Y_b)_K = (h/2) Y_ab,
        //   (Y_a, P_k)_K = (h/2) [2/(2a+1) d_ka - 2/(2a+5) d_k,a+2]
        const size_t N = P.nloc;
        std::vector<double> Ahat(N * N, 0.0), Bhat;
        std::vector<std::vector<double>> KY(d), MY(d), BY(d);
        for (int k = 0; k < d; ++k) {
            KY[k].assign((size_t)n * n, 0.0);
            MY[k].assign((size_t)n * n, 0.0);
            BY[k].assign((size_t)n * n, 0.0);
            for (int a = 0; a < n; ++a) {
                KY[k][(size_t)a * n + a] = (2.0 / P.h[k]) * 2.0 * (2 * a + 3);
                for (int b = 0; b < n; ++b) MY[k][(size_t)a * n + b] = 0.5 * P.h[k] * yab_ref(a, b);
                for (int kk = 0; kk < n; ++kk) {
                    double v = 0.0;
                    if (kk == a) v = 2.0 / (2 * a + 1);
                    else if (kk == a + 2) v = -2.0 / (2 * a + 5);
                    BY[k][(size_t)a * n + kk] = 0.5 * P.h[k] * v;
                }
            }
        }
        for (int dir = 0; dir < d; ++dir) {
            std::vector<std::vector<double>> mats(d);
            for (int k = 0; k < d; ++k) mats[k] = (k == dir) ? KY[k] : MY[k];
            std::vector<double> T;
            kron_into(mats, n, d, T);
            for (size_t i = 0; i < T.size(); ++i) Ahat[i] += T[i];
        }
        kron_into(BY, n, d, Bhat);
        std::vector<double> L = Ahat;
        if (!cholesky((int)N, L)) throw std::runtime_error("A-hat not SPD");
        // Y = L^{-1} Bhat; C = Y^T Y
        std::vector<double> Y = Bhat;
        for (size_t col = 0; col < N; ++col)
            for (size_t i = 0; i < N; ++i) {
                double s = Y[i * N + col];
                for (size_t k = 0; k < i; ++k) s -= L[i * N + k] * Y[k * N + col];
                Y[i * N + col] = s / L[i * N + i];
            }
        P.Cblk.assign(N * N, 0.0);
        for (size_t i = 0; i < N; ++i)
            for (size_t j = 0; j <= i; ++j) {
                double s = 0.0;
                for (size_t k = 0; k < N; ++k) s += Y[k * N + i] * Y[k * N + j];
                P.Cblk[i * N + j] = P.Cblk[j * N + i] = s;
            }
    }
    P.bf.assign(P.Nu0, 0.0);
    P.ulift.assign(P.Nu_full, 0.0);
    P.rA.assign(P.Nu0, 0.0);
    P.rB.assign(P.Npsi, 0.0);
    P.phiq.assign(P.Nq, 0.0);
    P.phiz.assign(P.Npsi, 0.0);
}

static void cell_multi(const HostProblem& P, size_t c, int* cm) {
    for (int j = 0; j < P.d; ++j) { cm[j] = (int)(c % P.m[j]); c /= P.m[j]; }
}

void latent_points(const HostProblem& P, std::vector<double>& pts) {
    const int d = P.d, n = P.n;
    pts.assign(P.Nq * d, 0.0);
    for (size_t c = 0; c < P.Nc; ++c) {
        int cm[kMaxDim];
        cell_multi(P, c, cm);
        for (size_t q = 0; q < P.nloc; ++q) {
            size_t qq = q;
            for (int j = 0; j < d; ++j) {
                int qi = (int)(qq % n);
                qq /= n;
                pts[(c * P.nloc + q) * d + j] = P.lo[j] + (cm[j] + 0.5 * (P.yq[qi] + 1.0)) * P.h[j];
            }
        }
    }
}

// (f, v_i) over the interior dofs with (p+2)^d Gauss points per cell.
void compute_rhs(HostProblem& P, hpg_field_fn f, void* user, bool is_const, double cval) {
    const int d = P.d, p = P.p, nq = p + 2;
    std::vector<double> y, w;
    gauss_legendre(nq, y, w);
    // local 1D U values at the points: [hatL, hatR, W_0..W_{p-2}], W_a = (P_a - P_{a+2})/(2a+3)
    std::vector<double> U((size_t)(p + 1) * nq);
    std::vector<double> Pl(p + 3), dPl(p + 3);
    for (int i = 0; i < nq; ++i) {
        legendre_all(p + 1, y[i], Pl.data(), dPl.data());
        U[(size_t)0 * nq + i] = 0.5 * (1.0 - y[i]);
        U[(size_t)1 * nq + i] = 0.5 * (1.0 + y[i]);
        for (int a = 0; a + 2 <= p; ++a) U[(size_t)(2 + a) * nq + i] = (Pl[a] - Pl[a + 2]) / (2 * a + 3);
    }
    size_t npc = 1, nlc = 1;
    for (int j = 0; j < d; ++j) { npc *= nq; nlc *= (p + 1); }
    std::vector<double> X(npc * d), fv(npc), T, T2;
    std::fill(P.bf.begin(), P.bf.end(), 0.0);
    for (size_t c = 0; c < P.Nc; ++c) {
        int cm[kMaxDim];
        cell_multi(P, c, cm);
        for (size_t q = 0; q < npc; ++q) {
            size_t qq = q;
            for (int j = 0; j < d; ++j) {
                int qi = (int)(qq % nq);
                qq /= nq;
                X[q * d + j] = P.lo[j] + (cm[j] + 0.5 * (y[qi] + 1.0)) * P.h[j];
            }
        }
        if (is_const) std::fill(fv.begin(), fv.end(), cval);
        else f((int)npc, d, X.data(), fv.data(), nullptr == user ? nullptr : user);
        // T[q] = w(q) detJ sign f(q), then contract each direction with U
        T.assign(npc, 0.0);
        for (size_t q = 0; q < npc; ++q) {
            size_t qq = q;
            double wt = P.detJ * P.sign;
            for (int j = 0; j < d; ++j) { wt *= w[qq % nq]; qq /= nq; }
            T[q] = wt * fv[q];
        }
        // contract direction by direction: index layout x fastest
        size_t cur_inner = 1;
        std::vector<int> dims(d, nq);
        for (int j = 0; j < d; ++j) {
            size_t outer = 1;
            for (int k = j + 1; k < d; ++k) outer *= dims[k];
            size_t inner = cur_inner;
            T2.assign(outer * (p + 1) * inner, 0.0);
            for (size_t o = 0; o < outer; ++o)
                for (int a = 0; a < p + 1; ++a)
                    for (size_t in = 0; in < inner; ++in) {
                        double s = 0.0;
                        for (int q = 0; q < nq; ++q) s += U[(size_t)a * nq + q] * T[(o * nq + q) * inner + in];
                        T2[(o * (p + 1) + a) * inner + in] = s;
                    }
            T.swap(T2);
            dims[j] = p + 1;
            cur_inner *= (p + 1);
        }
        // scatter local (p+1)^d into interior dofs
        for (size_t L = 0; L < nlc; ++L) {
            size_t ll = L, gi = 0, stride = 1;
            bool interior = true;
            for (int j = 0; j < d; ++j) {
                int a = (int)(ll % (p + 1));
                ll /= (p + 1);
                const Dir1D& D = P.dir[j];
                int g = a == 0 ? cm[j] : (a == 1 ? cm[j] + 1 : D.m + 1 + cm[j] * (p - 1) + (a - 2));
                int ii = D.int_of_glob(g);
                if (ii < 0) { interior = false; break; }
                gi += (size_t)ii * stride;
                stride *= D.n1;
            }
            if (interior) P.bf[gi] += T[L];
        }
    }
}

// phi at the latent Gauss points (sign applied); (phi, zeta) is formed on the device.
void compute_phi(HostProblem& P, const double* phi_q) {
    for (size_t i = 0; i < P.Nq; ++i) P.phiq[i] = P.sign * phi_q[i];
    P.has_phi = true;
}

// Dirichlet lifting: per boundary face, the tensor product over the tangential
// directions of the 1D rule Pi (vertex values + H^1_0 projection of the
// remainder onto the bubbles), applied to samples of g on the face.
void compute_lifting(HostProblem& P, hpg_field_fn g, void* user) {
    std::fill(P.ulift.begin(), P.ulift.end(), 0.0);
    std::fill(P.rA.begin(), P.rA.end(), 0.0);
    std::fill(P.rB.begin(), P.rB.end(), 0.0);
    if (!g) return;
    const int d = P.d, p = P.p, nqc = 2 * p + 2;
    std::vector<double> y, w;
    gauss_legendre(nqc, y, w);
    std::vector<double> Pl(p + 3), dPl(p + 3);
    // 1D sample points and Pi (N1 x ns) per direction
    std::vector<std::vector<double>> spts(d), Pi(d);
    std::vector<int> ns(d);
    for (int j = 0; j < d; ++j) {
        const Dir1D& D = P.dir[j];
        int m = D.m;
        ns[j] = m + 1 + m * nqc;
        spts[j].resize(ns[j]);
        Pi[j].assign((size_t)D.N1 * ns[j], 0.0);
        for (int v = 0; v <= m; ++v) { spts[j][v] = D.lo + v * D.h; Pi[j][(size_t)v * ns[j] + v] = 1.0; }
        for (int c = 0; c < m; ++c) {
            int base = m + 1 + c * nqc;
            for (int q = 0; q < nqc; ++q) spts[j][base + q] = D.lo + (c + 0.5 * (y[q] + 1.0)) * D.h;
            for (int b = 0; b + 2 <= p; ++b) {
                int row = m + 1 + c * (p - 1) + b;
                double sl = 0.0, sr = 0.0;
                for (int q = 0; q < nqc; ++q) {
                    legendre_all(b + 1, y[q], Pl.data(), dPl.data());
                    double wt = 0.5 * (2 * b + 3) * w[q] * dPl[b + 1];
                    Pi[j][(size_t)row * ns[j] + base + q] += wt;
                    sl += wt * 0.5 * (1.0 - y[q]);
                    sr += wt * 0.5 * (1.0 + y[q]);
                }
                Pi[j][(size_t)row * ns[j] + c] -= sl;
                Pi[j][(size_t)row * ns[j] + c + 1] -= sr;
            }
        }
    }
    for (int fj = 0; fj < d; ++fj)
        for (int side = 0; side < 2; ++side) {
            const Dir1D& Dn = P.dir[fj];
            double xf = side == 0 ? Dn.lo : Dn.lo + Dn.m * Dn.h;
            int gf = side == 0 ? 0 : Dn.m;
            // tangential directions
            std::vector<int> tdirs;
            for (int j = 0; j < d; ++j) if (j != fj) tdirs.push_back(j);
            size_t npts = 1;
            for (int j : tdirs) npts *= ns[j];
            std::vector<double> X(npts * d), gv(npts);
            for (size_t s = 0; s < npts; ++s) {
                size_t ss = s;
                for (int j : tdirs) { X[s * d + j] = spts[j][ss % ns[j]]; ss /= ns[j]; }
                X[s * d + fj] = xf;
            }
            g((int)npts, d, X.data(), gv.data(), user);
            for (auto& v : gv) v *= P.sign;
            // contract tangential directions with Pi
            std::vector<double> T = gv, T2;
            std::vector<size_t> dims;
            for (int j : tdirs) dims.push_back(ns[j]);
            size_t inner = 1;
            for (size_t t = 0; t < tdirs.size(); ++t) {
                int j = tdirs[t];
                size_t outer = 1;
                for (size_t u = t + 1; u < tdirs.size(); ++u) outer *= dims[u];
                int N1 = P.dir[j].N1;
                T2.assign(outer * N1 * inner, 0.0);
                for (size_t o = 0; o < outer; ++o)
                    for (int a = 0; a < N1; ++a)
                        for (size_t in = 0; in < inner; ++in) {
                            double s = 0.0;
                            for (size_t q = 0; q < dims[t]; ++q)
                                s += Pi[j][(size_t)a * ns[j] + q] * T[(o * dims[t] + q) * inner + in];
                            T2[(o * N1 + a) * inner + in] = s;
                        }
                T.swap(T2);
                dims[t] = N1;
                inner *= N1;
            }
            // write coefficients of dofs with index gf in direction fj
            size_t ncoef = T.size();
            for (size_t s = 0; s < ncoef; ++s) {
                size_t ss = s, full = 0, stride = 1;
                int idx[kMaxDim];
                for (size_t t = 0; t < tdirs.size(); ++t) { idx[tdirs[t]] = (int)(ss % dims[t]); ss /= dims[t]; }
                idx[fj] = gf;
                for (int j = 0; j < d; ++j) { full += (size_t)idx[j] * stride; stride *= P.dir[j].N1; }
                P.ulift[full] = T[s];
            }
        }
    // lifting terms: rA = (A u_lift) on interior rows, rB = B^T u_lift (full columns)
    // A = sum_k (x)_j (k == j ? A_j : M_j) over full 1D operators
    const size_t Nf = P.Nu_full;
    for (size_t I = 0; I < P.Nu0; ++I) {
        size_t ii = I;
        int gi[kMaxDim];
        for (int j = 0; j < d; ++j) { gi[j] = P.dir[j].glob_of_int((int)(ii % P.dir[j].n1)); ii /= P.dir[j].n1; }
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            // iterate over the tensor stencil
            const Ell* ops[kMaxDim];
            for (int j = 0; j < d; ++j) ops[j] = (j == k) ? &P.dir[j].A : &P.dir[j].M;
            int cnt[kMaxDim], e[kMaxDim] = {0, 0, 0};
            for (int j = 0; j < d; ++j) cnt[j] = ops[j]->cnt[gi[j]];
            bool done = false;
            for (int j = 0; j < d; ++j) if (cnt[j] == 0) done = true;
            while (!done) {
                double v = 1.0;
                size_t full = 0, stride = 1;
                for (int j = 0; j < d; ++j) {
                    size_t off = (size_t)gi[j] * kEll + e[j];
                    v *= ops[j]->val[off];
                    full += (size_t)ops[j]->col[off] * stride;
                    stride *= P.dir[j].N1;
                }
                s += v * P.ulift[full];
                int j = 0;
                while (j < d) { if (++e[j] < cnt[j]) break; e[j] = 0; ++j; }
                if (j == d) done = true;
            }
        }
        P.rA[I] = s;
    }
    (void)Nf;
    // rB[psi index] = sum over full u of B(u, psi) u_lift(u); B = (x)_j B_j (obstacle),
    // gradient component k: (x)_j (j == k ? Bd_j : B_j)
    for (size_t Ifull = 0; Ifull < P.Nu_full; ++Ifull) {
        double uv = P.ulift[Ifull];
        if (uv == 0.0) continue;
        size_t ii = Ifull;
        int gi[kMaxDim];
        for (int j = 0; j < d; ++j) { gi[j] = (int)(ii % P.dir[j].N1); ii /= P.dir[j].N1; }
        for (int comp = 0; comp < P.ncomp; ++comp) {
            const Ell* ops[kMaxDim];
            for (int j = 0; j < d; ++j)
                ops[j] = (P.kind == HPG_GRADIENT && j == comp) ? &P.dir[j].Bd : &P.dir[j].B;
            int cnt[kMaxDim], e[kMaxDim] = {0, 0, 0};
            bool done = false;
            for (int j = 0; j < d; ++j) { cnt[j] = ops[j]->cnt[gi[j]]; if (!cnt[j]) done = true; }
            while (!done) {
                double v = uv;
                size_t cell = 0, cstride = 1, loc = 0, lstride = 1;
                for (int j = 0; j < d; ++j) {
                    size_t off = (size_t)gi[j] * kEll + e[j];
                    v *= ops[j]->val[off];
                    int col = ops[j]->col[off];
                    cell += (size_t)(col / P.n) * cstride;
                    loc += (size_t)(col % P.n) * lstride;
                    cstride *= P.m[j];
                    lstride *= P.n;
                }
                P.rB[(cell * P.ncomp + comp) * P.nloc + loc] += v;
                int j = 0;
                while (j < d) { if (++e[j] < cnt[j]) break; e[j] = 0; ++j; }
                if (j == d) done = true;
            }
        }
    }
}

// u_h at one point from full coefficients (host; used by hpg_eval_u).
double eval_u_point(const HostProblem& P, const std::vector<double>& u, const double* x) {
    const int d = P.d, p = P.p;
    int cm[kMaxDim];
    double vals[kMaxDim][kMaxN + 3];
    int glob[kMaxDim][kMaxN + 3];
    std::vector<double> Pl(p + 3), dPl(p + 3);
    for (int j = 0; j < d; ++j) {
        const Dir1D& D = P.dir[j];
        int c = (int)std::floor((x[j] - D.lo) / D.h);
        c = std::min(std::max(c, 0), D.m - 1);
        cm[j] = c;
        double y = 2.0 * (x[j] - (D.lo + c * D.h)) / D.h - 1.0;
        legendre_all(p + 1, y, Pl.data(), dPl.data());
        vals[j][0] = 0.5 * (1.0 - y);
        vals[j][1] = 0.5 * (1.0 + y);
        glob[j][0] = c;
        glob[j][1] = c + 1;
        for (int a = 0; a + 2 <= p; ++a) {
            vals[j][2 + a] = (Pl[a] - Pl[a + 2]) / (2 * a + 3);
            glob[j][2 + a] = D.m + 1 + c * (p - 1) + a;
        }
    }
    (void)cm;
    double s = 0.0;
    int e[kMaxDim] = {0, 0, 0};
    while (true) {
        double v = 1.0;
        size_t full = 0, stride = 1;
        for (int j = 0; j < d; ++j) {
            v *= vals[j][e[j]];
            full += (size_t)glob[j][e[j]] * stride;
            stride *= P.dir[j].N1;
        }
        s += v * u[full];
        int j = 0;
        while (j < d) { if (++e[j] < p + 1) break; e[j] = 0; ++j; }
        if (j == d) break;
    }
    return s;
}

}  // namespace hpg

namespace hpg {

double mass_norm2(const HostProblem& P, const std::vector<double>& e) {
    // apply the 1D mass matrix along each axis in turn (full numbering, x fastest)
    std::vector<double> cur(e), nxt(e.size());
    size_t inner = 1;
    for (int j = 0; j < P.d; ++j) {
        const Dir1D& D = P.dir[j];
        const size_t N1 = (size_t)D.N1, outer = e.size() / (inner * N1);
        for (size_t o = 0; o < outer; ++o)
            for (size_t r = 0; r < N1; ++r)
                for (size_t i = 0; i < inner; ++i) {
                    double acc = 0.0;
                    for (int t = 0; t < D.M.cnt[r]; ++t) {
                        const size_t c = (size_t)D.M.col[r * kEll + t];
                        acc += D.M.val[r * kEll + t] * cur[(o * N1 + c) * inner + i];
                    }
                    nxt[(o * N1 + r) * inner + i] = acc;
                }
        std::swap(cur, nxt);
        inner *= N1;
    }
    double s = 0.0;
    for (size_t i = 0; i < e.size(); ++i) s += e[i] * cur[i];
    return s;
}

}  // namespace hpg

namespace hpg {

namespace {
// entry (r, c) of a padded-ELL operator (0 if absent)
double ell_at(const Ell& E, int r, int c) {
    double v = 0.0;
    for (int e = 0; e < E.cnt[r]; ++e)
        if (E.col[(size_t)r * kEll + e] == c) v += E.val[(size_t)r * kEll + e];
    return v;
}
}  // namespace

void build_ainv_precond(HostProblem& P) {
    AinvPrecond& ap = P.ap;
    if (ap.built) return;
    const int d = P.d, nbub = P.p - 1;
    // coarse space: the interior vertex hats of each axis, interior 1D indices 0 .. m-2
    for (int j = 0; j < d; ++j) {
        const Dir1D& D = P.dir[j];
        const int nv = D.m - 1;
        ap.nv[j] = nv;
        if (nv < 1) continue;
        std::vector<double> Ad((size_t)nv * nv, 0.0), Md((size_t)nv * nv, 0.0);
        for (int a = 0; a < nv; ++a)
            for (int b = 0; b < nv; ++b) {
                Ad[(size_t)a * nv + b] = ell_at(D.Ai, a, b);
                Md[(size_t)a * nv + b] = ell_at(D.Mi, a, b);
            }
        pencil_eigen(nv, Ad, Md, ap.Vc[j], ap.lamc[j]);
    }
    // entity blocks: type t = mask of the axes that carry bubbles (t = 0 is the coarse space)
    size_t off = 0;
    for (int t = 1; t < (1 << d); ++t) {
        int nb = 1;
        long long ne = 1;
        for (int j = 0; j < d; ++j) {
            const bool bub = (t >> j) & 1;
            if (bub) nb *= nbub;
            ne *= bub ? P.dir[j].m : P.dir[j].m - 1;
        }
        ap.bsize[t] = nb;
        ap.nent[t] = (nbub > 0) ? ne : 0;
        ap.boff[t] = (long long)off;
        if (ap.nent[t] == 0) continue;
        // B[l][l'] = sum_k prod_j (k == j ? A_j : M_j)(e_j(l), e_j(l')): hat axes take the
        // diagonal entry of an interior vertex, bubble axes the bubble block of cell 0
        // (identical for every vertex and cell of a uniform mesh)
        std::vector<double> B((size_t)nb * nb, 0.0);
        for (int l = 0; l < nb; ++l)
            for (int lp = 0; lp < nb; ++lp) {
                int bl[kMaxDim], blp[kMaxDim];
                int rl = l, rlp = lp;
                for (int j = 0; j < d; ++j) {
                    if ((t >> j) & 1) { bl[j] = rl % nbub; rl /= nbub; blp[j] = rlp % nbub; rlp /= nbub; }
                    else { bl[j] = blp[j] = -1; }
                }
                double sum = 0.0;
                for (int k = 0; k < d; ++k) {
                    double prod = 1.0;
                    for (int j = 0; j < d; ++j) {
                        const Dir1D& D = P.dir[j];
                        const Ell& E = (k == j) ? D.Ai : D.Mi;
                        const int r = bl[j] < 0 ? 0 : D.m - 1 + bl[j];
                        const int c = blp[j] < 0 ? 0 : D.m - 1 + blp[j];
                        prod *= ell_at(E, r, c);
                    }
                    sum += prod;
                }
                B[(size_t)l * nb + lp] = sum;
            }
        // inverse through the Cholesky factor: B^{-1} = L^{-T} L^{-1}
        std::vector<double> L = B;
        if (!cholesky(nb, L)) throw std::runtime_error("stiffness entity block not SPD");
        std::vector<double> X((size_t)nb * nb, 0.0);   // X = L^{-1}
        for (int c = 0; c < nb; ++c)
            for (int i = 0; i < nb; ++i) {
                double v = (i == c) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) v -= L[(size_t)i * nb + k] * X[(size_t)k * nb + c];
                X[(size_t)i * nb + c] = v / L[(size_t)i * nb + i];
            }
        ap.Binv.resize(off + (size_t)nb * nb);
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < nb; ++c) {
                double v = 0.0;
                for (int k = std::max(i, c); k < nb; ++k) v += X[(size_t)k * nb + i] * X[(size_t)k * nb + c];
                ap.Binv[off + (size_t)i * nb + c] = v;
            }
        off += (size_t)nb * nb;
    }
    ap.built = true;
}

}  // namespace hpg

namespace hpg {

namespace {
// the interior 1D indices of the local dofs of cell c (left hat, right hat when interior,
// then the bubbles), in the order the cell-patch blocks use
void cell_dofs_1d(const Dir1D& D, int c, std::vector<int>& L) {
    L.clear();
    if (c >= 1) L.push_back(c - 1);                  // vertex c (interior index c - 1)
    if (c + 1 <= D.m - 1) L.push_back(c);            // vertex c + 1
    for (int b = 0; b < D.p - 1; ++b) L.push_back(D.m - 1 + c * (D.p - 1) + b);
}
}  // namespace

void build_ainv_cells(HostProblem& P) {
    AinvPrecond& ap = P.ap;
    if (ap.cells_built) return;
    const int d = P.d;
    for (int k = 0; k < 64; ++k) ap.csize[k] = -1;
    size_t off = 0;
    // one representative cell per class: code per axis from (left end interior, right end interior)
    for (int k = 0; k < (1 << (2 * d)); ++k) {
        int cell[kMaxDim] = {0, 0, 0};
        bool present = true;
        for (int j = 0; j < d; ++j) {
            const int code = (k >> (2 * j)) & 3, m = P.dir[j].m;
            // code bit 0: a left interior vertex, bit 1: a right interior vertex
            if (code == 0) { present = present && m == 1; cell[j] = 0; }
            else if (code == 1) { present = present && m >= 2; cell[j] = m - 1; }
            else if (code == 2) { present = present && m >= 2; cell[j] = 0; }
            else { present = present && m >= 3; cell[j] = 1; }
        }
        if (!present) continue;
        std::vector<int> L[kMaxDim];
        int nb = 1, n1d[kMaxDim] = {1, 1, 1};
        for (int j = 0; j < d; ++j) {
            cell_dofs_1d(P.dir[j], cell[j], L[j]);
            n1d[j] = (int)L[j].size();
            nb *= n1d[j];
        }
        std::vector<double> B((size_t)nb * nb, 0.0);
        for (int l = 0; l < nb; ++l)
            for (int lp = 0; lp < nb; ++lp) {
                int il[kMaxDim], ilp[kMaxDim];
                int rl = l, rlp = lp;
                for (int j = 0; j < d; ++j) {
                    il[j] = L[j][rl % n1d[j]];
                    rl /= n1d[j];
                    ilp[j] = L[j][rlp % n1d[j]];
                    rlp /= n1d[j];
                }
                double sum = 0.0;
                for (int q = 0; q < d; ++q) {
                    double prod = 1.0;
                    for (int j = 0; j < d; ++j) prod *= ell_at(q == j ? P.dir[j].Ai : P.dir[j].Mi, il[j], ilp[j]);
                    sum += prod;
                }
                B[(size_t)l * nb + lp] = sum;
            }
        std::vector<double> Lf = B;
        if (!cholesky(nb, Lf)) throw std::runtime_error("stiffness cell block not SPD");
        std::vector<double> X((size_t)nb * nb, 0.0);
        for (int c = 0; c < nb; ++c)
            for (int i = 0; i < nb; ++i) {
                double v = (i == c) ? 1.0 : 0.0;
                for (int q = 0; q < i; ++q) v -= Lf[(size_t)i * nb + q] * X[(size_t)q * nb + c];
                X[(size_t)i * nb + c] = v / Lf[(size_t)i * nb + i];
            }
        ap.Cinv.resize(off + (size_t)nb * nb);
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < nb; ++c) {
                double v = 0.0;
                for (int q = std::max(i, c); q < nb; ++q) v += X[(size_t)q * nb + i] * X[(size_t)q * nb + c];
                ap.Cinv[off + (size_t)i * nb + c] = v;
            }
        ap.csize[k] = nb;
        ap.coff[k] = (long long)off;
        ap.cmax = std::max(ap.cmax, nb);
        off += (size_t)nb * nb;
    }
    ap.cells_built = true;
}

}  // namespace hpg

namespace hpg {

void build_ainv_stars(HostProblem& P) {
    AinvPrecond& ap = P.ap;
    if (ap.stars_built) return;
    const int nbub = P.p - 1;
    for (int j = 0; j < P.d; ++j) {
        const Dir1D& D = P.dir[j];
        // the star of interior vertex v = 1: bubbles of cell 0, hat of vertex 1, bubbles of
        // cell 1 (every interior vertex's star has the same 1D matrices on a uniform mesh)
        std::vector<int> L;
        if (D.m >= 2) {
            for (int b = 0; b < nbub; ++b) L.push_back(D.m - 1 + b);
            L.push_back(0);
            for (int b = 0; b < nbub; ++b) L.push_back(D.m - 1 + nbub + b);
        } else {
            for (int b = 0; b < nbub; ++b) L.push_back(D.m - 1 + b);
        }
        const int n = (int)L.size();
        ap.ns[j] = n;
        std::vector<double> Ad((size_t)n * n), Md((size_t)n * n);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                Ad[(size_t)a * n + b] = ell_at(D.Ai, L[a], L[b]);
                Md[(size_t)a * n + b] = ell_at(D.Mi, L[a], L[b]);
            }
        pencil_eigen(n, Ad, Md, ap.Vs[j], ap.lams[j]);
    }
    ap.stars_built = true;
}

}  // namespace hpg
