// CUDA kernels of libhpg (sm_103a).  Every step of the hpG Newton--Krylov path
// runs here: Gauss evaluation of the latent nonlinearity, residuals, the
// matrix-free Newton and Schur operators by sum factorisation and sparse
// Kronecker stencils, the S-hat cell-block factorisation, the fast-diagonalisation
// inverse of A_alpha, and GMRES.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <cfloat>
#include <cmath>

#include "device.h"

namespace hpg {

namespace {

// kernels launched (or replayed from graphs) by the calling host thread: a solve
// runs on one host thread, also when several solves are in flight on others
thread_local long long t_launches = 0;
inline void note_launch() { ++t_launches; }

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    // deterministic block reduction (fixed tree)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;  // valid in thread 0
}

__device__ __forceinline__ void decompose(long long i, int d, const int* n1, int* ix) {
    for (int j = 0; j < d; ++j) { ix[j] = (int)(i % n1[j]); i /= n1[j]; }
}

// sum over the tensor stencil of prod_j S_j[r_j] applied to an interior-u vector
template <int D, typename T, typename Tx>
__device__ __forceinline__ T gather_u(const Sten<T>* const* S, const int* r, const int* n1, const Tx* x) {
    T s = T(0);
    if (D == 2) {
        const int c0 = S[0]->cnt[r[0]], c1 = S[1]->cnt[r[1]];
        const int* col0 = S[0]->col + (size_t)r[0] * kEll;
        const T* val0 = S[0]->val + (size_t)r[0] * kEll;
        for (int e1 = 0; e1 < c1; ++e1) {
            const long long base = (long long)S[1]->col[(size_t)r[1] * kEll + e1] * n1[0];
            T t = T(0);
            for (int e0 = 0; e0 < c0; ++e0) t += val0[e0] * (T)x[base + col0[e0]];
            s += S[1]->val[(size_t)r[1] * kEll + e1] * t;
        }
    } else {
        const int c0 = S[0]->cnt[r[0]], c1 = S[1]->cnt[r[1]], c2 = S[2]->cnt[r[2]];
        const int* col0 = S[0]->col + (size_t)r[0] * kEll;
        const T* val0 = S[0]->val + (size_t)r[0] * kEll;
        for (int e2 = 0; e2 < c2; ++e2) {
            const long long b2 = (long long)S[2]->col[(size_t)r[2] * kEll + e2] * n1[1];
            T t2 = T(0);
            for (int e1 = 0; e1 < c1; ++e1) {
                const long long base = (b2 + S[1]->col[(size_t)r[1] * kEll + e1]) * n1[0];
                T t = T(0);
                for (int e0 = 0; e0 < c0; ++e0) t += val0[e0] * (T)x[base + col0[e0]];
                t2 += S[1]->val[(size_t)r[1] * kEll + e1] * t;
            }
            s += S[2]->val[(size_t)r[2] * kEll + e2] * t2;
        }
    }
    return s;
}

// (B^T x)[cell, comp, k] (interior u -> psi)
template <int D, typename T, typename Tx>
__device__ __forceinline__ T apply_BT_entry(const Geo<T>& g, const int* cm, int comp, const int* km, const Tx* x) {
    const Sten<T>* S[kMaxDim];
    int r[kMaxDim];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        S[j] = (g.kind == HPG_GRADIENT && j == comp) ? &g.BdT[j] : &g.BT[j];
        r[j] = cm[j] * g.n + km[j];
    }
    return gather_u<D, T, Tx>(S, r, g.n1, x);
}

template <typename T>
__device__ __forceinline__ void cell_multi(const Geo<T>& g, long long c, int* cm) {
    for (int j = 0; j < g.d; ++j) { cm[j] = (int)(c % g.m[j]); c /= g.m[j]; }
}

// One sum-factorisation pass along axis `ax` over `cnt` tensors of n^d each:
// out[.., a, ..] = sum_k M(a, k) in[.., k, ..] with M(a,k) = mat[a*n+k] (or mat[k*n+a] if transp)
template <typename T>
__device__ __forceinline__ void sf_pass(const T* in, T* out, const T* mat, bool transp, int n, int nloc, int cnt,
                                        int stride, int lt = -1, int nthr = 0) {
    if (lt < 0) { lt = threadIdx.x; nthr = blockDim.x; }
    for (int i = lt; i < nloc * cnt; i += nthr) {
        const int t = i / nloc, li = i - t * nloc;
        const int a = (li / stride) % n;
        const int base = t * nloc + li - a * stride;
        T s = T(0);
        if (!transp)
            for (int k = 0; k < n; ++k) s += mat[a * n + k] * in[base + k * stride];
        else
            for (int k = 0; k < n; ++k) s += mat[k * n + a] * in[base + k * stride];
        out[i] = s;
    }
}

}  // namespace

long long kernel_launch_count() { return t_launches; }
void note_kernel_launches(long long n) { t_launches += n; }

// ============================================================ tiled u-row applies
// y[i] over interior u-dofs i of  cA * (A x)[i] + cB * (B z)[i]  (+ residual terms),
// with A = sum_k (x)_j (j == k ? A_j : M_j) and B = (x)_j B_j (gradient: component
// c uses the derivative Gram Bd_c along axis c).  Each block owns a tile of the
// tensor grid and first stages the 1D stencil rows of its tile ranges in shared
// memory, so every term of the gather costs one independent global load.
template <int D>
struct UTile;
template <>
struct UTile<2> { static constexpr int T0 = 32, T1 = 8, T2 = 1; };
template <>
struct UTile<3> { static constexpr int T0 = 8, T1 = 8, T2 = 4; };

enum { OP_A = 0, OP_M = 1, OP_B = 2, OP_BD = 3, NOPS = 4 };

template <typename T, int TMAX>
struct StenTile {
    int cnt[NOPS][kMaxDim][TMAX];
    int col[NOPS][kMaxDim][TMAX][kEll];
    T val[NOPS][kMaxDim][TMAX][kEll];
};

template <typename T>
__device__ __forceinline__ const Sten<T>& op_of(const Geo<T>& g, int op, int j) {
    return op == OP_A ? g.A[j] : (op == OP_M ? g.M[j] : (op == OP_B ? g.B[j] : g.Bd[j]));
}

template <int D>
struct UTileMax {
    static constexpr int T0 = UTile<D>::T0, T1 = UTile<D>::T1, T2 = UTile<D>::T2;
    static constexpr int v = T0 > T1 ? (T0 > T2 ? T0 : T2) : (T1 > T2 ? T1 : T2);
};

// Value boxes of a u-row tile (staged path): the x values at the tile's u-column
// lists (capX = prod cap of tu) and, per component, the psi values at its psi-column
// lists (capZ = prod cap of tp), both converted to T.
template <typename T>
__host__ __device__ inline long long urow_box_x(const Geo<T>& g) {
    long long c = 1;
    for (int j = 0; j < g.d; ++j) c *= g.tu[j].cap;
    return c;
}
template <typename T>
__host__ __device__ inline long long urow_box_z(const Geo<T>& g) {
    long long c = 1;
    for (int j = 0; j < g.d; ++j) c *= g.tp[j].cap;
    return c;
}

// Body of the tiled u-row apply for the tile with linear index `blin`
// (x-tiles fastest); `stp` points to the block's shared StenTile, followed (staged
// path) by the tile's value boxes.  Staged: the x and psi values the tile's rows
// touch are first copied into shared memory (all loads in flight together, one
// barrier), and the gathers read the boxes through the stencils' tile-local columns.
template <int D, typename T, typename Tx, typename Tz, bool HAS_A, bool HAS_B, bool RESID>
__device__ __forceinline__ void k_urow_body(const Geo<T>& g, T cA, const Tx* __restrict__ x, T cB,
                                            const Tz* __restrict__ z, const Tz* __restrict__ z2,
                                            const double* __restrict__ rA, const double* __restrict__ bf,
                                            double* __restrict__ yres, double* __restrict__ part,
                                            Tx* __restrict__ y, int blin, void* stp) {
    constexpr int T0 = UTile<D>::T0, T1 = UTile<D>::T1, T2 = UTile<D>::T2;
    constexpr int TMAX = UTileMax<D>::v;
    StenTile<T, TMAX>& st = *reinterpret_cast<StenTile<T, TMAX>*>(stp);
    T* xs = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(stp) + sizeof(StenTile<T, TMAX>));
    T* zs = xs + (HAS_A ? urow_box_x(g) : 0);
    const long long capZ = urow_box_z(g);
    __shared__ double sh[32];
    const int tile[kMaxDim] = {T0, T1, T2};
    const int gx = (g.n1[0] + T0 - 1) / T0, gy = (g.n1[1] + T1 - 1) / T1;
    const int tix[kMaxDim] = {blin % gx, (blin / gx) % gy, blin / (gx * gy)};
    const int org[kMaxDim] = {tix[0] * T0, tix[1] * T1, tix[2] * T2};
    const bool grad = g.kind == HPG_GRADIENT;
    const bool staged = g.staged != 0;
    // FP64, unstaged path: rows along axis 0 in the order perm0 (equal stencil counts side
    // by side, so the lanes of a warp run loops of equal length); the staged path keeps the
    // natural order its column lists were built for, and the FP32 kernels (bound by gather
    // latency, not arithmetic) are compiled without it
    const int* perm0 = (sizeof(T) == 8 && !staged) ? g.perm0 : nullptr;
    // stage the stencil rows of this tile (tile-local columns on the staged path)
    for (int op = 0; op < NOPS; ++op) {
        if ((op == OP_A || op == OP_M) && !HAS_A) continue;
        if (op == OP_B && !HAS_B) continue;
        if (op == OP_BD && !(HAS_B && grad)) continue;
        for (int j = 0; j < D; ++j) {
            const Sten<T>& S = op_of(g, op, j);
            const int* cols = staged ? S.lcol : S.col;
            for (int e = threadIdx.x; e < tile[j] * kEll; e += blockDim.x) {
                const int l = e / kEll, k = e % kEll, pos = org[j] + l;
                if (pos < g.n1[j]) {
                    const int r = (j == 0 && perm0) ? perm0[pos] : pos;
                    st.col[op][j][l][k] = cols[(size_t)r * kEll + k];
                    st.val[op][j][l][k] = S.val[(size_t)r * kEll + k];
                    if (k == 0) st.cnt[op][j][l] = S.cnt[r];
                } else if (k == 0) {
                    st.cnt[op][j][l] = 0;
                }
            }
        }
    }
    int L[kMaxDim] = {1, 1, 1}, Pn[kMaxDim] = {1, 1, 1};
    if (staged) {
        const int n1x = g.n1[0], n1y = g.n1[1];
        if (HAS_A) {
            for (int j = 0; j < D; ++j) L[j] = g.tu[j].count[tix[j]];
            const int* ux = g.tu[0].list + (size_t)tix[0] * g.tu[0].cap;
            const int* uy = g.tu[1].list + (size_t)tix[1] * g.tu[1].cap;
            const int* uz = D == 3 ? g.tu[2].list + (size_t)tix[2] * g.tu[2].cap : nullptr;
            const int tot = L[0] * L[1] * L[2];
            for (int e = threadIdx.x; e < tot; e += blockDim.x) {
                const int lx = e % L[0], ly = (e / L[0]) % L[1], lz = e / (L[0] * L[1]);
                const long long zz = D == 3 ? uz[lz] : 0;
                xs[e] = (T)x[(zz * n1y + uy[ly]) * n1x + ux[lx]];
            }
        }
        if (HAS_B) {
            for (int j = 0; j < D; ++j) Pn[j] = g.tp[j].count[tix[j]];
            const int* px = g.tp[0].list + (size_t)tix[0] * g.tp[0].cap;
            const int* py = g.tp[1].list + (size_t)tix[1] * g.tp[1].cap;
            const int* pz = D == 3 ? g.tp[2].list + (size_t)tix[2] * g.tp[2].cap : nullptr;
            const int tot = Pn[0] * Pn[1] * Pn[2];
            const int n = g.n;
            for (int e = threadIdx.x; e < tot * g.ncomp; e += blockDim.x) {
                const int comp = e / tot, le = e - comp * tot;
                const int lx = le % Pn[0], ly = (le / Pn[0]) % Pn[1], lz = le / (Pn[0] * Pn[1]);
                const int p0 = px[lx], p1 = py[ly], p2 = D == 3 ? pz[lz] : 0;
                const long long cell = (p0 >> 8) + (long long)g.m[0] * ((p1 >> 8) + (long long)g.m[1] * (p2 >> 8));
                const long long idx = (cell * g.ncomp + comp) * g.nloc + (p0 & 255) + n * ((p1 & 255) + n * (p2 & 255));
                T v = (T)z[idx];
                if (z2) v -= (T)z2[idx];
                zs[(long long)comp * capZ + le] = v;
            }
        }
    }
    __syncthreads();
    const int l0 = threadIdx.x % T0, l1 = (threadIdx.x / T0) % T1, l2 = threadIdx.x / (T0 * T1);
    const int p0 = org[0] + l0, r1 = org[1] + l1, r2 = (D == 3) ? org[2] + l2 : 0;
    const bool inside = p0 < g.n1[0] && r1 < g.n1[1] && (D == 2 || r2 < g.n1[2]);
    const int r0 = (perm0 && inside) ? perm0[p0] : p0;
    const int n1x = g.n1[0], n1y = g.n1[1];
    double v = 0.0;
    long long i = 0;
    if (inside) {
        i = r0 + (long long)n1x * (r1 + (long long)n1y * r2);
        T acc = T(0);
        if (HAS_A) {
            // x values: the staged box [lz][ly][lx] or the global vector
            const long long sy = staged ? L[0] : n1x, sz = staged ? (long long)L[0] * L[1] : (long long)n1x * n1y;
            T sa = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int o0 = (k == 0) ? OP_A : OP_M, o1 = (k == 1) ? OP_A : OP_M, o2 = (k == 2) ? OP_A : OP_M;
                const int c0 = st.cnt[o0][0][l0], c1 = st.cnt[o1][1][l1];
                if (D == 2) {
                    for (int e1 = 0; e1 < c1; ++e1) {
                        const long long base = (long long)st.col[o1][1][l1][e1] * sy;
                        T t = T(0);
                        if (staged)
                            for (int e0 = 0; e0 < c0; ++e0) t += st.val[o0][0][l0][e0] * xs[base + st.col[o0][0][l0][e0]];
                        else
                            for (int e0 = 0; e0 < c0; ++e0)
                                t += st.val[o0][0][l0][e0] * (T)x[base + st.col[o0][0][l0][e0]];
                        sa += st.val[o1][1][l1][e1] * t;
                    }
                } else {
                    const int c2 = st.cnt[o2][2][l2];
                    for (int e2 = 0; e2 < c2; ++e2) {
                        const long long b2 = (long long)st.col[o2][2][l2][e2] * sz;
                        T t2 = T(0);
                        for (int e1 = 0; e1 < c1; ++e1) {
                            const long long base = b2 + (long long)st.col[o1][1][l1][e1] * sy;
                            T t = T(0);
                            if (staged)
                                for (int e0 = 0; e0 < c0; ++e0)
                                    t += st.val[o0][0][l0][e0] * xs[base + st.col[o0][0][l0][e0]];
                            else
                                for (int e0 = 0; e0 < c0; ++e0)
                                    t += st.val[o0][0][l0][e0] * (T)x[base + st.col[o0][0][l0][e0]];
                            t2 += st.val[o1][1][l1][e1] * t;
                        }
                        sa += st.val[o2][2][l2][e2] * t2;
                    }
                }
            }
            acc += cA * sa;
        }
        if (HAS_B) {
            T sb = T(0);
            const int n = g.n;
            for (int comp = 0; comp < g.ncomp; ++comp) {
                const int o0 = (grad && comp == 0) ? OP_BD : OP_B, o1 = (grad && comp == 1) ? OP_BD : OP_B,
                          o2 = (grad && comp == 2) ? OP_BD : OP_B;
                const int c0 = st.cnt[o0][0][l0], c1 = st.cnt[o1][1][l1];
                const int c2 = (D == 3) ? st.cnt[o2][2][l2] : 1;
                const T* zc = zs + (long long)comp * capZ;
                for (int e2 = 0; e2 < c2; ++e2) {
                    int cz = 0, kz = 0;
                    T vz = T(1);
                    if (D == 3) {
                        const int p2 = st.col[o2][2][l2][e2];
                        cz = p2 >> 8; kz = p2 & 255; vz = st.val[o2][2][l2][e2];
                    }
                    T t2 = T(0);
                    for (int e1 = 0; e1 < c1; ++e1) {
                        const int p1 = st.col[o1][1][l1][e1];
                        T t = T(0);
                        if (staged) {
                            // tile-local columns: positions in the psi-column lists
                            const long long base = ((long long)(D == 3 ? st.col[o2][2][l2][e2] : 0) * Pn[1] + p1) * Pn[0];
                            for (int e0 = 0; e0 < c0; ++e0) t += st.val[o0][0][l0][e0] * zc[base + st.col[o0][0][l0][e0]];
                        } else {
                            const int cy = p1 >> 8, ky = p1 & 255;
                            for (int e0 = 0; e0 < c0; ++e0) {
                                const int p0 = st.col[o0][0][l0][e0];
                                const int cx = p0 >> 8, kx = p0 & 255;
                                const long long cell = cx + (long long)g.m[0] * (cy + (long long)g.m[1] * cz);
                                const long long idx = (cell * g.ncomp + comp) * g.nloc + kx + n * (ky + n * kz);
                                T zv = (T)z[idx];
                                if (z2) zv -= (T)z2[idx];
                                t += st.val[o0][0][l0][e0] * zv;
                            }
                        }
                        t2 += st.val[o1][1][l1][e1] * t;
                    }
                    sb += vz * t2;
                }
            }
            acc += cB * sb;
        }
        if (RESID) {
            const double r = (double)acc + (double)cA * (rA[i] - bf[i]);
            yres[i] = r;
            v = r * r;
        } else {
            y[i] = (Tx)acc;
        }
    }
    if (RESID) {
        v = block_sum(v, sh);
        if (threadIdx.x == 0) part[blin] = v;
    }
}

// Grid: x, y tiles along axes 0, 1; z = (tiles along axis 2) x (problems of the batch),
// the problem index slowest.  cA is read per problem from Bat::par (kParAlpha) when
// `ca_from_par` is set (the residual's alpha).
template <int D, typename T, typename Tx, typename Tz, bool HAS_A, bool HAS_B, bool RESID>
__global__ void __launch_bounds__(256)
    k_urow(Geo<T> g, T cA, const Tx* __restrict__ x, T cB, const Tz* __restrict__ z, const Tz* __restrict__ z2,
           const double* __restrict__ rA, const double* __restrict__ bf, double* __restrict__ yres,
           double* __restrict__ part, Tx* __restrict__ y, const int* skip, Bat bt, int ca_from_par) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tz = (int)gridDim.z / bt.np;
    const int pb = (int)blockIdx.z / tz, bz = (int)blockIdx.z - pb * tz;
    long long off;
    if (!bat_enter(bt, pb, &off)) return;
    skip = bsh(skip, off);
    if (skip && *skip) return;
    x = bsh(x, off); z = bsh(z, off); z2 = bsh(z2, off); rA = bsh(rA, off); bf = bsh(bf, off);
    yres = bsh(yres, off); part = bsh(part, off); y = bsh(y, off);
    if (ca_from_par) cA = (T)bt.par[pb * kBatPar + kParAlpha];
    const int blin = (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * bz));
    k_urow_body<D, T, Tx, Tz, HAS_A, HAS_B, RESID>(g, cA, x, cB, z, z2, rA, bf, yres, part, y, blin, smraw);
}

// dynamic shared memory of a tiled u-row launch: the stencil tile, then the value
// boxes it stages (only on the staged path)
template <int D, typename T>
static size_t urow_smem(const Geo<T>& g, bool has_a, bool has_b) {
    size_t b = sizeof(StenTile<T, UTileMax<D>::v>);
    if (g.staged) b += (size_t)((has_a ? urow_box_x(g) : 0) + (has_b ? g.ncomp * urow_box_z(g) : 0)) * sizeof(T);
    return b;
}

// the staged path is taken when the boxes of the heaviest launch (residual / Newton
// apply: x box and psi boxes) fit this budget next to the stencil tile
constexpr size_t kUrowBoxBudget = 96 * 1024;

template <typename T>
bool urow_boxes_fit(const Geo<T>& g) {
    return (size_t)(urow_box_x(g) + g.ncomp * urow_box_z(g)) * sizeof(T) <= kUrowBoxBudget;
}
template bool urow_boxes_fit<float>(const Geo<float>&);
template bool urow_boxes_fit<double>(const Geo<double>&);

int utile_extent(int d, int axis) {
    if (d == 2) return axis == 0 ? UTile<2>::T0 : (axis == 1 ? UTile<2>::T1 : 1);
    return axis == 0 ? UTile<3>::T0 : (axis == 1 ? UTile<3>::T1 : UTile<3>::T2);
}

template <int D>
static dim3 utile_grid(const int* n1, int np = 1) {
    return dim3((n1[0] + UTile<D>::T0 - 1) / UTile<D>::T0, (n1[1] + UTile<D>::T1 - 1) / UTile<D>::T1,
                (D == 3 ? (n1[2] + UTile<D>::T2 - 1) / UTile<D>::T2 : 1) * np);
}

static long long utile_blocks(int d, const int* n1) {
    const dim3 gr = d == 2 ? utile_grid<2>(n1) : utile_grid<3>(n1);
    return (long long)gr.x * gr.y * gr.z;
}


void add_kernel_launches(long long n) { t_launches += n; }

// ====================================================================== eval
// Obstacle: g_q = w_q |J| exp(-psi(x_q)), eg = V^T g per cell (Section 5, Quadrature).
// Gradient: psi_q (d comps), s = 1 + |psi_q|^2, G = phi psi / sqrt(s) projected into eg,
// Jacobian J_ab = phi (s d_ab - psi_a psi_b) s^{-3/2} (times w|J|) packed into gw.
__global__ void k_eval(Geo<double> g, const double* __restrict__ psi, const double* __restrict__ phiq,
                       double* __restrict__ gw, float* __restrict__ gwf, double* __restrict__ eg,
                       int* __restrict__ flag, Bat bt) {
    extern __shared__ double sm[];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    psi = bsh(psi, off); phiq = bsh(phiq, off); gw = bsh(gw, off); gwf = bsh(gwf, off); eg = bsh(eg, off);
    flag = bsh(flag, off);
    const int n = g.n, nloc = (int)g.nloc, nc = g.ncomp;
    double* a = sm;
    double* b = sm + nc * nloc;
    double* Vq = sm + 2 * nc * nloc;
    const long long c = blockIdx.x;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Vq[i] = g.Vq[i];
    for (int i = threadIdx.x; i < nc * nloc; i += blockDim.x) a[i] = psi[c * nc * nloc + i];
    __syncthreads();
    double *in = a, *out = b;
    int stride = 1;
    for (int ax = 0; ax < g.d; ++ax) {
        sf_pass(in, out, Vq, false, n, nloc, nc, stride);
        __syncthreads();
        double* t = in; in = out; out = t;
        stride *= n;
    }
    // in: Gauss values per component
    const int gs = (g.kind == HPG_GRADIENT) ? g.d * (g.d + 1) / 2 : 1;
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
        double w = g.detJ;
        int qq = q;
        for (int ax = 0; ax < g.d; ++ax) { w *= g.wq[qq % n]; qq /= n; }
        const long long gq = c * nloc + q;
        if (g.kind != HPG_GRADIENT) {
            const double pv = in[q];
            if (!(pv >= -700.0) || !isfinite(pv)) atomicOr(flag, 1);
            const double v = w * exp(-pv);
            out[q] = v;
            gw[gq] = v;
            if (gwf) gwf[gq] = (float)v;
        } else {
            double pv[kMaxDim];
            double s = 1.0;
            for (int k = 0; k < nc; ++k) { pv[k] = in[k * nloc + q]; s += pv[k] * pv[k]; }
            if (!isfinite(s)) atomicOr(flag, 1);
            const double ph = phiq[gq];
            const double rs = 1.0 / sqrt(s);
            const double r3 = rs * rs * rs;
            for (int k = 0; k < nc; ++k) out[k * nloc + q] = w * ph * pv[k] * rs;
            int e = 0;
            for (int k = 0; k < nc; ++k)
                for (int l = k; l < nc; ++l, ++e) {
                    const double jv = w * ph * ((k == l ? s : 0.0) - pv[k] * pv[l]) * r3;
                    gw[gq * gs + e] = jv;
                    if (gwf) gwf[gq * gs + e] = (float)jv;
                }
        }
    }
    __syncthreads();
    { double* t = in; in = out; out = t; }
    stride = 1;
    for (int ax = 0; ax < g.d; ++ax) {
        sf_pass(in, out, Vq, true, n, nloc, nc, stride);
        __syncthreads();
        double* t = in; in = out; out = t;
        stride *= n;
    }
    for (int i = threadIdx.x; i < nc * nloc; i += blockDim.x) eg[c * nc * nloc + i] = in[i];
}

cudaError_t launch_eval(const Geo<double>& g, const double* psi, const double* phiq, double* gw, float* gwf,
                        double* eg, int* flag, cudaStream_t s, const Bat& bt) {
    const size_t smem = (size_t)(2 * g.ncomp * g.nloc + g.n * g.n) * sizeof(double);
    const int threads = g.nloc * g.ncomp >= 256 ? 256 : 128;
    k_eval<<<dim3((unsigned)g.Nc, bt.np), threads, smem, s>>>(g, psi, phiq, gw, gwf, eg, flag, bt);
    note_launch();
    return cudaGetLastError();
}

// (phi, zeta) = V^T (w |J| phi_q) per cell (the same Gauss rule as the latent terms)
__global__ void k_project(Geo<double> g, const double* __restrict__ phiq, double* __restrict__ phiz) {
    extern __shared__ double sm[];
    const int n = g.n, nloc = (int)g.nloc;
    double* a = sm;
    double* b = sm + nloc;
    double* Vq = sm + 2 * nloc;
    const long long c = blockIdx.x;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Vq[i] = g.Vq[i];
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
        double w = g.detJ;
        int qq = q;
        for (int ax = 0; ax < g.d; ++ax) { w *= g.wq[qq % n]; qq /= n; }
        a[q] = w * phiq[c * nloc + q];
    }
    __syncthreads();
    double *in = a, *out = b;
    int stride = 1;
    for (int ax = 0; ax < g.d; ++ax) {
        sf_pass(in, out, Vq, true, n, nloc, 1, stride);
        __syncthreads();
        double* t = in; in = out; out = t;
        stride *= n;
    }
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) phiz[c * nloc + i] = in[i];
}

cudaError_t launch_project(const Geo<double>& g, const double* phiq, double* phiz, cudaStream_t s) {
    const size_t smem = (size_t)(2 * g.nloc + g.n * g.n) * sizeof(double);
    k_project<<<(unsigned)g.Nc, 128, smem, s>>>(g, phiq, phiz);
    note_launch();
    return cudaGetLastError();
}

// ================================================================== residual
template <int D>
__global__ void k_residual_psi(Geo<double> g, const double* __restrict__ u, const double* __restrict__ eg,
                               const double* __restrict__ rB, const double* __restrict__ phiz,
                               double* __restrict__ F, double* __restrict__ part, Bat bt) {
    __shared__ double sh[32];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    u = bsh(u, off); eg = bsh(eg, off); rB = bsh(rB, off); phiz = bsh(phiz, off); F = bsh(F, off);
    part = bsh(part, off);
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (j < g.Npsi) {
        const long long cell = j / g.nb;
        const int rem = (int)(j - cell * g.nb);
        const int comp = rem / (int)g.nloc;
        int km[kMaxDim], cm[kMaxDim];
        int kk = rem - comp * (int)g.nloc;
        for (int t = 0; t < D; ++t) { km[t] = kk % g.n; kk /= g.n; }
        cell_multi(g, cell, cm);
        const double bt_ = apply_BT_entry<D, double, double>(g, cm, comp, km, u);
        if (g.kind == HPG_GRADIENT) v = bt_ + rB[j] - eg[j];
        else v = bt_ + rB[j] + eg[j] - phiz[j];
        F[j] = v;
    }
    v = block_sum(v * v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

int n_res_partials(const Geo<double>& g) {
    return (int)(utile_blocks(g.d, g.n1) + (g.Npsi + 255) / 256);
}

int n_res_partials_for(int d, const int* n1, long long Npsi) {
    return (int)(utile_blocks(d, n1) + (Npsi + 255) / 256);
}

cudaError_t launch_residual(const Geo<double>& g, const double* u, const double* psi, const double* psi_prev,
                            const double* eg, const double* rA, const double* rB, const double* bf,
                            const double* phiz, double alpha, double* F, double* part, cudaStream_t s,
                            const Bat& bt) {
    const int bu = (int)utile_blocks(g.d, g.n1), bp = (int)((g.Npsi + 255) / 256);
    const int from_par = bt.par ? 1 : 0;
    if (g.d == 2) {
        k_urow<2, double, double, double, true, true, true><<<utile_grid<2>(g.n1, bt.np), 256,
                                                                 urow_smem<2>(g, true, true), s>>>(
            g, alpha, u, 1.0, psi, psi_prev, rA, bf, F, part, nullptr, nullptr, bt, from_par);
        note_launch();
        k_residual_psi<2><<<dim3(bp, bt.np), 256, 0, s>>>(g, u, eg, rB, phiz, F + g.Nu0, part + bu, bt);
        note_launch();
    } else {
        k_urow<3, double, double, double, true, true, true><<<utile_grid<3>(g.n1, bt.np), 256,
                                                                 urow_smem<3>(g, true, true), s>>>(
            g, alpha, u, 1.0, psi, psi_prev, rA, bf, F, part, nullptr, nullptr, bt, from_par);
        note_launch();
        k_residual_psi<3><<<dim3(bp, bt.np), 256, 0, s>>>(g, u, eg, rB, phiz, F + g.Nu0, part + bu, bt);
        note_launch();
    }
    return cudaGetLastError();
}

__global__ void k_reduce_sum(const double* __restrict__ part, int count, double* __restrict__ out, Bat bt) {
    __shared__ double sh[32];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.x, &off)) return;
    part = bsh(part, off);
    out = bsh(out, off);
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v += part[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[0] = v;
}

cudaError_t launch_reduce_sum(const double* part, int count, double* out, cudaStream_t s, const Bat& bt) {
    k_reduce_sum<<<bt.np, 1024, 0, s>>>(part, count, out, bt);
    note_launch();
    return cudaGetLastError();
}

// ==================================================================== factor
// Assemble -S-hat_K = D_K + beta M_K + C/alpha (obstacle) or D_K + beta K_K (gradient)
// by sum factorisation over the Gauss points, factor it (Cholesky, L L^T), invert
// L (X = L^{-1}, kept transposed in the upper triangle), and write (-S-hat_K)^{-1} = X^T X.
// The thread group is the whole block (WARP false: lt = threadIdx.x, nthr = blockDim.x,
// block barriers) or one warp (WARP true: lt = lane, nthr = 32, warp barriers).
template <typename T, bool WARP = false>
__device__ void assemble_D_block(const Geo<T>& g, const T* __restrict__ gw, long long cell, int gs, int ge,
                                 const T* Vq, T* bufA, T* bufB, int lt = -1, int nthr = 0) {
    if (lt < 0) { lt = threadIdx.x; nthr = blockDim.x; }
    // stage 0: X0[q] = gw[q]; stage s contracts q_{d-s-1}; final X_d = D (nloc x nloc) in bufA
    const int n = g.n, d = g.d, nloc = (int)g.nloc;
    T* cur = ((d % 2) == 0) ? bufA : bufB;
    for (int q = lt; q < nloc; q += nthr) cur[q] = gw[(cell * nloc + q) * gs + ge];
    if (WARP) __syncwarp(); else __syncthreads();
    int nq_out = nloc;      // n^{d-s}
    int ns = 1;             // n^s
    for (int st = 0; st < d; ++st) {
        T* nxt = (((d - st - 1) % 2) == 0) ? bufA : bufB;
        const int nq_new = nq_out / n;          // n^{d-s-1}
        const int ns_new = ns * n;
        const int total = nq_new * ns_new * ns_new;
        for (int o = lt; o < total; o += nthr) {
            const int J = o % ns_new;
            const int rest = o / ns_new;
            const int I = rest % ns_new;
            const int Qp = rest / ns_new;
            const int i = I % n, Is = I / n;
            const int j = J % n, Js = J / n;
            T s = T(0);
            for (int q = 0; q < n; ++q) {
                const T w = Vq[q * n + i] * Vq[q * n + j];
                s += w * cur[(((long long)(Qp + nq_new * q) * ns + Is) * ns) + Js];
            }
            nxt[o] = s;
        }
        if (WARP) __syncwarp(); else __syncthreads();
        cur = nxt;
        nq_out = nq_new;
        ns = ns_new;
    }
}

template <typename T>
__global__ void k_factor(Geo<T> g, const T* __restrict__ gw, T alpha_inv, T beta, T* __restrict__ Sinv,
                         double* __restrict__ dump, int* __restrict__ flag, T* __restrict__ gwork, int use_smem,
                         Bat bt) {
    extern __shared__ unsigned char smraw[];
    long long off;
    const int pb = (int)blockIdx.y;
    if (!bat_enter(bt, pb, &off)) return;
    gw = bsh(gw, off); Sinv = bsh(Sinv, off); dump = bsh(dump, off); flag = bsh(flag, off); gwork = bsh(gwork, off);
    if (bt.par) alpha_inv = (T)(1.0 / bt.par[pb * kBatPar + kParAlpha]);
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = g.n, nloc = (int)g.nloc, nb = (int)g.nb, nc = g.ncomp;
    const long long cell = blockIdx.x;
    // workspace layout: A (nb^2) | bufA (nloc^2, gradient only) | bufB (n^{2d-1}) | Vq (n^2) | ldiag (nb)
    size_t nbuf_b = 1;
    for (int t = 0; t < 2 * g.d - 1; ++t) nbuf_b *= n;
    T* base = use_smem ? sm : gwork + cell * ((size_t)nb * nb + (nc > 1 ? (size_t)nloc * nloc : 0) + nbuf_b + n * n + nb);
    T* A = base;
    T* bufA = (nc > 1) ? A + (size_t)nb * nb : A;
    T* bufB = bufA + (nc > 1 ? (size_t)nloc * nloc : (size_t)nb * nb);
    T* Vq = bufB + nbuf_b;
    T* ldiag = Vq + n * n;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Vq[i] = g.Vq[i];
    __syncthreads();
    const int gs = (g.kind == HPG_GRADIENT) ? g.d * (g.d + 1) / 2 : 1;
    if (nc == 1) {
        assemble_D_block(g, gw, cell, 1, 0, Vq, A, bufB);
        for (int o = threadIdx.x; o < nloc * nloc; o += blockDim.x) {
            const int I = o / nloc, J = o % nloc;
            T v = A[o] + g.C[o] * alpha_inv;
            if (I == J) v += beta * g.Mpsi[I];
            A[o] = v;
        }
    } else {
        int e = 0;
        for (int ca = 0; ca < nc; ++ca)
            for (int cb = ca; cb < nc; ++cb, ++e) {
                assemble_D_block(g, gw, cell, gs, e, Vq, bufA, bufB);
                for (int o = threadIdx.x; o < nloc * nloc; o += blockDim.x) {
                    const int I = o / nloc, J = o % nloc;
                    T v = bufA[o];
                    if (ca == cb) v += beta * g.Kpsi[o];
                    A[(size_t)(ca * nloc + I) * nb + cb * nloc + J] = v;
                    A[(size_t)(cb * nloc + J) * nb + ca * nloc + I] = v;
                }
                __syncthreads();
            }
    }
    __syncthreads();
    if (dump)
        for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) dump[cell * nb * nb + o] = (double)A[o];
    // Cholesky (right-looking), lower triangle; two barriers per column: every thread
    // takes the pivot's square root itself (the pivot is final after the previous
    // step) and scales its part of column k; the trailing update runs warps over rows
    // and lanes over columns j <= i (no index division, no idle upper half)
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
    __syncthreads();
    __shared__ T piv;
    for (int k = 0; k < nb; ++k) {
        T lkk;
        if constexpr (sizeof(T) == 8) {
            // FP64 square roots are costly on this GPU's FP64 pipe: one thread takes it
            if (threadIdx.x == 0) {
                T pv = A[(size_t)k * nb + k];
                if (!(pv > T(0))) { bad = 1; pv = T(1); }
                piv = sqrt(pv);
            }
            __syncthreads();
            lkk = piv;
        } else {
            T pv = A[(size_t)k * nb + k];
            if (!(pv > T(0))) {
                if (threadIdx.x == 0) bad = 1;
                pv = T(1);
            }
            lkk = sqrt(pv);
        }
        for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) A[(size_t)i * nb + k] /= lkk;
        __syncthreads();
        if (threadIdx.x == 0) A[(size_t)k * nb + k] = lkk;
        for (int i = k + 1 + ty; i < nb; i += nty) {
            const T lik = A[(size_t)i * nb + k];
            for (int j = k + 1 + tx; j <= i; j += 32) A[(size_t)i * nb + j] -= lik * A[(size_t)j * nb + k];
        }
        __syncthreads();
    }
    // non-SPD pivot: bit 1 of flag[1] (flag[0] holds the evaluation's flags, which each
    // line-search trial clears; this one stays set until the next solve)
    if (threadIdx.x == 0 && bad) atomicOr(flag + 1, 2);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) ldiag[i] = A[(size_t)i * nb + i];
    __syncthreads();
    // X = L^{-1}, column j per thread; X[i][j] stored at A[j][i] (i >= j)
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        A[(size_t)j * nb + j] = T(1) / ldiag[j];
        for (int i = j + 1; i < nb; ++i) {
            T s = T(0);
            for (int k = j; k < i; ++k) s += A[(size_t)i * nb + k] * A[(size_t)j * nb + k];
            A[(size_t)j * nb + i] = -s / ldiag[i];
        }
    }
    __syncthreads();
    // Sinv[i][j] = sum_{k >= max(i,j)} X[k][i] X[k][j] = sum_k A[i][k] A[j][k]
    T* out = Sinv + cell * (long long)nb * nb;
    for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
        const int i = o / nb, j = o % nb;
        const int k0 = i > j ? i : j;
        T s = T(0);
        for (int k = k0; k < nb; ++k) s += A[(size_t)i * nb + k] * A[(size_t)j * nb + k];
        out[o] = s;
    }
}

// ---- one warp per cell (blocks of at most kFactorWarpMaxNb) ----------------------
// The block kernel above runs one cell per 256-thread block and spends its time in
// block barriers (two per Cholesky column) and in a triangular inverse with one busy
// thread per column.  Here each warp owns one cell: it assembles -S-hat_K in shared
// memory (the same sum factorisation) and inverts it in place by Gauss-Jordan
// elimination without pivoting -- the block is SPD, so every pivot is positive; a
// non-positive one is flagged as for the Cholesky.  Lane l owns columns l, l + 32 and
// l + 64 of the block; step k first copies column k (the elimination multipliers) to a
// per-warp buffer, so the lanes only ever write their own columns and synchronise with
// __syncwarp.  Work per cell: nb^3 multiply-adds, all 32 lanes busy at every step.
constexpr int kFactorWarpMaxNb = 96;

__host__ __device__ inline size_t factor_warp_elems(int n, int d, int nb, int nc) {
    size_t nloc = 1, nbuf_b = 1;
    for (int t = 0; t < d; ++t) nloc *= n;
    for (int t = 0; t < 2 * d - 1; ++t) nbuf_b *= n;
    // A (nb^2) | bufA (nloc^2, gradient only) | bufB (n^{2d-1}) | Vq (n^2) | column k (nb) or
    // the two row buffers of the register variant (2 x 64), 16-byte aligned
    size_t e = (size_t)nb * nb + (nc > 1 ? nloc * nloc : 0) + nbuf_b + (size_t)n * n;
    e = (e + 3) & ~(size_t)3;
    return e + (nb > 128 ? (size_t)nb : 128);
}

// R > 0: the register variant for nb <= 32 R.  Lane l keeps rows l + 32 r (r < R) of
// the block in registers, padded to 32 R columns (and with identity rows past nb);
// step k has the owner of row k publish it through a double-buffered shared row, and
// every lane eliminates with one multiply-add per register -- no shared-memory
// traffic per element, so the elimination runs at the FMA rate.
template <typename T, int R>
__global__ void __launch_bounds__(128)
    k_factor_warp(Geo<T> g, const T* __restrict__ gw, T alpha_inv, T beta, T* __restrict__ Sinv,
                  double* __restrict__ dump, int* __restrict__ flag, int wpb, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    const int pb = (int)blockIdx.y;
    if (!bat_enter(bt, pb, &off)) return;
    gw = bsh(gw, off); Sinv = bsh(Sinv, off); dump = bsh(dump, off); flag = bsh(flag, off);
    if (bt.par) alpha_inv = (T)(1.0 / bt.par[pb * kBatPar + kParAlpha]);
    const int n = g.n, nloc = (int)g.nloc, nb = (int)g.nb, nc = g.ncomp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long cell = (long long)blockIdx.x * wpb + warp;
    if (cell >= g.Nc) return;                    // whole warps only; no block barrier below
    const size_t per = factor_warp_elems(n, g.d, nb, nc);
    T* A = reinterpret_cast<T*>(smraw) + (size_t)warp * per;
    T* bufA = (nc > 1) ? A + (size_t)nb * nb : A;
    T* bufB = bufA + (nc > 1 ? (size_t)nloc * nloc : (size_t)nb * nb);
    T* Vq = bufB;
    {
        size_t nbuf_b = 1;
        for (int t = 0; t < 2 * g.d - 1; ++t) nbuf_b *= n;
        Vq = bufB + nbuf_b;
    }
    T* colk = reinterpret_cast<T*>(smraw) + (size_t)warp * per + (per - (nb > 128 ? nb : 128));
    for (int i = lane; i < n * n; i += 32) Vq[i] = g.Vq[i];
    __syncwarp();
    const int gs = (g.kind == HPG_GRADIENT) ? g.d * (g.d + 1) / 2 : 1;
    if (nc == 1) {
        assemble_D_block<T, true>(g, gw, cell, 1, 0, Vq, A, bufB, lane, 32);
        for (int o = lane; o < nloc * nloc; o += 32) {
            const int I = o / nloc, J = o % nloc;
            T v = A[o] + g.C[o] * alpha_inv;
            if (I == J) v += beta * g.Mpsi[I];
            A[o] = v;
        }
    } else {
        int e = 0;
        for (int ca = 0; ca < nc; ++ca)
            for (int cb = ca; cb < nc; ++cb, ++e) {
                assemble_D_block<T, true>(g, gw, cell, gs, e, Vq, bufA, bufB, lane, 32);
                for (int o = lane; o < nloc * nloc; o += 32) {
                    const int I = o / nloc, J = o % nloc;
                    T v = bufA[o];
                    if (ca == cb) v += beta * g.Kpsi[o];
                    A[(size_t)(ca * nloc + I) * nb + cb * nloc + J] = v;
                    A[(size_t)(cb * nloc + J) * nb + ca * nloc + I] = v;
                }
                __syncwarp();
            }
    }
    __syncwarp();
    if (dump)
        for (int o = lane; o < nb * nb; o += 32) dump[cell * nb * nb + o] = (double)A[o];
    bool bad = false;
    if constexpr (R > 0) {
        constexpr int NM = 32 * R;
        T a[R][NM];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
#pragma unroll
            for (int j = 0; j < NM; ++j) a[r][j] = (i < nb && j < nb) ? A[(size_t)i * nb + j] : T(i == j ? 1 : 0);
        }
        T* rb0 = colk;
        T* rb1 = colk + 64;
        // the published row moves in 16-byte words: 4 floats (2 doubles) per load
        constexpr int VW = 16 / (int)sizeof(T);
        using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            if (k >= nb) break;
            T* rb = (k & 1) ? rb1 : rb0;
            if (lane == (k & 31)) {
#pragma unroll
                for (int q = 0; q < NM / VW; ++q) {
                    V16 v;
                    T* vt = reinterpret_cast<T*>(&v);
#pragma unroll
                    for (int u = 0; u < VW; ++u) vt[u] = a[k >> 5][VW * q + u];
                    reinterpret_cast<V16*>(rb)[q] = v;
                }
            }
            __syncwarp();
            T row[NM];
#pragma unroll
            for (int q = 0; q < NM / VW; ++q) {
                const V16 v = reinterpret_cast<const V16*>(rb)[q];
                const T* vt = reinterpret_cast<const T*>(&v);
#pragma unroll
                for (int u = 0; u < VW; ++u) row[VW * q + u] = vt[u];
            }
            T p = row[k];
            if (!(p > T(0))) { bad = true; p = T(1); }
            const T inv = T(1) / p;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool is_k = lane + 32 * r == k;
                const T f = a[r][k];
                const T fp = is_k ? T(1) - inv : f * inv;
#pragma unroll
                for (int j = 0; j < NM; ++j)
                    if (j != k) a[r][j] -= fp * row[j];
                a[r][k] = is_k ? inv : -fp;
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            if (i < nb)
#pragma unroll
                for (int j = 0; j < NM; ++j)
                    if (j < nb) A[(size_t)i * nb + j] = a[r][j];
        }
        __syncwarp();
    } else {
    for (int k = 0; k < nb; ++k) {
        for (int i = lane; i < nb; i += 32) colk[i] = A[(size_t)i * nb + k];
        __syncwarp();
        T p = colk[k];
        if (!(p > T(0))) { bad = true; p = T(1); }
        const T inv = T(1) / p;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int j = lane + 32 * c;
            if (j >= nb) break;
            const T rk = (j == k) ? inv : A[(size_t)k * nb + j] * inv;
            for (int i = 0; i < nb; ++i) {
                T* a = &A[(size_t)i * nb + j];
                if (i == k) *a = rk;
                else *a = ((j == k) ? T(0) : *a) - colk[i] * rk;
            }
        }
        __syncwarp();
    }
    }
    if (bad && lane == 0) atomicOr(flag + 1, 2);
    T* out = Sinv + cell * (long long)nb * nb;
    for (int o = lane; o < nb * nb; o += 32) out[o] = A[o];
}

// Blocks of 33 .. 64 rows: one cell per block of 64 threads, thread t keeping row t of the
// block in registers (64 columns, identity rows past nb).  In FP32 the same assembly and the
// same Gauss-Jordan updates as k_factor_warp<float, 2> (hence the same bits) with half the
// registers per thread, so more cells are resident per SM (FP32 only: in FP64 the
// shared-memory elimination of k_factor_warp<double, 0> is faster).  The pivot row moves through shared
// memory (double-buffered, one block barrier per step) and is read as 16-byte words.
template <typename T>
__global__ void __launch_bounds__(64)
    k_factor_rows(Geo<T> g, const T* __restrict__ gw, T alpha_inv, T beta, T* __restrict__ Sinv,
                  double* __restrict__ dump, int* __restrict__ flag, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    const int pb = (int)blockIdx.y;
    if (!bat_enter(bt, pb, &off)) return;
    gw = bsh(gw, off); Sinv = bsh(Sinv, off); dump = bsh(dump, off); flag = bsh(flag, off);
    if (bt.par) alpha_inv = (T)(1.0 / bt.par[pb * kBatPar + kParAlpha]);
    const int n = g.n, nloc = (int)g.nloc, nb = (int)g.nb, nc = g.ncomp;
    const int t = threadIdx.x;
    const long long cell = blockIdx.x;
    const size_t per = factor_warp_elems(n, g.d, nb, nc);
    T* A = reinterpret_cast<T*>(smraw);
    T* bufA = (nc > 1) ? A + (size_t)nb * nb : A;
    T* bufB = bufA + (nc > 1 ? (size_t)nloc * nloc : (size_t)nb * nb);
    T* Vq = bufB;
    {
        size_t nbuf_b = 1;
        for (int q = 0; q < 2 * g.d - 1; ++q) nbuf_b *= n;
        Vq = bufB + nbuf_b;
    }
    T* rbuf = A + (per - (nb > 128 ? nb : 128));
    for (int i = t; i < n * n; i += 64) Vq[i] = g.Vq[i];
    __syncthreads();
    const int gs = (g.kind == HPG_GRADIENT) ? g.d * (g.d + 1) / 2 : 1;
    if (nc == 1) {
        assemble_D_block<T, false>(g, gw, cell, 1, 0, Vq, A, bufB, t, 64);
        for (int o = t; o < nloc * nloc; o += 64) {
            const int I = o / nloc, J = o % nloc;
            T v = A[o] + g.C[o] * alpha_inv;
            if (I == J) v += beta * g.Mpsi[I];
            A[o] = v;
        }
    } else {
        int e = 0;
        for (int ca = 0; ca < nc; ++ca)
            for (int cb = ca; cb < nc; ++cb, ++e) {
                assemble_D_block<T, false>(g, gw, cell, gs, e, Vq, bufA, bufB, t, 64);
                for (int o = t; o < nloc * nloc; o += 64) {
                    const int I = o / nloc, J = o % nloc;
                    T v = bufA[o];
                    if (ca == cb) v += beta * g.Kpsi[o];
                    A[(size_t)(ca * nloc + I) * nb + cb * nloc + J] = v;
                    A[(size_t)(cb * nloc + J) * nb + ca * nloc + I] = v;
                }
                __syncthreads();
            }
    }
    __syncthreads();
    if (dump)
        for (int o = t; o < nb * nb; o += 64) dump[cell * nb * nb + o] = (double)A[o];
    constexpr int NM = 64;
    constexpr int VW = 16 / (int)sizeof(T);
    using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    T a[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) a[j] = (t < nb && j < nb) ? A[(size_t)t * nb + j] : T(t == j ? 1 : 0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
        if (k >= nb) break;
        T* rb = rbuf + (k & 1) * 64;
        if (t == k) {
#pragma unroll
            for (int q = 0; q < NM / VW; ++q) {
                V16 v;
                T* vt = reinterpret_cast<T*>(&v);
#pragma unroll
                for (int u = 0; u < VW; ++u) vt[u] = a[VW * q + u];
                reinterpret_cast<V16*>(rb)[q] = v;
            }
        }
        __syncthreads();
        T p = rb[k];
        if (!(p > T(0))) { bad = true; p = T(1); }
        const T inv = T(1) / p;
        const bool is_k = t == k;
        const T f = a[k];
        const T fp = is_k ? T(1) - inv : f * inv;
#pragma unroll
        for (int q = 0; q < NM / VW; ++q) {
            const V16 r = reinterpret_cast<const V16*>(rb)[q];
            const T* rr = reinterpret_cast<const T*>(&r);
#pragma unroll
            for (int u = 0; u < VW; ++u)
                if (VW * q + u != k) a[VW * q + u] -= fp * rr[u];
        }
        a[k] = is_k ? inv : -fp;
    }
    __syncthreads();
    if (t < nb)
#pragma unroll
        for (int j = 0; j < NM; ++j)
            if (j < nb) A[(size_t)t * nb + j] = a[j];
    __syncthreads();
    if (bad && t == 0) atomicOr(flag + 1, 2);
    T* out = Sinv + cell * (long long)nb * nb;
    for (int o = t; o < nb * nb; o += 64) out[o] = A[o];
}

// the factorisation workspace of a cell stays in shared memory up to this size
// (227 KB per block on this GPU, less the kernel's static shared memory)
constexpr size_t kFactorSmemMax = 225 * 1024;

static size_t factor_ws_elems(int n, int d, int nb, int nc) {
    size_t nloc = 1, nbuf_b = 1;
    for (int t = 0; t < d; ++t) nloc *= n;
    for (int t = 0; t < 2 * d - 1; ++t) nbuf_b *= n;
    return (size_t)nb * nb + (nc > 1 ? nloc * nloc : 0) + nbuf_b + (size_t)n * n + nb;
}

size_t factor_smem_bytes(int nb, int elem) { return (size_t)nb * nb * elem; }

size_t factor_workspace_elems(int n, int d, int nb, int nc, long long Nc, int elem) {
    const size_t elems = factor_ws_elems(n, d, nb, nc);
    return elems * elem <= kFactorSmemMax ? 0 : elems * (size_t)Nc;
}

template <typename T>
cudaError_t launch_factor(const Geo<T>& g, const T* gw, double alpha, double beta, T* Sinv, double* dump,
                          int* flag, T* gwork, cudaStream_t s, const Bat& bt) {
    const size_t elems = factor_ws_elems(g.n, g.d, (int)g.nb, g.ncomp);
    const size_t bytes = elems * sizeof(T);
    const int use_smem = bytes <= kFactorSmemMax;
    if (g.nb <= kFactorWarpMaxNb) {
        const size_t per = factor_warp_elems(g.n, g.d, (int)g.nb, g.ncomp) * sizeof(T);
        const int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, kFactorSmemMax / per));
        const unsigned blocks = (unsigned)((g.Nc + wpb - 1) / wpb);
        const dim3 grid(blocks, bt.np);
        const T ai = (T)(1.0 / alpha), be = (T)beta;
        // registers hold 32 R columns per row: R = 2 for FP32 up to 64, R = 1 up to 32
        bool done = false;
        if (g.nb <= 32) {
            k_factor_warp<T, 1><<<grid, 32 * wpb, per * wpb, s>>>(g, gw, ai, be, Sinv, dump, flag, wpb, bt);
            done = true;
        }
        // FP32: one cell per 64-thread block, a row per thread (k_factor_rows); in FP64 that form
        // measured slower than the shared-memory elimination (589 against 476 us on 1024 cells
        // of 49 rows)
        if constexpr (sizeof(T) == 4)
            if (!done && g.nb <= 64) {
                k_factor_rows<T><<<dim3((unsigned)g.Nc, bt.np), 64, per, s>>>(g, gw, ai, be, Sinv, dump, flag, bt);
                done = true;
            }
        if (!done) k_factor_warp<T, 0><<<grid, 32 * wpb, per * wpb, s>>>(g, gw, ai, be, Sinv, dump, flag, wpb, bt);
        note_launch();
        return cudaGetLastError();
    }
    if (!use_smem && !gwork) return cudaErrorInvalidValue;
    k_factor<T><<<dim3((unsigned)g.Nc, bt.np), 256, use_smem ? bytes : 0, s>>>(
        g, gw, (T)(1.0 / alpha), (T)beta, Sinv, dump, flag, gwork, use_smem, bt);
    note_launch();
    return cudaGetLastError();
}

// =================================================================== precond
// z = -(-S-hat_K)^{-1} v per cell.  The inverse is symmetric, so row i of the
// stored block is also its column i: a warp takes four rows at a time and reads
// them along k with coalesced loads (16 per lane in flight), then reduces each
// row over its lanes (fixed shuffle tree, deterministic).  `rsplit` blocks share
// a cell's rows when there are few cells.  The apply streams N_c nb^2 words and
// is bandwidth-bound.
template <typename T, typename Tin, typename Tout>
__global__ void __launch_bounds__(256)
    k_precond(Geo<T> g, const T* __restrict__ Sinv, const Tin* __restrict__ v, Tout* __restrict__ z, IterCtl ctl,
              int rsplit, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    ctl.skip = bsh(ctl.skip, off);
    ctl.jptr = bsh(ctl.jptr, off);
    if (ctl.skip && *ctl.skip) return;
    Sinv = bsh(Sinv, off); v = bsh(v, off); z = bsh(z, off);
    const int nb = (int)g.nb;
    T* vs = reinterpret_cast<T*>(smraw);      // nb
    const long long cell = blockIdx.x / rsplit;
    const int part = (int)(blockIdx.x - cell * rsplit);
    const Tin* vin = v + (ctl.jptr ? (long long)(*ctl.jptr) * ctl.jstride : 0LL);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) vs[i] = (T)vin[cell * nb + i];
    __syncthreads();
    const T* S = Sinv + cell * (long long)nb * nb;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rc = (nb + rsplit - 1) / rsplit;
    const int r0 = part * rc, r1 = (r0 + rc < nb) ? r0 + rc : nb;
    for (int i0 = r0 + 4 * wid; i0 < r1; i0 += 4 * nw) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        const bool full_rows = i0 + 3 < r1;
        for (int k0 = 0; k0 < nb; k0 += 128) {
            T a[4][4];
            if (full_rows && k0 + 128 <= nb) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 4; ++u) a[r][u] = S[(size_t)(i0 + r) * nb + k0 + lane + 32 * u];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[r] += a[r][u] * vs[k0 + lane + 32 * u];
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + lane + 32 * u;
                        a[r][u] = (i0 + r < r1 && k < nb) ? S[(size_t)(i0 + r) * nb + k] : T(0);
                    }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + lane + 32 * u;
                        if (k < nb) acc[r] += a[r][u] * vs[k];
                    }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            T t = acc[r];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0 && i0 + r < r1) z[cell * nb + i0 + r] = (Tout)(-t);
        }
    }
}

// FP64 variant: the FP64 pipe (1/64 of the FP32 rate) makes the padded lanes and
// the shuffle reductions of the row form cost more than they save, so each
// thread owns one row and walks k (exactly nb^2 FMAs per cell, no reduction).
template <typename Tin, typename Tout>
__global__ void k_precond_f64(Geo<double> g, const double* __restrict__ Sinv, const Tin* __restrict__ v,
                              Tout* __restrict__ z, IterCtl ctl, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    ctl.skip = bsh(ctl.skip, off);
    ctl.jptr = bsh(ctl.jptr, off);
    if (ctl.skip && *ctl.skip) return;
    Sinv = bsh(Sinv, off); v = bsh(v, off); z = bsh(z, off);
    double* vs = reinterpret_cast<double*>(smraw);
    const int nb = (int)g.nb;
    const long long cell = blockIdx.x;
    const Tin* vin = v + (ctl.jptr ? (long long)(*ctl.jptr) * ctl.jstride : 0LL);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) vs[i] = (double)vin[cell * nb + i];
    __syncthreads();
    const double* S = Sinv + cell * (long long)nb * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = 0;
        for (; k + 3 < nb; k += 4) {
            s0 += S[(size_t)k * nb + i] * vs[k];
            s1 += S[(size_t)(k + 1) * nb + i] * vs[k + 1];
            s2 += S[(size_t)(k + 2) * nb + i] * vs[k + 2];
            s3 += S[(size_t)(k + 3) * nb + i] * vs[k + 3];
        }
        for (; k < nb; ++k) s0 += S[(size_t)k * nb + i] * vs[k];
        z[cell * nb + i] = (Tout)(-((s0 + s1) + (s2 + s3)));
    }
}

// Small FP32 blocks (nb <= 128): the block is symmetric, so z_i = -sum_k S[k][i] v_k
// with one thread per i reads rows of S with consecutive threads on consecutive words
// (coalesced), four independent accumulators, and several cells share a 256-thread
// block (groups of nb rounded up to a warp) -- no lane padding to 128 columns and no
// shuffle reductions, which the row form spends on blocks of 49 or 64.
template <typename T, typename Tin, typename Tout>
__global__ void __launch_bounds__(256)
    k_precond_col(Geo<T> g, const T* __restrict__ Sinv, const Tin* __restrict__ v, Tout* __restrict__ z, IterCtl ctl,
                  int gsz, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    ctl.skip = bsh(ctl.skip, off);
    ctl.jptr = bsh(ctl.jptr, off);
    if (ctl.skip && *ctl.skip) return;
    Sinv = bsh(Sinv, off); v = bsh(v, off); z = bsh(z, off);
    const int nb = (int)g.nb;
    const int cpb = blockDim.x / gsz;
    const int grp = threadIdx.x / gsz, i = threadIdx.x - grp * gsz;
    const long long cell = (long long)blockIdx.x * cpb + grp;
    T* vs = reinterpret_cast<T*>(smraw) + (size_t)grp * gsz;
    const Tin* vin = v + (ctl.jptr ? (long long)(*ctl.jptr) * ctl.jstride : 0LL);
    const bool live = grp < cpb && cell < g.Nc;
    if (live && i < nb) vs[i] = (T)vin[cell * nb + i];
    __syncthreads();
    if (!live || i >= nb) return;
    const T* S = Sinv + cell * (long long)nb * nb;
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    int k = 0;
    for (; k + 3 < nb; k += 4) {
        s0 += S[(size_t)k * nb + i] * vs[k];
        s1 += S[(size_t)(k + 1) * nb + i] * vs[k + 1];
        s2 += S[(size_t)(k + 2) * nb + i] * vs[k + 2];
        s3 += S[(size_t)(k + 3) * nb + i] * vs[k + 3];
    }
    for (; k < nb; ++k) s0 += S[(size_t)k * nb + i] * vs[k];
    z[cell * nb + i] = (Tout)(-((s0 + s1) + (s2 + s3)));
}

// blocks per cell: enough blocks for two per SM when cells are few
static int precond_rsplit(long long Nc, long long nb) {
    int r = 1;
    while (r < 8 && Nc * r < 304 && nb / (r * 2) >= 32) r *= 2;
    return r;
}

template <typename T, typename Tin, typename Tout>
cudaError_t launch_precond(const Geo<T>& g, const T* Sinv, const Tin* v, Tout* z, cudaStream_t s, IterCtl ctl,
                           const Bat& bt) {
    if constexpr (sizeof(T) == 8) {
        const int threads = g.nb <= 64 ? 64 : (g.nb <= 128 ? 128 : 256);
        k_precond_f64<Tin, Tout><<<dim3((unsigned)g.Nc, bt.np), threads, g.nb * sizeof(double), s>>>(g, Sinv, v, z,
                                                                                                     ctl, bt);
        note_launch();
        return cudaGetLastError();
    }
    if (g.nb <= 128) {
        const int gsz = (int)((g.nb + 31) / 32) * 32, cpb = 256 / gsz;
        const dim3 grid((unsigned)((g.Nc + cpb - 1) / cpb), bt.np);
        k_precond_col<T, Tin, Tout><<<grid, 256, (size_t)cpb * gsz * sizeof(T), s>>>(g, Sinv, v, z, ctl, gsz, bt);
        note_launch();
        return cudaGetLastError();
    }
    // the row split serves one problem with few cells; a batch already fills the GPU
    const int rsplit = precond_rsplit(g.Nc * bt.np, g.nb);
    const size_t smem = (size_t)g.nb * sizeof(T);
    k_precond<T, Tin, Tout><<<dim3((unsigned)(g.Nc * rsplit), bt.np), 256, smem, s>>>(g, Sinv, v, z, ctl, rsplit, bt);
    note_launch();
    return cudaGetLastError();
}

// ==================================================================== B, B^T
template <typename T, typename Tin, typename Tout>
cudaError_t launch_bapply(const Geo<T>& g, const Tin* z, Tout* y, cudaStream_t s, const int* skip, const Bat& bt) {
    if (g.d == 2)
        k_urow<2, T, Tout, Tin, false, true, false><<<utile_grid<2>(g.n1, bt.np), 256, urow_smem<2>(g, false, true),
                                                      s>>>(g, T(0), (const Tout*)nullptr, T(1), z, (const Tin*)nullptr,
                                                           nullptr, nullptr, nullptr, nullptr, y, skip, bt, 0);
    else
        k_urow<3, T, Tout, Tin, false, true, false><<<utile_grid<3>(g.n1, bt.np), 256, urow_smem<3>(g, false, true),
                                                      s>>>(g, T(0), (const Tout*)nullptr, T(1), z, (const Tin*)nullptr,
                                                           nullptr, nullptr, nullptr, nullptr, y, skip, bt, 0);
    note_launch();
    return cudaGetLastError();
}

template <int D, typename T, typename Tin, typename Tout>
__global__ void k_btapply(Geo<T> g, const Tin* __restrict__ x, Tout* __restrict__ y, Bat bt) {
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    x = bsh(x, off);
    y = bsh(y, off);
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.Npsi) return;
    const long long cell = j / g.nb;
    const int rem = (int)(j - cell * g.nb);
    const int comp = rem / (int)g.nloc;
    int km[kMaxDim], cm[kMaxDim];
    int kk = rem - comp * (int)g.nloc;
    for (int t = 0; t < D; ++t) { km[t] = kk % g.n; kk /= g.n; }
    cell_multi(g, cell, cm);
    y[j] = (Tout)apply_BT_entry<D, T, Tin>(g, cm, comp, km, x);
}

template <typename T, typename Tin, typename Tout>
cudaError_t launch_btapply(const Geo<T>& g, const Tin* x, Tout* y, cudaStream_t s, const Bat& bt) {
    const dim3 b((unsigned)((g.Npsi + 255) / 256), bt.np);
    if (g.d == 2) k_btapply<2, T, Tin, Tout><<<b, 256, 0, s>>>(g, x, y, bt);
    else k_btapply<3, T, Tin, Tout><<<b, 256, 0, s>>>(g, x, y, bt);
    note_launch();
    return cudaGetLastError();
}

// ======================================================================= FDM
// One pass of the fast diagonalisation is a batched small GEMM
//   C[b](M x N) = A[b](M x K) * B[b](K x N)
// with general strides.  K = n1 <= ~400, so each CTA stages the whole K extent
// of its A row-panel and B column-panel in shared memory at once (all global
// loads in flight together, one barrier) and then runs the K loop from shared
// memory with a 4x2 register tile per thread.  The last forward pass applies
// the diagonal scaling 1 / (alpha (lam_0 + lam_1 (+ lam_2))) in its epilogue.
struct GemmArgs {
    int M, N, K, batch;
    long long sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb;
    int dA, dB;   // 1: the operand is per-problem data (moved by the batch offset); 0: a shared constant
};

// GEMM launches stack the problems of a batch in blockIdx.z above the GEMM batch
// index: z = problem * a.batch + b.  Moves the per-problem operands, the output,
// the device alpha and the skip flag to the block's problem.
#define GEMM_BATCH_ENTER()                                   \
    const int prob_ = (int)blockIdx.z / a.batch;             \
    long long boff_;                                         \
    if (!bat_enter(bt, prob_, &boff_)) return;               \
    skip = bsh(skip, boff_);                                 \
    if (skip && *skip) return;                               \
    if (a.dA) Ap = bsh(Ap, boff_);                           \
    if (a.dB) Bp = bsh(Bp, boff_);                           \
    Cp = bsh(Cp, boff_);                                     \
    sc.alpha_dev = bsh(sc.alpha_dev, boff_);

struct FdmScale {
    int on;
    int d;
    int n1[kMaxDim];
    const double* alpha_dev;   // alpha on the device (graph-friendly); null: use alpha_host
    double alpha_host;
    double shift;              // added to the eigenvalue sums: (A + shift M)^{-1} (0 for A_alpha^{-1})
};

// Asynchronous 4/8-byte global->shared copy (LDGSTS); `valid` false zero-fills.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem, bool valid) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    const int src = valid ? (int)sizeof(T) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gmem), "r"(src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(gmem), "r"(src));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// CTA tile BM x BN, TM x TN outputs per thread, KS warp groups splitting K.
// Panels are staged in shared memory as [k][m] and [k][n] (the inner index
// contiguous), walked so that consecutive threads write consecutive shared
// words (no bank conflicts); when the global operand is transposed the L1 line
// is reused across k.  Each of the KS groups runs a contiguous K range; the
// partial tiles are summed in group order (deterministic) before the epilogue.
template <typename T, int BM, int BN, int TM, int TN, int KS>
__global__ void __launch_bounds__((BM / TM) * (BN / TN) * KS)
    k_gemm_fullk(GemmArgs a, const T* __restrict__ Ap, const T* __restrict__ Bp, T* __restrict__ Cp,
                 FdmScale sc, const T* __restrict__ l0, const T* __restrict__ l1, const T* __restrict__ l2,
                 const int* skip, Bat bt) {
    constexpr int NG = (BM / TM) * (BN / TN);     // threads per group
    constexpr int NT = NG * KS;
    extern __shared__ __align__(16) unsigned char smraw[];
    GEMM_BATCH_ENTER()
    T* As = reinterpret_cast<T*>(smraw);          // [K][BM]
    T* Bs = As + (size_t)a.K * BM;                // [K][BN]
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int b = (int)blockIdx.z - prob_ * a.batch;
    const T* A = Ap + (long long)b * a.sAb;
    const T* B = Bp + (long long)b * a.sBb;
    T* C = Cp + (long long)b * a.sCb;
    const int K = a.K;
    for (int e = tid; e < BM * K; e += NT) {
        const int mm = e % BM, kk = e / BM, gm = m0 + mm;
        const bool ok = gm < a.M;
        cp_async_elem(&As[e], ok ? A + (long long)gm * a.sAm + (long long)kk * a.sAk : A, ok);
    }
    for (int e = tid; e < BN * K; e += NT) {
        const int nn = e % BN, kk = e / BN, gn = n0 + nn;
        const bool ok = gn < a.N;
        cp_async_elem(&Bs[e], ok ? B + (long long)kk * a.sBk + (long long)gn * a.sBn : B, ok);
    }
    cp_async_wait_all();
    __syncthreads();
    const int grp = tid / NG, gt = tid % NG;
    const int tx = gt % (BN / TN), ty = gt / (BN / TN);
    const int kchunk = (K + KS - 1) / KS;
    const int kb = grp * kchunk, ke = (kb + kchunk < K) ? kb + kchunk : K;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[i][jj] = T(0);
    const T* ap = As + ty * TM;
    const T* bp = Bs + tx * TN;
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        T av[TM], bv[TN];
        // vector shared loads (the panel rows are 16-byte aligned)
        if (sizeof(T) == 4 && TM % 4 == 0 && TN % 4 == 0) {
#pragma unroll
            for (int q = 0; q < TM / 4; ++q) {
                const float4 va = *reinterpret_cast<const float4*>(ap + (size_t)k * BM + 4 * q);
                av[4 * q] = (T)va.x; av[4 * q + 1] = (T)va.y; av[4 * q + 2] = (T)va.z; av[4 * q + 3] = (T)va.w;
            }
#pragma unroll
            for (int q = 0; q < TN / 4; ++q) {
                const float4 vb = *reinterpret_cast<const float4*>(bp + (size_t)k * BN + 4 * q);
                bv[4 * q] = (T)vb.x; bv[4 * q + 1] = (T)vb.y; bv[4 * q + 2] = (T)vb.z; bv[4 * q + 3] = (T)vb.w;
            }
        } else if (sizeof(T) == 4 && TM == 4 && TN == 2) {
            const float4 va = *reinterpret_cast<const float4*>(ap + (size_t)k * BM);
            const float2 vb = *reinterpret_cast<const float2*>(bp + (size_t)k * BN);
            av[0] = (T)va.x; av[1] = (T)va.y; av[2] = (T)va.z; av[3] = (T)va.w;
            bv[0] = (T)vb.x; bv[1] = (T)vb.y;
        } else if (sizeof(T) == 8 && TM == 2 && TN == 2) {
            const double2 va = *reinterpret_cast<const double2*>(ap + (size_t)k * BM);
            const double2 vb = *reinterpret_cast<const double2*>(bp + (size_t)k * BN);
            av[0] = (T)va.x; av[1] = (T)va.y;
            bv[0] = (T)vb.x; bv[1] = (T)vb.y;
        } else {
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = ap[(size_t)k * BM + i];
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) bv[jj] = bp[(size_t)k * BN + jj];
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) acc[i][jj] += av[i] * bv[jj];
    }
    if (KS > 1) {
        // deterministic reduction of the group partials through shared memory
        __syncthreads();
        T* red = As;                               // (KS-1) x NG x TM*TN, reuses the panels
        if (grp > 0)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) red[((size_t)(grp - 1) * NG + gt) * (TM * TN) + i * TN + jj] = acc[i][jj];
        __syncthreads();
        if (grp > 0) return;
        for (int g2 = 1; g2 < KS; ++g2)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[i][jj] += red[((size_t)(g2 - 1) * NG + gt) * (TM * TN) + i * TN + jj];
    }
    T ainv = T(1);
    if (sc.on) ainv = (T)(1.0 / (sc.alpha_dev ? *sc.alpha_dev : sc.alpha_host));
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int gm = m0 + ty * TM + i, gn = n0 + tx * TN + jj;
            if (gm < a.M && gn < a.N) {
                const long long off = (long long)gm * a.sCm + (long long)gn * a.sCn;
                T v = acc[i][jj];
                if (sc.on) {
                    // interior-tensor position of this output -> eigenvalue indices
                    long long lin = off + (long long)b * a.sCb;
                    const int i0 = (int)(lin % sc.n1[0]);
                    lin /= sc.n1[0];
                    const int i1 = (int)(lin % sc.n1[1]);
                    T lsum = l0[i0] + l1[i1];
                    if (sc.d == 3) lsum += l2[(int)(lin / sc.n1[1])];
                    lsum += (decltype(lsum))sc.shift;
                    v = v * ainv / lsum;
                }
                C[off] = v;
            }
        }
}

// fallback for K beyond the shared-memory budget: classic K-tiled GEMM
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm_tiled(GemmArgs a, const T* __restrict__ Ap, const T* __restrict__ Bp, T* __restrict__ Cp,
                 FdmScale sc, const T* __restrict__ l0, const T* __restrict__ l1, const T* __restrict__ l2,
                 const int* skip, Bat bt) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    GEMM_BATCH_ENTER()
    constexpr int NT = (BM / TM) * (BN / TN);
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int b = (int)blockIdx.z - prob_ * a.batch;
    const T* A = Ap + (long long)b * a.sAb;
    const T* B = Bp + (long long)b * a.sBb;
    T* C = Cp + (long long)b * a.sCb;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    const bool a_kfast = (a.sAk == 1);
    const bool b_nfast = (a.sBn == 1);
    for (int k0 = 0; k0 < a.K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NT) {
            int mm, kk;
            if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < a.M && gk < a.K) ? A[(long long)gm * a.sAm + (long long)gk * a.sAk] : T(0);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            int nn, kk;
            if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < a.N && gk < a.K) ? B[(long long)gk * a.sBk + (long long)gn * a.sBn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
    T ainv = T(1);
    if (sc.on) ainv = (T)(1.0 / (sc.alpha_dev ? *sc.alpha_dev : sc.alpha_host));
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gm = m0 + ty * TM + i, gn = n0 + tx * TN + j;
            if (gm < a.M && gn < a.N) {
                const long long off = (long long)gm * a.sCm + (long long)gn * a.sCn;
                T v = acc[i][j];
                if (sc.on) {
                    long long lin = off + (long long)b * a.sCb;
                    const int i0 = (int)(lin % sc.n1[0]);
                    lin /= sc.n1[0];
                    const int i1 = (int)(lin % sc.n1[1]);
                    T lsum = l0[i0] + l1[i1];
                    if (sc.d == 3) lsum += l2[(int)(lin / sc.n1[1])];
                    lsum += (decltype(lsum))sc.shift;
                    v = v * ainv / lsum;
                }
                C[off] = v;
            }
        }
}

// ---- pipelined variant for batches --------------------------------------------
// The whole-K tiles above stage a CTA's entire K panels before computing and rely on
// several CTAs per SM to hide that.  For batched launches (many CTAs of identical
// shape) this variant streams K in chunks of 16 through a four-deep ring of shared
// buffers (cp.async groups: chunks c + 1 .. c + 3 load while chunk c computes) with a 4 x 4
// register tile per thread.  It keeps KS separate accumulators -- K split into the
// same KS contiguous ranges as the whole-K tile with that KS, each summed in k order,
// then added in range order -- so it gives the same bits as those tiles.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T, int BM, int BN, int TM, int TN, int KS>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm_pipe(GemmArgs a, const T* __restrict__ Ap, const T* __restrict__ Bp, T* __restrict__ Cp, FdmScale sc,
                const T* __restrict__ l0, const T* __restrict__ l1, const T* __restrict__ l2, const int* skip,
                Bat bt) {
    constexpr int BK = 16, NT = (BM / TM) * (BN / TN), NS = 4;   // NS chunks in flight
    __shared__ __align__(16) T As[NS][BK][BM];
    __shared__ __align__(16) T Bs[NS][BK][BN];
    GEMM_BATCH_ENTER()
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int b = (int)blockIdx.z - prob_ * a.batch;
    const T* A = Ap + (long long)b * a.sAb;
    const T* B = Bp + (long long)b * a.sBb;
    T* C = Cp + (long long)b * a.sCb;
    const int K = a.K;
    const int kchunk = (K + KS - 1) / KS;
    // stage K indices [k0, min(k0 + BK, kend)) into buffer buf (zero outside)
    auto stage = [&](int buf, int k0, int kend) {
        for (int e = tid; e < BM * BK; e += NT) {
            const int mm = e % BM, kk = e / BM, gm = m0 + mm, k = k0 + kk;
            const bool ok = gm < a.M && k < kend;
            cp_async_elem(&As[buf][kk][mm], ok ? A + (long long)gm * a.sAm + (long long)k * a.sAk : A, ok);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            const int nn = e % BN, kk = e / BN, gn = n0 + nn, k = k0 + kk;
            const bool ok = gn < a.N && k < kend;
            cp_async_elem(&Bs[buf][kk][nn], ok ? B + (long long)k * a.sBk + (long long)gn * a.sBn : B, ok);
        }
    };
    // the t-th chunk in summation order: ranges in order, chunks of BK inside each
    auto chunk_of = [&](int t, int& k0, int& kend) -> bool {
        for (int g = 0; g < KS; ++g) {
            const int gb = g * kchunk, ge = min(K, gb + kchunk);
            if (gb >= ge) continue;
            const int nc = (ge - gb + BK - 1) / BK;
            if (t < nc) { k0 = gb + t * BK; kend = ge; return true; }
            t -= nc;
        }
        return false;
    };
    T acc[KS][TM][TN];
#pragma unroll
    for (int g = 0; g < KS; ++g)
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) acc[g][i][jj] = T(0);
#pragma unroll
    for (int st = 0; st < NS - 1; ++st) {
        int k0, ke;
        if (chunk_of(st, k0, ke)) stage(st, k0, ke);
        cp_async_commit();                            // (an empty group when there is no chunk)
    }
    int t = 0;
#pragma unroll
    for (int g = 0; g < KS; ++g) {
        const int gb = g * kchunk, ge = min(K, gb + kchunk);
        for (int k0 = gb; k0 < ge; k0 += BK) {
            {
                int nk0, nke;
                if (chunk_of(t + NS - 1, nk0, nke)) stage((t + NS - 1) % NS, nk0, nke);
                cp_async_commit();
            }
            cp_async_wait_group<NS - 1>();           // chunk t has landed
            __syncthreads();
            const int buf = t % NS, kn = min(BK, ge - k0);
            for (int kk = 0; kk < kn; ++kk) {
                T av[TM], bv[TN];
                if constexpr (sizeof(T) == 4 && TM == 4 && TN == 4) {
                    const float4 va = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM]);
                    const float4 vb = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * TN]);
                    av[0] = va.x; av[1] = va.y; av[2] = va.z; av[3] = va.w;
                    bv[0] = vb.x; bv[1] = vb.y; bv[2] = vb.z; bv[3] = vb.w;
                } else {
#pragma unroll
                    for (int i = 0; i < TM; ++i) av[i] = As[buf][kk][ty * TM + i];
#pragma unroll
                    for (int jj = 0; jj < TN; ++jj) bv[jj] = Bs[buf][kk][tx * TN + jj];
                }
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int jj = 0; jj < TN; ++jj) acc[g][i][jj] += av[i] * bv[jj];
            }
            __syncthreads();
            ++t;
        }
    }
    cp_async_wait_group<0>();
#pragma unroll
    for (int g = 1; g < KS; ++g)
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) acc[0][i][jj] += acc[g][i][jj];
    T ainv = T(1);
    if (sc.on) ainv = (T)(1.0 / (sc.alpha_dev ? *sc.alpha_dev : sc.alpha_host));
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int gm = m0 + ty * TM + i, gn = n0 + tx * TN + jj;
            if (gm < a.M && gn < a.N) {
                const long long off = (long long)gm * a.sCm + (long long)gn * a.sCn;
                T v = acc[0][i][jj];
                if (sc.on) {
                    long long lin = off + (long long)b * a.sCb;
                    const int i0 = (int)(lin % sc.n1[0]);
                    lin /= sc.n1[0];
                    const int i1 = (int)(lin % sc.n1[1]);
                    T lsum = l0[i0] + l1[i1];
                    if (sc.d == 3) lsum += l2[(int)(lin / sc.n1[1])];
                    lsum += (decltype(lsum))sc.shift;
                    v = v * ainv / lsum;
                }
                C[off] = v;
            }
        }
}

// ---- split-K pipelined variant with 8 x 8 register tiles -------------------------
// For batches.  The 4 x 4 tiles of k_gemm_pipe load 2 floats from shared memory per
// multiply-add and are bound by shared-memory bandwidth; here each thread holds 8 x 8
// outputs (1 float per 4 multiply-adds).  To keep enough threads per tile, the KS warp
// groups of a CTA take the KS K ranges in parallel -- each streams its range in chunks of
// 16 through its own three-deep ring of shared buffers, synchronising on its own named
// barrier -- and the group partials are added in range order at the end, the summation
// of the whole-K tiles with the same KS (the same bits).
template <typename T, int BM, int BN, int TM, int TN, int KS>
__global__ void __launch_bounds__((BM / TM) * (BN / TN) * KS, 2)
    k_gemm_pipe2(GemmArgs a, const T* __restrict__ Ap, const T* __restrict__ Bp, T* __restrict__ Cp, FdmScale sc,
                 const T* __restrict__ l0, const T* __restrict__ l1, const T* __restrict__ l2, const int* skip,
                 Bat bt) {
    constexpr int BK = 16, NS = 3, NG = (BM / TM) * (BN / TN);
    // panel rows padded by 4 floats: the k-contiguous staging writes 16 k's of one row,
    // which would otherwise all fall in one bank
    constexpr int BMP = BM + 4, BNP = BN + 4;
    constexpr int STAGE = BK * (BMP + BNP);
    static_assert(NG % BM == 0 && NG % BN == 0 && NG % BK == 0, "staging map");
    constexpr int EA = BM * BK / NG, EB = BN * BK / NG;
    extern __shared__ __align__(16) unsigned char smraw[];
    GEMM_BATCH_ENTER()
    const int tid = threadIdx.x, grp = tid / NG, gt = tid - grp * NG;
    const int tx = gt % (BN / TN), ty = gt / (BN / TN);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int b = (int)blockIdx.z - prob_ * a.batch;
    const T* A = Ap + (long long)b * a.sAb;
    const T* B = Bp + (long long)b * a.sBb;
    T* C = Cp + (long long)b * a.sCb;
    const int K = a.K;
    const int kchunk = (K + KS - 1) / KS;
    T* ring = reinterpret_cast<T*>(smraw) + (size_t)grp * NS * STAGE;
    const int kb = grp * kchunk, ke = min(K, kb + kchunk);
    const int nch = kb < ke ? (ke - kb + BK - 1) / BK : 0;
    // staging map of each operand, fixed per thread: consecutive threads take consecutive
    // global words (along k when the operand is k-contiguous, else along m / n)
    const bool ak = a.sAk == 1, bk = a.sBk == 1;
    const int a_mm = ak ? gt / BK : gt % BM, a_kk = ak ? gt % BK : gt / BM;
    const int a_dm = ak ? NG / BK : 0, a_dk = ak ? 0 : NG / BM;
    const int b_nn = bk ? gt / BK : gt % BN, b_kk = bk ? gt % BK : gt / BN;
    const int b_dn = bk ? NG / BK : 0, b_dk = bk ? 0 : NG / BN;
    auto stage = [&](int buf, int k0) {
        T* As = ring + (size_t)buf * STAGE;
        T* Bs = As + BK * BMP;
#pragma unroll
        for (int q = 0; q < EA; ++q) {
            const int mm = a_mm + q * a_dm, kk = a_kk + q * a_dk, gm = m0 + mm, k = k0 + kk;
            const bool ok = gm < a.M && k < ke;
            cp_async_elem(&As[kk * BMP + mm], ok ? A + (long long)gm * a.sAm + (long long)k * a.sAk : A, ok);
        }
#pragma unroll
        for (int q = 0; q < EB; ++q) {
            const int nn = b_nn + q * b_dn, kk = b_kk + q * b_dk, gn = n0 + nn, k = k0 + kk;
            const bool ok = gn < a.N && k < ke;
            cp_async_elem(&Bs[kk * BNP + nn], ok ? B + (long long)k * a.sBk + (long long)gn * a.sBn : B, ok);
        }
    };
    auto group_sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(NG) : "memory"); };
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[i][jj] = T(0);
#pragma unroll
    for (int st = 0; st < NS - 1; ++st) {
        if (st < nch) stage(st, kb + st * BK);
        cp_async_commit();
    }
    for (int c = 0; c < nch; ++c) {
        if (c + NS - 1 < nch) stage((c + NS - 1) % NS, kb + (c + NS - 1) * BK);
        cp_async_commit();
        cp_async_wait_group<NS - 1>();
        group_sync();
        const T* As = ring + (size_t)(c % NS) * STAGE;
        const T* Bs = As + BK * BMP;
        const int kn = min(BK, ke - (kb + c * BK));
        auto step = [&](int kk) {
            T av[TM], bv[TN];
            if constexpr (sizeof(T) == 4 && TM % 4 == 0 && TN % 4 == 0) {
#pragma unroll
                for (int q = 0; q < TM / 4; ++q) {
                    const float4 v4 = *reinterpret_cast<const float4*>(&As[kk * BMP + ty * TM + 4 * q]);
                    av[4 * q] = v4.x; av[4 * q + 1] = v4.y; av[4 * q + 2] = v4.z; av[4 * q + 3] = v4.w;
                }
#pragma unroll
                for (int q = 0; q < TN / 4; ++q) {
                    const float4 v4 = *reinterpret_cast<const float4*>(&Bs[kk * BNP + tx * TN + 4 * q]);
                    bv[4 * q] = v4.x; bv[4 * q + 1] = v4.y; bv[4 * q + 2] = v4.z; bv[4 * q + 3] = v4.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i) av[i] = As[kk * BMP + ty * TM + i];
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) bv[jj] = Bs[kk * BNP + tx * TN + jj];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[i][jj] += av[i] * bv[jj];
        };
        if (kn == BK) {
#pragma unroll 4
            for (int kk = 0; kk < BK; ++kk) step(kk);
        } else {
            for (int kk = 0; kk < kn; ++kk) step(kk);
        }
        group_sync();
    }
    cp_async_wait_group<0>();
    if (KS > 1) {
        // group partials through shared memory, added in range order (deterministic)
        __syncthreads();
        T* red = reinterpret_cast<T*>(smraw);
        if (grp > 0)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) red[((size_t)(grp - 1) * NG + gt) * (TM * TN) + i * TN + jj] = acc[i][jj];
        __syncthreads();
        if (grp > 0) return;
        for (int g2 = 1; g2 < KS; ++g2)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[i][jj] += red[((size_t)(g2 - 1) * NG + gt) * (TM * TN) + i * TN + jj];
    }
    T ainv = T(1);
    if (sc.on) ainv = (T)(1.0 / (sc.alpha_dev ? *sc.alpha_dev : sc.alpha_host));
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int gm = m0 + ty * TM + i, gn = n0 + tx * TN + jj;
            if (gm < a.M && gn < a.N) {
                const long long off = (long long)gm * a.sCm + (long long)gn * a.sCn;
                T v = acc[i][jj];
                if (sc.on) {
                    long long lin = off + (long long)b * a.sCb;
                    const int i0 = (int)(lin % sc.n1[0]);
                    lin /= sc.n1[0];
                    const int i1 = (int)(lin % sc.n1[1]);
                    T lsum = l0[i0] + l1[i1];
                    if (sc.d == 3) lsum += l2[(int)(lin / sc.n1[1])];
                    lsum += (decltype(lsum))sc.shift;
                    v = v * ainv / lsum;
                }
                C[off] = v;
            }
        }
}

template <typename T, int BM, int BN, int TM, int TN, int KS>
constexpr size_t pipe2_smem() {
    constexpr size_t ring = (size_t)KS * 3 * 16 * (BM + 4 + BN + 4) * sizeof(T);
    constexpr size_t red = (size_t)(KS - 1) * (BM / TM) * (BN / TN) * TM * TN * sizeof(T);
    return ring > red ? ring : red;
}

// ---- tensor-core variant of the FP32 pass (tcgen05, 3xTF32) ------------------
// C = A B on the 5th-generation tensor cores.  Each operand is split as x = hi + lo
// with hi = x rounded to TF32 (10-bit mantissa) and lo = x - hi (exact in FP32);
// C accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor memory (lo*lo is below
// FP32 rounding), which keeps the FP32-level accuracy of the SIMT passes.  One CTA
// of 4 warps computes a 128 x BN tile:
//  1. the whole K extent of its A row-panel and B column-panel is staged raw in
//     shared memory with 4-byte cp.async ([k][m] and [k][n]);
//  2. per chunk of 32 along K, all threads split the panels into hi/lo tiles in
//     the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
//     matrix; 128 bytes between core matrices along K, BK/4 x 128 bytes between
//     8-row groups), fence them to the tensor-core (async) proxy, and thread 0
//     issues 3 x 4 tcgen05.mma (M = 128, N = BN, K = 8) and commits them to the
//     buffer's mbarrier; with two buffers a chunk's split overlaps the previous
//     chunk's MMAs;
//  3. each warp reads its 32 TMEM lanes (tile rows) with tcgen05.ld and stores
//     them, with the FDM eigenvalue scaling on the last forward pass.
// Every mbarrier wait is bounded (about 0.1 s of spinning); on time-out the tile is
// written as NaN, which the solver's finiteness checks report, after a second
// bounded wait for the MMAs in flight, and TMEM is released in every case.
constexpr int kTcBM = 128, kTcBK = 32;
constexpr size_t kTcSmemMax = 225 * 1024;   // dynamic; the static mbarriers fit in the rest of 227 KB

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05 format): start, leading (K) and stride
// (8-row group) byte offsets, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// bounded spin with the non-blocking test (a suspended try_wait wakes up late)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    lo = x - hi;
}

template <int BN>
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, uint32_t* v);
template <>
__device__ __forceinline__ void tmem_ld_row<16>(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld_row<32>(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

// Raw panel layout in shared memory: when the operand is contiguous along k in
// global memory the panel is kept as [row][Kp + 4] (coalesced loads), otherwise as
// [k][rows + 8]; the pads make the core-matrix split below bank-conflict-free.
struct TcPanel {
    int kfast;    // 1: [row][ld], 0: [k][ld]
    int ld;       // leading dimension (floats)
};

__host__ __device__ inline TcPanel tc_panel(bool kfast, int rows, int Kp) {
    return kfast ? TcPanel{1, Kp + 4} : TcPanel{0, rows + 8};
}

__host__ __device__ inline size_t tc_panel_floats(const TcPanel& t, int rows, int Kp) {
    return (size_t)(t.kfast ? rows : Kp) * t.ld;
}

// dynamic shared memory of k_gemm_tc: nbuf hi/lo stages + raw K-panels (+ the output
// tile, which reuses the raw region)
template <int BN>
static size_t tc_smem_bytes(const GemmArgs& a, int nbuf) {
    const int Kp = ((a.K + kTcBK - 1) / kTcBK) * kTcBK;
    const size_t stage = 2 * (size_t)kTcBM * kTcBK + 2 * (size_t)BN * kTcBK;
    const TcPanel pa = tc_panel(a.sAk == 1, kTcBM, Kp), pb = tc_panel(a.sBk == 1, BN, Kp);
    const size_t raw = tc_panel_floats(pa, kTcBM, Kp) + tc_panel_floats(pb, BN, Kp);
    const size_t out = (size_t)kTcBM * (BN + 1);
    return (nbuf * stage + (raw > out ? raw : out)) * sizeof(float);
}

// stage rows x Kp of an operand (element (r, k) at G[r * sr + k * sk], zero outside
// rows_valid x K) into the raw panel; consecutive threads take consecutive global
// addresses along the contiguous direction
__device__ __forceinline__ void tc_stage(float* P, const TcPanel& t, const float* G, long long sr, long long sk,
                                         int rows, int rows_valid, int K, int Kp, int tid, int nthr) {
    if (t.kfast) {
        for (int e = tid; e < rows * Kp; e += nthr) {
            const int r = e / Kp, k = e - r * Kp;
            const bool ok = r < rows_valid && k < K;
            cp_async_elem(&P[(size_t)r * t.ld + k], ok ? G + (long long)r * sr + (long long)k * sk : G, ok);
        }
    } else {
        for (int e = tid; e < rows * Kp; e += nthr) {
            const int k = e / rows, r = e - k * rows;
            const bool ok = r < rows_valid && k < K;
            cp_async_elem(&P[(size_t)k * t.ld + r], ok ? G + (long long)r * sr + (long long)k * sk : G, ok);
        }
    }
}

// split rows x 32 (k0 .. k0+31) of a raw panel into hi/lo core-matrix tiles: a warp
// writes one whole core matrix (8 rows x 4 k) per instruction
__device__ __forceinline__ void tc_split(const float* P, const TcPanel& t, int rows, int k0, float* Hi, float* Lo,
                                         int tid, int nthr) {
    for (int e = tid; e < rows * kTcBK; e += nthr) {
        const int cm = e >> 5, w = e & 31;
        const int g = cm / (kTcBK / 4), c = cm - g * (kTcBK / 4);
        const int r = 8 * g + (w >> 2), k = k0 + 4 * c + (w & 3);
        const float x = t.kfast ? P[(size_t)r * t.ld + k] : P[(size_t)k * t.ld + r];
        float h, l;
        tf32_split(x, h, l);
        Hi[e] = h;
        Lo[e] = l;
    }
}

template <int BN>
__global__ void __launch_bounds__(256, 1)
    k_gemm_tc(GemmArgs a, const float* __restrict__ Ap, const float* __restrict__ Bp, float* __restrict__ Cp,
              FdmScale sc, const float* __restrict__ l0, const float* __restrict__ l1, const float* __restrict__ l2,
              const int* skip, int nbuf, Bat bt) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    GEMM_BATCH_ENTER()
    constexpr int BM = kTcBM, BK = kTcBK, NT = 256;
    constexpr int ATILE = BM * BK, BTILE = BN * BK, STAGE = 2 * ATILE + 2 * BTILE;
    constexpr uint32_t SBO = (BK / 4) * 128;              // bytes between 8-row core-matrix groups
    const int K = a.K;
    const int nch = (K + BK - 1) / BK;
    const int Kp = nch * BK;
    const TcPanel pa = tc_panel(a.sAk == 1, BM, Kp), pb = tc_panel(a.sBk == 1, BN, Kp);
    float* stage = reinterpret_cast<float*>(smraw);       // nbuf x [A_hi, A_lo, B_hi, B_lo]
    float* As = stage + nbuf * STAGE;
    float* Bs = As + tc_panel_floats(pa, BM, Kp);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, b = (int)blockIdx.z - prob_ * a.batch;
    const float* A = Ap + (long long)b * a.sAb + (long long)m0 * a.sAm;
    const float* B = Bp + (long long)b * a.sBb + (long long)n0 * a.sBn;
    float* C = Cp + (long long)b * a.sCb;
    tc_stage(As, pa, A, a.sAm, a.sAk, BM, a.M - m0, K, Kp, tid, NT);
    tc_stage(Bs, pb, B, a.sBn, a.sBk, BN, a.N - n0, K, Kp, tid, NT);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_addr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cp_async_wait_all();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // kind::tf32 instruction descriptor: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9,
    // 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        const int buf = c % nbuf;
        float* Ah = stage + buf * STAGE;
        float* Al = Ah + ATILE;
        float* Bh = Al + ATILE;
        float* Bl = Bh + BTILE;
        if (c >= nbuf) ok = mbar_wait(smem_addr(&mbar[buf]), (uint32_t)(((c - nbuf) / nbuf) & 1)) && ok;
        tc_split(As, pa, BM, c * BK, Ah, Al, tid, NT);
        tc_split(Bs, pb, BN, c * BK, Bh, Bl, tid, NT);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_addr(Ah), al = smem_addr(Al), bh = smem_addr(Bh), bl = smem_addr(Bl);
            for (int st = 0; st < BK / 8; ++st) {
                const uint32_t off = (uint32_t)st * 256;  // two core matrices (8 along K) per MMA
                tc_mma_tf32(tmem, tc_desc(ah + off, 128, SBO), tc_desc(bh + off, 128, SBO), idesc,
                            (c > 0 || st > 0) ? 1u : 0u);
                tc_mma_tf32(tmem, tc_desc(ah + off, 128, SBO), tc_desc(bl + off, 128, SBO), idesc, 1u);
                tc_mma_tf32(tmem, tc_desc(al + off, 128, SBO), tc_desc(bh + off, 128, SBO), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&mbar[buf]))
                         : "memory");
        }
    }
    const uint32_t last_bar = smem_addr(&mbar[(nch - 1) % nbuf]);
    const uint32_t last_par = (uint32_t)(((nch - 1) / nbuf) & 1);
    ok = mbar_wait(last_bar, last_par) && ok;
    if (!ok) mbar_wait(last_bar, last_par);               // one more bounded wait for the MMAs in flight
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // TMEM -> shared output tile [BM][BN + 1] (reuses the raw panels) -> global.  After a
    // timed-out wait the accumulator is not read at all: the tile is written as NaN, which
    // the solver's finiteness checks report as a failed solve.
    float* Cs = As;
    if (warp < 4) {
        const int r = warp * 32 + lane;
        if (__all_sync(0xffffffffu, ok)) {        // warp-uniform: tcgen05.ld is a warp-wide instruction
            uint32_t v[BN];
            tmem_ld_row<BN>(tmem + ((uint32_t)(warp * 32) << 16), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < BN; ++j) Cs[r * (BN + 1) + j] = __uint_as_float(v[j]);
        } else {
#pragma unroll
            for (int j = 0; j < BN; ++j) Cs[r * (BN + 1) + j] = __int_as_float(0x7fc00000);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
    float ainv = 1.0f;
    if (sc.on) ainv = (float)(1.0 / (sc.alpha_dev ? *sc.alpha_dev : sc.alpha_host));
    const bool nfast = a.sCn == 1;
    for (int e = tid; e < BM * BN; e += NT) {
        const int r = nfast ? e / BN : e % BM, j = nfast ? e % BN : e / BM;
        const int gm = m0 + r, gn = n0 + j;
        if (gm < a.M && gn < a.N) {
            const long long off = (long long)gm * a.sCm + (long long)gn * a.sCn;
            float val = Cs[r * (BN + 1) + j];
            if (sc.on) {
                long long lin = off + (long long)b * a.sCb;
                const int i0 = (int)(lin % sc.n1[0]);
                lin /= sc.n1[0];
                const int i1 = (int)(lin % sc.n1[1]);
                float lsum = l0[i0] + l1[i1];
                if (sc.d == 3) lsum += l2[(int)(lin / sc.n1[1])];
                    lsum += (decltype(lsum))sc.shift;
                val = val * ainv / lsum;
            }
            C[off] = val;
        }
    }
}

template <int BN>
static cudaError_t launch_gemm_tc(const GemmArgs& a, const float* A, const float* B, float* Cp, const FdmScale& sc,
                                  const float* l0, const float* l1, const float* l2, cudaStream_t s, const int* skip,
                                  const Bat& bt) {
    int nbuf = 2;
    if (tc_smem_bytes<BN>(a, nbuf) > kTcSmemMax) nbuf = 1;
    const size_t smem = tc_smem_bytes<BN>(a, nbuf);
    if (smem > kTcSmemMax) return cudaErrorInvalidValue;       // K too long for whole-K staging
    dim3 grid((a.N + BN - 1) / BN, (a.M + kTcBM - 1) / kTcBM, a.batch * bt.np);
    k_gemm_tc<BN><<<grid, 256, smem, s>>>(a, A, B, Cp, sc, l0, l1, l2, skip, nbuf, bt);
    note_launch();
    return cudaGetLastError();
}

// Tile choice: FP32 uses 32x32 tiles (4x2 per thread) -- the pass is latency-
// bound at these sizes; FP64 runs at a small fraction of the FP32 rate, so it
// uses 16x16 tiles to spread the work over all SMs.
// Tile variants of the fast-diagonalisation GEMM pass; which one runs for a
// given (dim, n1, precision) is picked at set-up by timing them on the device
// (autotune_fdm).  FP32 passes are latency-bound (few, short K loops), FP64
// passes are FP64-ALU-bound (~1/64 of the FP32 rate), so the candidates differ.
template <typename T, int BM_, int BN_, int TM_, int TN_, int KS_>
struct Tile { static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, KS = KS_, PIPE = 0; };
// the pipelined K-chunked kernel (k_gemm_pipe) with the same parameters
template <typename T, int BM_, int BN_, int TM_, int TN_, int KS_>
struct PTile { static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, KS = KS_, PIPE = 1; };
// the split-K pipelined kernel (k_gemm_pipe2)
template <typename T, int BM_, int BN_, int TM_, int TN_, int KS_>
struct QTile { static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, KS = KS_, PIPE = 2; };

template <typename T, typename C>
static cudaError_t launch_tile(const GemmArgs& a, const T* A, const T* B, T* Cp, const FdmScale& sc, const T* l0,
                               const T* l1, const T* l2, cudaStream_t s, const int* skip, const Bat& bt) {
    constexpr int BM = C::BM, BN = C::BN, TM = C::TM, TN = C::TN, KS = C::KS;
    if constexpr (C::PIPE == 2) {
        dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, a.batch * bt.np);
        k_gemm_pipe2<T, BM, BN, TM, TN, KS><<<grid, (BM / TM) * (BN / TN) * KS, pipe2_smem<T, BM, BN, TM, TN, KS>(),
                                              s>>>(a, A, B, Cp, sc, l0, l1, l2, skip, bt);
        note_launch();
        return cudaGetLastError();
    } else if constexpr (C::PIPE == 1) {
        dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, a.batch * bt.np);
        k_gemm_pipe<T, BM, BN, TM, TN, KS><<<grid, (BM / TM) * (BN / TN), 0, s>>>(a, A, B, Cp, sc, l0, l1, l2, skip,
                                                                                bt);
        note_launch();
        return cudaGetLastError();
    }
    const size_t red = (size_t)(KS - 1) * (BM / TM) * (BN / TN) * TM * TN * sizeof(T);
    const size_t smem = std::max((size_t)a.K * (BM + BN) * sizeof(T), red);
    if (smem <= 200 * 1024) {
        dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, a.batch * bt.np);
        k_gemm_fullk<T, BM, BN, TM, TN, KS><<<grid, (BM / TM) * (BN / TN) * KS, smem, s>>>(a, A, B, Cp, sc, l0, l1,
                                                                                        l2, skip, bt);
    } else {
        dim3 grid((a.N + 31) / 32, (a.M + 31) / 32, a.batch * bt.np);
        k_gemm_tiled<T, 32, 32, 16, 2, 2><<<grid, 256, 0, s>>>(a, A, B, Cp, sc, l0, l1, l2, skip, bt);
    }
    note_launch();
    return cudaGetLastError();
}

// The last FP32 SIMT tiles (8 x 4 outputs per thread) serve batches: more multiply-adds
// per shared load, for launches that fill the GPU many times over.  Tiles with the same
// KS add the same products in the same order, so they give the same bits.
using F32Tiles = std::tuple<Tile<float, 32, 16, 4, 2, 4>, Tile<float, 32, 32, 4, 2, 2>, Tile<float, 32, 16, 4, 2, 2>,
                            Tile<float, 16, 16, 2, 2, 4>, Tile<float, 32, 32, 4, 2, 4>, Tile<float, 64, 32, 8, 4, 4>,
                            Tile<float, 64, 32, 8, 4, 2>, Tile<float, 64, 64, 8, 8, 4>, PTile<float, 64, 64, 4, 4, 4>,
                            PTile<float, 32, 64, 4, 4, 4>, PTile<float, 64, 64, 4, 4, 2>, PTile<float, 32, 64, 4, 4, 2>,
                            QTile<float, 64, 64, 8, 8, 4>, QTile<float, 64, 32, 8, 4, 4>, QTile<float, 64, 64, 8, 8, 2>>;
using F64Tiles = std::tuple<Tile<double, 16, 16, 2, 2, 1>, Tile<double, 16, 16, 2, 2, 2>,
                            Tile<double, 32, 16, 4, 2, 1>, Tile<double, 16, 8, 2, 2, 2>>;
template <typename T>
struct TileSet;
template <>
struct TileSet<float> { using type = F32Tiles; };
template <>
struct TileSet<double> { using type = F64Tiles; };

// FP32 variants: the SIMT tiles, then the tcgen05 3xTF32 kernel with BN = 16 and 32
constexpr int kTcVariants = 2;
// ... then the TMA-fed tcgen05 passes (fdm_tma.cu) with N tiles of 64, 128 and 256
int fdm_tile_count(int elem) {
    return elem == 4 ? (int)std::tuple_size<F32Tiles>::value + kTcVariants + fdm_tma_variants()
                     : (int)std::tuple_size<F64Tiles>::value;
}

template <typename Set, size_t I = 0>
static int tile_ks_of(int idx) {
    if constexpr (I < std::tuple_size<Set>::value) {
        if (idx == (int)I) return std::tuple_element<I, Set>::type::KS;
        return tile_ks_of<Set, I + 1>(idx);
    } else {
        return 0;
    }
}

// K split of a variant (its summation order); 0 for the tensor-core variants that split
// in shared memory, -1 - v for TMA variant v (each its own order: groups keep it)
int fdm_tile_ks(int elem, int idx) {
    if (elem == 4) {
        const int tv = idx - (int)std::tuple_size<F32Tiles>::value - kTcVariants;
        if (tv >= 0) return -1 - tv;
        return tile_ks_of<F32Tiles>(idx);
    }
    return tile_ks_of<F64Tiles>(idx);
}

template <typename T, size_t I = 0>
static cudaError_t launch_tile_idx(int idx, const GemmArgs& a, const T* A, const T* B, T* Cp, const FdmScale& sc,
                                   const T* l0, const T* l1, const T* l2, cudaStream_t s, const int* skip,
                                   const Bat& bt) {
    using Set = typename TileSet<T>::type;
    if constexpr (I < std::tuple_size<Set>::value) {
        if (idx == (int)I)
            return launch_tile<T, typename std::tuple_element<I, Set>::type>(a, A, B, Cp, sc, l0, l1, l2, s, skip, bt);
        return launch_tile_idx<T, I + 1>(idx, a, A, B, Cp, sc, l0, l1, l2, s, skip, bt);
    } else {
        if constexpr (sizeof(T) == 4) {
            const int t = idx - (int)std::tuple_size<Set>::value;
            if (t == 0) return launch_gemm_tc<16>(a, A, B, Cp, sc, l0, l1, l2, s, skip, bt);
            if (t == 1) return launch_gemm_tc<32>(a, A, B, Cp, sc, l0, l1, l2, s, skip, bt);
        }
        return cudaErrorInvalidValue;
    }
}

template <typename T, size_t I = 0>
static void configure_tiles() {
    using Set = typename TileSet<T>::type;
    if constexpr (I < std::tuple_size<Set>::value) {
        using C = typename std::tuple_element<I, Set>::type;
        if constexpr (C::PIPE == 0)
            cudaFuncSetAttribute(k_gemm_fullk<T, C::BM, C::BN, C::TM, C::TN, C::KS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if constexpr (C::PIPE == 2)
            cudaFuncSetAttribute(k_gemm_pipe2<T, C::BM, C::BN, C::TM, C::TN, C::KS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        configure_tiles<T, I + 1>();
    }
}

template <typename T>
static cudaError_t gemm(const GemmArgs& a, const T* A, const T* B, T* C, const FdmScale& sc, const Geo<T>& g,
                        cudaStream_t s, const int* skip, const Bat& bt) {
    const T* l0 = g.lam[0];
    const T* l1 = g.d > 1 ? g.lam[1] : g.lam[0];
    const T* l2 = g.d > 2 ? g.lam[2] : g.lam[0];
    return launch_tile_idx<T>(g.gemm_cfg, a, A, B, C, sc, l0, l1, l2, s, skip, bt);
}

// A_alpha^{-1} x = alpha^{-1} (V (x) V (x) V) diag(1 / sum lam) (V^T (x) V^T (x) V^T) x
template <typename T>
cudaError_t launch_fdm(const Geo<T>& g, const double* alpha_dev, double alpha, const T* x, T* y, T* work1, T* work2,
                       cudaStream_t s, const int* skip, const Bat& bt, double shift) {
    if constexpr (sizeof(T) == 4) {
        const int tv = g.gemm_cfg - (int)std::tuple_size<F32Tiles>::value - kTcVariants;
        if (tv >= 0) {
            if (!g.tma || !g.tma->ready) return cudaErrorInvalidValue;
            return launch_fdm_tma(*g.tma, tv, alpha_dev, alpha, x, y, s, skip, bt, shift);
        }
    }
    const int d = g.d;
    long long inner[kMaxDim], outer[kMaxDim];
    for (int ax = 0; ax < d; ++ax) {
        inner[ax] = 1;
        outer[ax] = 1;
        for (int j = 0; j < ax; ++j) inner[ax] *= g.n1[j];
        for (int j = ax + 1; j < d; ++j) outer[ax] *= g.n1[j];
    }
    FdmScale off{};
    FdmScale on{};
    on.on = 1;
    on.d = d;
    for (int j = 0; j < kMaxDim; ++j) on.n1[j] = g.n1[j];
    on.alpha_dev = alpha_dev;
    on.alpha_host = alpha;
    on.shift = shift;
    // pass along axis ax: out[o][a][i] = sum_k W(a,k) in[o][k][i]; W = V^T (fwd) or V (bwd)
    auto pass = [&](int ax, bool fwd, const T* in, T* out, const FdmScale& sc) -> cudaError_t {
        const int n1 = g.n1[ax];
        const T* V = g.V[ax];   // row-major V[k][a]
        GemmArgs a{};
        if (inner[ax] == 1) {
            a.M = (int)outer[ax]; a.N = n1; a.K = n1; a.batch = 1;
            a.sAm = n1; a.sAk = 1; a.sAb = 0;
            if (fwd) { a.sBk = n1; a.sBn = 1; } else { a.sBk = 1; a.sBn = n1; }
            a.sBb = 0;
            a.sCm = n1; a.sCn = 1; a.sCb = 0;
            a.dA = 1; a.dB = 0;
            return gemm<T>(a, in, V, out, sc, g, s, skip, bt);
        }
        a.M = n1; a.N = (int)inner[ax]; a.K = n1; a.batch = (int)outer[ax];
        // W = V^T (forward) read K-contiguous from the stored transpose when there is one
        const T* Wm = V;
        if (fwd && g.VT[ax]) { Wm = g.VT[ax]; a.sAm = n1; a.sAk = 1; }
        else if (fwd) { a.sAm = 1; a.sAk = n1; }
        else { a.sAm = n1; a.sAk = 1; }
        a.sAb = 0;
        a.sBk = inner[ax]; a.sBn = 1; a.sBb = (long long)n1 * inner[ax];
        a.sCm = inner[ax]; a.sCn = 1; a.sCb = (long long)n1 * inner[ax];
        a.dA = 0; a.dB = 1;
        return gemm<T>(a, Wm, in, out, sc, g, s, skip, bt);
    };
    cudaError_t e;
    const T* cur = x;
    T* bufs[2] = {work1, work2};
    int bi = 0;
    for (int ax = 0; ax < d; ++ax) {
        if ((e = pass(ax, true, cur, bufs[bi], ax == d - 1 ? on : off)) != cudaSuccess) return e;
        cur = bufs[bi];
        bi ^= 1;
    }
    for (int ax = 0; ax < d; ++ax) {
        T* dst = (ax == d - 1) ? y : bufs[bi];
        if ((e = pass(ax, false, cur, dst, off)) != cudaSuccess) return e;
        cur = dst;
        bi ^= 1;
    }
    return cudaGetLastError();
}

// ========================================================== D apply per cell
// out = sB * (B^T t) + sD * (D z + E z) for one cell, by a group of `nthr`
// threads (local id lt) with shared scratch `sm` of 3 nb + n^2 elements.  D z by
// sum factorisation: z -> Gauss values (V along each axis) -> times gw (or the
// 2x2/3x3 Jacobian) -> V^T back.  Every thread of the block must call this the
// same number of times (it contains block-wide barriers).
template <int D, typename T, typename Tz, typename Tt, typename Tout>
__device__ __forceinline__ void cellop_body(const Geo<T>& g, const T* __restrict__ gw, T beta, const Tz* __restrict__ z,
                                            const Tt* __restrict__ t, T sB, T sD, Tout* __restrict__ outp,
                                            long long cell, bool active, int lt, int nthr, T* sm) {
    const int n = g.n, nloc = (int)g.nloc, nc = g.ncomp, nb = (int)g.nb;
    T* a = sm;
    T* b = sm + nb;
    T* zc = sm + 2 * nb;
    T* Vq = sm + 3 * nb;
    for (int i = lt; i < n * n; i += nthr) Vq[i] = g.Vq[i];
    if (active)
        for (int i = lt; i < nb; i += nthr) { const T v = (T)z[cell * nb + i]; a[i] = v; zc[i] = v; }
    __syncthreads();
    T *in = a, *o = b;
    int stride = 1;
    for (int ax = 0; ax < D; ++ax) {
        if (active) sf_pass(in, o, Vq, false, n, nloc, nc, stride, lt, nthr);
        __syncthreads();
        T* tt = in; in = o; o = tt;
        stride *= n;
    }
    const int gs = (g.kind == HPG_GRADIENT) ? D * (D + 1) / 2 : 1;
    if (active)
        for (int q = lt; q < nloc; q += nthr) {
            const long long gq = cell * nloc + q;
            if (nc == 1) {
                o[q] = gw[gq] * in[q];
            } else {
                T zq[kMaxDim];
                for (int k = 0; k < nc; ++k) zq[k] = in[k * nloc + q];
                for (int k = 0; k < nc; ++k) {
                    T sacc = T(0);
                    for (int l = 0; l < nc; ++l) {
                        const int lo = k < l ? k : l, hi = k < l ? l : k;
                        const int e = lo * nc - lo * (lo - 1) / 2 + (hi - lo);
                        sacc += gw[gq * gs + e] * zq[l];
                    }
                    o[k * nloc + q] = sacc;
                }
            }
        }
    __syncthreads();
    { T* tt = in; in = o; o = tt; }
    stride = 1;
    for (int ax = 0; ax < D; ++ax) {
        if (active) sf_pass(in, o, Vq, true, n, nloc, nc, stride, lt, nthr);
        __syncthreads();
        T* tt = in; in = o; o = tt;
        stride *= n;
    }
    if (!active) return;
    int cm[kMaxDim];
    cell_multi(g, cell, cm);
    for (int i = lt; i < nb; i += nthr) {
        const int comp = i / nloc, li = i - comp * nloc;
        T ez;
        if (nc == 1) {
            ez = beta * g.Mpsi[li] * zc[i];
        } else {
            ez = T(0);
            for (int l = 0; l < nloc; ++l) ez += g.Kpsi[(size_t)li * nloc + l] * zc[comp * nloc + l];
            ez *= beta;
        }
        T acc = sD * (in[i] + ez);
        if (t) {
            int km[kMaxDim];
            int kk = li;
            for (int q = 0; q < D; ++q) { km[q] = kk % n; kk /= n; }
            acc += sB * apply_BT_entry<D, T, Tt>(g, cm, comp, km, t);
        }
        outp[cell * nb + i] = (Tout)acc;
    }
}

// Cells are processed by groups of gs threads, cpb cells per block (in the fused Newton
// apply gs = min(nb, 256) and cpb = 256 / gs, so that few lanes idle when nb is not a
// multiple of 32, 49 for n = 7); threads left over after cpb groups run on a scratch
// slot, inactive.
inline void cell_groups(long long nb, int* gs, int* cpb) {
    *gs = (int)(nb < 256 ? (nb > 0 ? nb : 1) : 256);
    *cpb = 256 / *gs;
}

template <int D, typename T, typename Tz, typename Tt, typename Tout>
__global__ void __launch_bounds__(256)
    k_cellop(Geo<T> g, const T* __restrict__ gw, T beta, const Tz* __restrict__ z, const Tt* __restrict__ t, T sB,
             T sD, Tout* __restrict__ out, IterCtl ctl, int gs, int cpb, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    ctl.skip = bsh(ctl.skip, off);
    ctl.jptr = bsh(ctl.jptr, off);
    if (ctl.skip && *ctl.skip) return;
    gw = bsh(gw, off); z = bsh(z, off); t = bsh(t, off); out = bsh(out, off);
    Tout* outp = out + (ctl.jptr ? (long long)(*ctl.jptr + 1) * ctl.jstride : 0LL);
    const int grp = threadIdx.x / gs, lt = threadIdx.x - grp * gs;
    const long long cell = (long long)blockIdx.x * cpb + grp;
    const size_t per = (size_t)(3 * g.nb + g.n * g.n);
    cellop_body<D, T, Tz, Tt, Tout>(g, gw, beta, z, t, sB, sD, outp, cell, grp < cpb && cell < g.Nc, lt, gs,
                                    reinterpret_cast<T*>(smraw) + (size_t)(grp < cpb ? grp : cpb) * per);
}

// One launch for G x: blocks [0, nu) are u-row tiles (alpha A x_u + B x_psi),
// the rest apply the psi rows B^T x_u - (D + E) x_psi to `cpb` cells each
// (groups of 256 / cpb threads), so both FP64 workloads share the SMs.
template <int D>
__global__ void __launch_bounds__(256)
    k_newton_fused(Geo<double> g, const double* __restrict__ gw, double alpha, double beta,
                   const double* __restrict__ x, double* __restrict__ y, int nu, int gs, int cpb, Bat bt) {
    extern __shared__ __align__(16) unsigned char smraw[];
    long long off;
    const int pbi = (int)blockIdx.y;
    if (!bat_enter(bt, pbi, &off)) return;
    gw = bsh(gw, off); x = bsh(x, off); y = bsh(y, off);
    if (bt.par) alpha = bt.par[pbi * kBatPar + kParAlpha];
    // u-row tiles and cell groups alternate in block order, so that the block
    // scheduler hands every SM a similar mix of the two kinds of work
    const int nc = (int)gridDim.x - nu;
    const int mn = nu < nc ? nu : nc;
    const int b = (int)blockIdx.x;
    const bool is_u = b < 2 * mn ? (b & 1) == 0 : nu > nc;
    const int idx = b < 2 * mn ? (b >> 1) : mn + (b - 2 * mn);
    if (is_u) {
        // u rows: reuse the tiled row kernel body through a grid-index remap
        k_urow_body<D, double, double, double, true, true, false>(
            g, alpha, x, 1.0, x + g.Nu0, nullptr, nullptr, nullptr, nullptr, nullptr, y, idx, smraw);
        return;
    }
    const int grp = threadIdx.x / gs, lt = threadIdx.x - grp * gs;
    const long long cell = (long long)idx * cpb + grp;
    const size_t per = (size_t)(3 * g.nb + g.n * g.n);
    cellop_body<D, double, double, double, double>(g, gw, beta, x + g.Nu0, x, 1.0, -1.0, y + g.Nu0, cell,
                                                   grp < cpb && cell < g.Nc, lt, gs,
                                                   reinterpret_cast<double*>(smraw) +
                                                       (size_t)(grp < cpb ? grp : cpb) * per);
}

template <typename T, typename Tout>
cudaError_t launch_schur_rest(const Geo<T>& g, const T* gw, double beta, const T* z, const T* t, Tout* w,
                              cudaStream_t s, IterCtl ctl, const Bat& bt) {
    // one cell per block for a single problem (measured faster than several cells per block
    // for the FP32 and FP64 Krylov-loop applies, which are latency-bound); a lockstep launch
    // over several problems packs floor(256 / nb) cells into 256-thread blocks, as the fused
    // Newton apply does.  Each cell's arithmetic is the same either way.
    int gs = g.nb <= 64 ? 64 : (g.nb <= 128 ? 128 : 256), cpb = 1, threads = gs;
    if (bt.np > 1 && g.nb <= 128) {
        gs = (int)g.nb;
        cpb = std::max(1, 256 / gs);
        threads = 256;
    }
    const size_t smem = (size_t)(cpb + 1) * (3 * g.nb + g.n * g.n) * sizeof(T);
    const dim3 blocks((unsigned)((g.Nc + cpb - 1) / cpb), bt.np);
    if (g.d == 2)
        k_cellop<2, T, T, T, Tout><<<blocks, threads, smem, s>>>(g, gw, (T)beta, z, t, T(-1), T(-1), w, ctl, gs, cpb,
                                                                bt);
    else
        k_cellop<3, T, T, T, Tout><<<blocks, threads, smem, s>>>(g, gw, (T)beta, z, t, T(-1), T(-1), w, ctl, gs, cpb,
                                                                bt);
    note_launch();
    return cudaGetLastError();
}

// G x (eq. pG-matrix) in one launch: u-row tiles and psi cells share the SMs.
cudaError_t launch_newton_apply(const Geo<double>& g, const double* gw, double alpha, double beta,
                                const double* x, double* y, cudaStream_t s, const Bat& bt) {
    // 2D: the u rows gather straight from global memory (measured on radial 32x32 p=8:
    // the staged boxes cut the blocks per SM of both halves more than they save,
    // 19.3 vs 15.8 us); 3D: staged (sine 3D: 76 vs 98 us)
    Geo<double> gu = g;
    if (g.d == 2) gu.staged = 0;
    const int nu = (int)utile_blocks(g.d, g.n1);
    int gs = 0, cpb = 0;
    cell_groups(g.nb, &gs, &cpb);
    const int nc = (int)((g.Nc + cpb - 1) / cpb);
    const size_t per = (size_t)(3 * g.nb + g.n * g.n) * sizeof(double);
    const size_t st = g.d == 2 ? urow_smem<2>(gu, true, true) : urow_smem<3>(gu, true, true);
    const size_t smem = std::max(st, (cpb + 1) * per);
    const dim3 grid(nu + nc, bt.np);
    if (g.d == 2) k_newton_fused<2><<<grid, 256, smem, s>>>(gu, gw, alpha, beta, x, y, nu, gs, cpb, bt);
    else k_newton_fused<3><<<grid, 256, smem, s>>>(gu, gw, alpha, beta, x, y, nu, gs, cpb, bt);
    note_launch();
    return cudaGetLastError();
}

// ==================================================================== vectors
// One-dimensional grids over n elements; blockIdx.y is the problem of a batch.
template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* __restrict__ x, Tout* __restrict__ y, long long n, Bat bt) {
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    x = bsh(x, off);
    y = bsh(y, off);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (Tout)x[i];
}
template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* x, Tout* y, long long n, cudaStream_t s, const Bat& bt) {
    k_convert<Tin, Tout><<<dim3((unsigned)((n + 255) / 256), bt.np), 256, 0, s>>>(x, y, n, bt);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long long n,
                        Bat bt) {
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    x = bsh(x, off);
    y = bsh(y, off);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}
cudaError_t launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s, const Bat& bt) {
    k_axpby<<<dim3((unsigned)((n + 255) / 256), bt.np), 256, 0, s>>>(a, x, b, y, n, bt);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
__global__ void k_sub_scaled(const double* __restrict__ x, double b, const T* __restrict__ z, double* __restrict__ y,
                             long long n, Bat bt) {
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    x = bsh(x, off);
    z = bsh(z, off);
    y = bsh(y, off);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] - b * (double)z[i];
}
template <typename T>
cudaError_t launch_sub_scaled(const double* x, double b, const T* z, double* y, long long n, cudaStream_t s,
                              const Bat& bt) {
    k_sub_scaled<T><<<dim3((unsigned)((n + 255) / 256), bt.np), 256, 0, s>>>(x, b, z, y, n, bt);
    note_launch();
    return cudaGetLastError();
}

// xt = x - lam dx; lam from Bat::par (kParLam) when given
__global__ void k_trial(const double* __restrict__ x, const double* __restrict__ dx, double lam,
                        double* __restrict__ xt, long long n, Bat bt) {
    long long off;
    const int pb = (int)blockIdx.y;
    if (!bat_enter(bt, pb, &off)) return;
    x = bsh(x, off);
    dx = bsh(dx, off);
    xt = bsh(xt, off);
    if (bt.par) lam = bt.par[pb * kBatPar + kParLam];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xt[i] = x[i] - lam * dx[i];
}
cudaError_t launch_trial(const double* x, const double* dx, double lam, double* xt, long long n, cudaStream_t s,
                         const Bat& bt) {
    k_trial<<<dim3((unsigned)((n + 255) / 256), bt.np), 256, 0, s>>>(x, dx, lam, xt, n, bt);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_sumsq(const double* __restrict__ x, long long n, double* __restrict__ part, Bat bt) {
    __shared__ double sh[32];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    x = bsh(x, off);
    part = bsh(part, off);
    double v = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v += x[i] * x[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}
cudaError_t launch_sumsq(const double* x, long long n, double* part, int* nparts, cudaStream_t s, const Bat& bt) {
    int b = (int)((n + 255) / 256);
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    k_sumsq<<<dim3(b, bt.np), 256, 0, s>>>(x, n, part, bt);
    note_launch();
    *nparts = b;
    return cudaGetLastError();
}

// y = x (n elements of T) and y = 0, per problem of a batch
template <typename T>
__global__ void k_copy(const T* __restrict__ x, T* __restrict__ y, long long n, Bat bt) {
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    x = bsh(x, off);
    y = bsh(y, off);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x ? x[i] : T(0);
}
template <typename T>
cudaError_t launch_copy(const T* x, T* y, long long n, cudaStream_t s, const Bat& bt) {
    long long b = (n + 255) / 256;
    if (b > 2048) b = 2048;
    if (b < 1) b = 1;
    k_copy<T><<<dim3((unsigned)b, bt.np), 256, 0, s>>>(x, y, n, bt);
    note_launch();
    return cudaGetLastError();
}

// *dst = par[pb][slot] for every problem of the batch (per-problem scalars into the problems' slabs)
__global__ void k_scatter_par(double* __restrict__ dst, int slot, Bat bt) {
    const int pb = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (pb >= bt.np) return;
    long long off;
    if (!bat_enter(bt, pb, &off)) return;
    *bsh(dst, off) = bt.par[pb * kBatPar + slot];
}
cudaError_t launch_scatter_par(double* dst, int slot, cudaStream_t s, const Bat& bt) {
    k_scatter_par<<<(bt.np + 63) / 64, 64, 0, s>>>(dst, slot, bt);
    note_launch();
    return cudaGetLastError();
}

// out[pb * nd + k] = d[k] of problem pb (k < nd), out[np * nd + pb * ni + k] = i[k]:
// the status words the host reads after a batched step, in one copy
__global__ void k_gather_status(const double* __restrict__ d, int nd, const int* __restrict__ iv, int ni,
                                double* __restrict__ out, Bat bt) {
    const int pb = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (pb >= bt.np) return;
    const long long off = bt.delta ? bt.delta[pb] : 0LL;
    const double* dp = bsh(d, off);
    const int* ip = bsh(iv, off);
    for (int k = 0; k < nd; ++k) out[pb * nd + k] = dp[k];
    for (int k = 0; k < ni; ++k) out[bt.np * nd + pb * ni + k] = (double)ip[k];
}
cudaError_t launch_gather_status(const double* d, int nd, const int* iv, int ni, double* out, cudaStream_t s,
                                 const Bat& bt) {
    k_gather_status<<<(bt.np + 63) / 64, 64, 0, s>>>(d, nd, iv, ni, out, bt);
    note_launch();
    return cudaGetLastError();
}

// ===================================================================== GMRES
// Right-preconditioned GMRES without restart; the iteration index j lives on
// the device (G.jdev) so that a chunk of iterations can be captured once in a
// CUDA graph and replayed.  Every kernel returns immediately once the
// converged/stop flag (G.iflag[0]) is set.  Classical Gram--Schmidt with one
// re-orthogonalisation (CGS2), fixed-order (deterministic) reductions.  The
// basis is stored in VT: double for the FP64 solves, float for the FP32 inner
// solves of the mixed path (their operator is FP32 as well; the FP64 refinement
// around them corrects what either loses).  Dot products, Hessenberg column,
// Givens rotations and residual estimate are FP64 for both.

template <typename VT>
__global__ void k_gm_start(VT* __restrict__ Vb, const double* __restrict__ b, long long N,
                           const double* __restrict__ part, int nparts, double rtol, double* __restrict__ scal,
                           double* __restrict__ gv, int kmax, int cap, int* __restrict__ iflag,
                           int* __restrict__ jdev, double* __restrict__ H, Bat bt) {
    __shared__ double sh[32];
    long long off;
    const int pb = (int)blockIdx.y;
    if (!bat_enter(bt, pb, &off)) return;
    Vb = bsh(Vb, off); b = bsh(b, off); part = bsh(part, off); scal = bsh(scal, off); gv = bsh(gv, off);
    iflag = bsh(iflag, off); jdev = bsh(jdev, off); H = bsh(H, off);
    if (bt.par) rtol = bt.par[pb * kBatPar + kParRtol];
    // the Hessenberg matrix starts at zero
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(kmax + 1) * kmax;
         i += (long long)gridDim.x * blockDim.x)
        H[i] = 0.0;
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[i];
    v = block_sum(v, sh);
    __shared__ double beta, binv;
    if (threadIdx.x == 0) {
        beta = sqrt(v);
        binv = beta > 0.0 ? 1.0 / beta : 0.0;
    }
    __syncthreads();
    const double bb = beta;
    const double inv = binv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        Vb[i] = (VT)(b[i] * inv);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scal[0] = bb;
        scal[1] = bb;
        scal[2] = rtol * bb;
        for (int i = 0; i <= kmax; ++i) gv[i] = 0.0;
        gv[0] = bb;
        iflag[0] = (bb == 0.0) ? 1 : 0;
        iflag[1] = 0;
        iflag[2] = 0;
        iflag[3] = 0;
        iflag[4] = cap;
        *jdev = 0;
    }
}

// ---- Arnoldi step: classical Gram-Schmidt with selective re-orthogonalisation
// (the Daniel-Gragg-Kaufman-Stewart test: a second pass only when the first one
// cancelled more than half of ||w||^2), four kernels:
//   dots(pass 1):   h1_i = <V_i, w> (i <= j) and ||w||^2
//   update(pass 1): w1 = w - V h1; H(:,j) = h1; ||w1||^2 = ||w||^2 - ||h1||^2
//                   (Pythagoras, V orthonormal); re-orthogonalise iff
//                   ||w1||^2 <= ||w||^2 / 2
//   dots(pass 2):   h2_i = <V_i, w1> and ||w1||^2            (skipped if not)
//   update(pass 2): V_{j+1} = (w1 - V h2) / ||w2||, ||w2||^2 = ||w1||^2 - ||h2||^2;
//                   the last block to finish applies the Givens rotations, tests
//                   convergence and advances j.
// In FP64 on this GPU the passes are bound by the FP64 FMA rate (one FMA per
// 8-byte basis word), so every kernel does (j+1) N FMAs and a few adds: a dot
// work item is one (vector, 1024-element chunk) pair per warp, 32 FMAs per lane
// before one shuffle reduction.  With a float basis the 32 per-lane products are
// summed in FP32 (two chains of 16) and only the shuffle tree and the chunk sums
// are FP64, so the passes are bound by memory instead.  Chunk partials are summed
// in chunk order by the last block of each vector group (deterministic).
constexpr int kDotChunk = 1024;      // elements per warp work item (32 per lane)
constexpr int kDotVec = 8;           // vectors per dot block (one per warp)

// VEC (float basis, N a multiple of 4): full chunks are read as float4, lane l
// holding elements 4l + 128q .. 4l + 128q + 3.
template <typename VT, bool VEC>
__global__ void __launch_bounds__(256)
    k_gm_dots2(const VT* __restrict__ Vb, const int* __restrict__ jdev, long long N, double* __restrict__ part,
               int kmax, const int* __restrict__ iflag, const int* __restrict__ reo, double* __restrict__ hsum,
               unsigned int* __restrict__ counter, Bat bt) {
    __shared__ __align__(16) VT ws[kDotChunk];
    __shared__ bool last;
    long long off;
    if (!bat_enter(bt, (int)blockIdx.z, &off)) return;
    Vb = bsh(Vb, off); jdev = bsh(jdev, off); part = bsh(part, off); iflag = bsh(iflag, off); reo = bsh(reo, off);
    hsum = bsh(hsum, off); counter = bsh(counter, off);
    if (iflag[0]) return;
    if (reo && *reo == 0) return;                        // second pass not needed
    const int j = *jdev;
    const int nvec = j + 2;                              // slot j+1 = ||w||^2
    const int i0 = blockIdx.y * kDotVec;
    if (i0 >= nvec) return;
    const long long e0 = (long long)blockIdx.x * kDotChunk;
    const int len = (N - e0 < kDotChunk) ? (int)(N - e0) : kDotChunk;
    const VT* w = Vb + (long long)(j + 1) * N + e0;
    // full chunks on the float4 path read w straight from global memory (L1 serves
    // the other warps); otherwise w is staged in shared memory first
    const bool direct = VEC && len == kDotChunk;
    // FP64 basis, full chunk: every warp reads w from global memory too (L1 serves the
    // other warps), so the basis loads do not wait behind a staging pass and a barrier;
    // the same products in the same order as from shared memory
    const bool wdir = sizeof(VT) == 8 && len == kDotChunk;
    if (!direct && !wdir) {
        for (int t = threadIdx.x; t < kDotChunk; t += blockDim.x) ws[t] = (t < len) ? w[t] : VT(0);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = i0 + wid;
    const long long ld = kmax + 2;
    if (i < nvec) {
        const VT* vi = (i <= j) ? Vb + (long long)i * N + e0 : nullptr;
        VT s0 = VT(0), s1 = VT(0);
        if (direct) {
            const float4* w4 = reinterpret_cast<const float4*>(w);
            if (vi) {
                const float4* v4 = reinterpret_cast<const float4*>(vi);
                float4 a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) a[q] = v4[lane + 32 * q];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 b = w4[lane + 32 * q];
                    s0 += a[q].x * b.x;
                    s1 += a[q].y * b.y;
                    s0 += a[q].z * b.z;
                    s1 += a[q].w * b.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 b = w4[lane + 32 * q];
                    s0 += b.x * b.x;
                    s1 += b.y * b.y;
                    s0 += b.z * b.z;
                    s1 += b.w * b.w;
                }
            }
        } else if (vi && wdir) {
#pragma unroll
            for (int q0 = 0; q0 < 32; q0 += 8) {
                VT a[8], b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    a[u] = vi[lane + 32 * (q0 + u)];
                    b[u] = w[lane + 32 * (q0 + u)];
                }
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    s0 += a[u] * b[u];
                    s1 += a[u + 1] * b[u + 1];
                }
            }
        } else if (wdir) {
#pragma unroll 8
            for (int q = 0; q < 32; q += 2) {
                const VT x0 = w[lane + 32 * q], x1 = w[lane + 32 * (q + 1)];
                s0 += x0 * x0;
                s1 += x1 * x1;
            }
        } else if (vi && len == kDotChunk) {
#pragma unroll
            for (int q0 = 0; q0 < 32; q0 += 8) {
                VT a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = vi[lane + 32 * (q0 + u)];
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    s0 += a[u] * ws[lane + 32 * (q0 + u)];
                    s1 += a[u + 1] * ws[lane + 32 * (q0 + u + 1)];
                }
            }
        } else if (vi) {
            for (int q = 0; q < 32; ++q) {
                const int e = lane + 32 * q;
                if (e < len) s0 += vi[e] * ws[e];
            }
        } else {
#pragma unroll 8
            for (int q = 0; q < 32; q += 2) {
                const VT x0 = ws[lane + 32 * q], x1 = ws[lane + 32 * (q + 1)];
                s0 += x0 * x0;
                s1 += x1 * x1;
            }
        }
        double t = (double)s0 + (double)s1;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) {
            part[(long long)blockIdx.x * ld + i] = t;
            __threadfence();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&counter[blockIdx.y], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    // the last chunk block of this vector group: chunk partials in chunk order,
    // one warp per vector, fixed shuffle tree
    __threadfence();
    if (i < nvec) {
        double t = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32) t += __ldcg(&part[(long long)c * ld + i]);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) hsum[i] = t;
    }
    if (threadIdx.x == 0) counter[blockIdx.y] = 0u;
}

// the final dot sums of the pass (written by the dot kernel's last blocks), and
// their copy in the basis type for the update
template <typename VT>
__device__ __forceinline__ void load_sums(const double* __restrict__ hsum, int nvec, double* h, VT* hv) {
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        h[i] = hsum[i];
        hv[i] = (VT)h[i];
    }
    __syncthreads();
}

// v - sum_{i < nv} h[i] V_i[e], in order of i, sixteen basis loads in flight
template <typename VT>
__device__ __forceinline__ VT sub_basis(const VT* __restrict__ Vb, long long N, long long e, const VT* h, int nv,
                                        VT v) {
    int i = 0;
    for (; i + 16 <= nv; i += 16) {
        VT a[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) a[u] = Vb[(long long)(i + u) * N + e];
#pragma unroll
        for (int u = 0; u < 16; ++u) v -= h[i + u] * a[u];
    }
    for (; i < nv; ++i) v -= h[i] * Vb[(long long)i * N + e];
    return v;
}

// sum_{i < n} h[i]^2 by warp 0 (lane-strided partials, then a fixed xor tree);
// the result is returned to lane 0 of warp 0
__device__ __forceinline__ double warp_sumsq(const double* h, int n) {
    const int lane = threadIdx.x & 31;
    double q = 0.0;
    for (int i = lane; i < n; i += 32) q += h[i] * h[i];
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    return q;
}

// Elements per block of the update kernels: FP64 one per thread; float 128.
template <typename VT>
constexpr int upd_elems() { return sizeof(VT) == 8 ? 256 : 128; }

// four float elements of lane `lane` in the 128-element block at `base`:
// VEC: the float4 at base + 4 lane (N a multiple of 4); else base + lane + 32 k
template <bool VEC>
__device__ __forceinline__ void load4(const float* __restrict__ v, long long base, int lane, long long N, float (&a)[4]) {
    if (VEC) {
        const long long e = base + 4 * lane;
        if (e < N) {
            const float4 t = *reinterpret_cast<const float4*>(v + e);
            a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
        } else {
            a[0] = a[1] = a[2] = a[3] = 0.f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long e = base + lane + 32 * k;
            a[k] = e < N ? v[e] : 0.f;
        }
    }
}

// w = (sub ? w - sum_{i <= j} hv[i] V_i : w) * scale on this block's elements,
// w = V_{j+1}.  FP64: one element per thread, the vectors in order (sub_basis).
// Float: 128 elements per block, four per lane; warp q sums the vectors
// i = q, q + 8, q + 16, ... (four loads in flight) and the eight warp partials
// are added in warp order, so the result is the same with and without VEC.
// Every thread of the block must call it (it has a barrier on the float path).
template <typename VT, bool VEC>
__device__ __forceinline__ void block_update(VT* __restrict__ Vb, long long N, int j, const VT* hv, bool sub,
                                             VT scale) {
    VT* w = Vb + (long long)(j + 1) * N;
    if constexpr (sizeof(VT) == 8) {
        const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (e < N) w[e] = (sub ? sub_basis(Vb, N, e, hv, j + 1, w[e]) : w[e]) * scale;
    } else {
        __shared__ __align__(16) float red[8][128];
        const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
        const long long base = (long long)blockIdx.x * 128;
        if (sub) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            int i = q;
            for (; i + 24 <= j; i += 32) {
                float a[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) load4<VEC>(Vb + (long long)(i + 8 * u) * N, base, lane, N, a[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[k] += hv[i + 8 * u] * a[u][k];
            }
            for (; i <= j; i += 8) {
                float a[4];
                load4<VEC>(Vb + (long long)i * N, base, lane, N, a);
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] += hv[i] * a[k];
            }
            if (VEC) {
                reinterpret_cast<float4*>(red[q])[lane] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) red[q][lane + 32 * k] = acc[k];
            }
        }
        __syncthreads();
        if (threadIdx.x < 128) {
            const long long e = base + threadIdx.x;
            if (e < N) {
                float t = 0.f;
                if (sub)
#pragma unroll
                    for (int r = 0; r < 8; ++r) t += red[r][threadIdx.x];
                w[e] = (w[e] - t) * scale;
            }
        }
    }
}

template <typename VT, bool VEC>
__global__ void __launch_bounds__(256)
    k_gm_update1(VT* __restrict__ Vb, const int* __restrict__ jdev, long long N, const double* __restrict__ hsum,
                 int kmax, double* __restrict__ H, double* __restrict__ scal, int* __restrict__ reo,
                 const int* __restrict__ force, const int* __restrict__ iflag, Bat bt) {
    __shared__ double h[kMaxKrylov + 2];
    __shared__ VT hv[kMaxKrylov + 2];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    Vb = bsh(Vb, off); jdev = bsh(jdev, off); hsum = bsh(hsum, off); H = bsh(H, off); scal = bsh(scal, off);
    reo = bsh(reo, off); force = bsh(force, off); iflag = bsh(iflag, off);
    if (iflag[0]) return;
    const int j = *jdev;
    load_sums(hsum, j + 2, h, hv);                  // h1[0..j], ||w||^2 in h[j+1]
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double q = warp_sumsq(h, j + 1);
        const double n1 = h[j + 1] - q;             // ||w1||^2
        const int r = (*force != 0) || !(n1 > 0.5 * h[j + 1]);
        if (threadIdx.x == 0) {
            *reo = r;
            scal[4] = n1;
        }
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= j; i += blockDim.x) H[(long long)j * (kmax + 1) + i] = h[i];
    block_update<VT, VEC>(Vb, N, j, hv, true, VT(1));
}

template <typename VT, bool VEC>
__global__ void __launch_bounds__(256)
    k_gm_update2(VT* __restrict__ Vb, const int* __restrict__ jdev_c, long long N, const double* __restrict__ hsum,
                 int kmax, double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                 double* __restrict__ gv, double* __restrict__ scal, int* __restrict__ iflag,
                 const int* __restrict__ reo, unsigned int* __restrict__ counter, int* __restrict__ jdev, Bat bt) {
    // dynamic shared memory sized for kmax: h, scol (kmax + 2), scs, ssn
    // (kmax) doubles, then hv (kmax + 2) in the basis type
    extern __shared__ __align__(16) double dsh[];
    double* h = dsh;
    double* scol = h + (kmax + 2);
    double* scs = scol + (kmax + 2);
    double* ssn = scs + kmax;
    VT* hv = reinterpret_cast<VT*>(ssn + kmax);
    __shared__ double shn, sinv;
    __shared__ bool last;
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    Vb = bsh(Vb, off); jdev_c = bsh(jdev_c, off); hsum = bsh(hsum, off); H = bsh(H, off); cs = bsh(cs, off);
    sn = bsh(sn, off); gv = bsh(gv, off); scal = bsh(scal, off); iflag = bsh(iflag, off); reo = bsh(reo, off);
    counter = bsh(counter, off); jdev = bsh(jdev, off);
    if (iflag[0]) return;
    const int j = *jdev_c;
    const bool second = *reo != 0;
    if (second) {
        load_sums(hsum, j + 2, h, hv);                  // h2[0..j], ||w1||^2 in h[j+1]
    } else {
        for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = 0.0;
        __syncthreads();
    }
    if (threadIdx.x < 32) {
        const double n2 = second ? h[j + 1] - warp_sumsq(h, j + 1) : scal[4];
        if (threadIdx.x == 0) {
            const double r = n2 > 0.0 ? sqrt(n2) : 0.0;
            shn = r;
            sinv = r > 0.0 ? 1.0 / r : 0.0;          // one FP64 division per block
        }
    }
    double hn;
    if constexpr (sizeof(VT) == 8) {
        // FP64: the subtraction does not wait for warp 0's norm; only the scaling does
        const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        VT* w = Vb + (long long)(j + 1) * N;
        VT v = VT(0);
        if (e < N) v = second ? sub_basis(Vb, N, e, hv, j + 1, w[e]) : w[e];
        __syncthreads();
        hn = shn;
        if (e < N) w[e] = v * (VT)sinv;
    } else {
        __syncthreads();
        hn = shn;
        block_update<VT, VEC>(Vb, N, j, hv, second, (VT)sinv);
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)(gridDim.x - 1));
    __syncthreads();
    if (!last) return;
    // the last block: every block has read j; H column, Givens, convergence, j += 1
    double* col = H + (long long)j * (kmax + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        scol[i] = col[i] + h[i];
        if (i < j) { scs[i] = cs[i]; ssn[i] = sn[i]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *counter = 0u;
        scol[j + 1] = hn;
        // previous rotations; the rotated entry i+1 is carried in a register
        double cr = scol[0];
        for (int i = 0; i < j; ++i) {
            const double b = scol[i + 1];
            scol[i] = scs[i] * cr + ssn[i] * b;
            cr = -ssn[i] * cr + scs[i] * b;
        }
        scol[j] = cr;
        const double a = scol[j], bq = scol[j + 1];
        const double r = hypot(a, bq);
        double c = 1.0, sgv = 0.0;
        if (r > 0.0) { c = a / r; sgv = bq / r; }
        cs[j] = c;
        sn[j] = sgv;
        scol[j] = r;
        scol[j + 1] = 0.0;
        const double gj = gv[j];
        gv[j + 1] = -sgv * gj;
        gv[j] = c * gj;
        const double res = fabs(sgv * gj);
        scal[1] = res;
        scal[3] = hn;
        iflag[1] = j + 1;
        int stop = 0;
        if (!(res > scal[2])) stop = 1;                                   // converged
        if (!(hn > 1e-300) || !isfinite(res)) { stop = 1; iflag[2] = 1; }  // breakdown
        if (j + 1 >= kmax || j + 1 >= iflag[4]) { stop = 1; iflag[3] = 1; }  // cap
        if (stop) iflag[0] = 1;
        else *jdev = j + 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = scol[i];
}

// Back substitution H y = g on the k completed columns; the packed upper
// triangle is staged in shared memory when it fits (use_smem), else read from H.
__global__ void k_gm_backsolve(const double* __restrict__ H, const double* __restrict__ gv, const int* __restrict__ iflag,
                               int kmax, double* __restrict__ y, int use_smem, Bat bt) {
    extern __shared__ double shH[];
    long long off;
    if (!bat_enter(bt, (int)blockIdx.x, &off)) return;
    H = bsh(H, off); gv = bsh(gv, off); iflag = bsh(iflag, off); y = bsh(y, off);
    const int k = iflag[1];
    if (use_smem) {
        for (int e = threadIdx.x; e < k * (k + 1) / 2; e += blockDim.x) {
            // e -> (column l, row i <= l) in packed column-major order
            int l = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
            while ((l + 1) * (l + 2) / 2 <= e) ++l;
            while (l * (l + 1) / 2 > e) --l;
            const int i = e - l * (l + 1) / 2;
            shH[e] = H[(long long)l * (kmax + 1) + i];
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l)
            s -= (use_smem ? shH[(size_t)l * (l + 1) / 2 + i] : H[(long long)l * (kmax + 1) + i]) * y[l];
        const double diag = use_smem ? shH[(size_t)i * (i + 1) / 2 + i] : H[(long long)i * (kmax + 1) + i];
        y[i] = diag != 0.0 ? s / diag : 0.0;
    }
}

template <typename VT>
__global__ void k_gm_combine(const VT* __restrict__ Vb, const double* __restrict__ y,
                             const int* __restrict__ iflag, long long N, double* __restrict__ x, Bat bt) {
    long long off;
    if (!bat_enter(bt, (int)blockIdx.y, &off)) return;
    Vb = bsh(Vb, off); y = bsh(y, off); iflag = bsh(iflag, off); x = bsh(x, off);
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int k = iflag[1];
    double s = 0.0;
    int i = 0;
    for (; i + 8 <= k; i += 8) {
        VT a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = Vb[(long long)(i + u) * N + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += y[i + u] * (double)a[u];
    }
    for (; i < k; ++i) s += y[i] * (double)Vb[(long long)i * N + e];
    x[e] = s;
}

// Body terminator of the device-side GMRES loop: keep looping while not stopped.
__global__ void k_gm_setcond(cudaGraphConditionalHandle h, const int* __restrict__ iflag) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, iflag[0] ? 0u : 1u);
}

cudaError_t launch_gm_setcond(cudaGraphConditionalHandle h, const int* iflag, cudaStream_t s) {
    k_gm_setcond<<<1, 32, 0, s>>>(h, iflag);
    note_launch();
    return cudaGetLastError();
}

// Batched loop: keep looping while any problem of the batch has not stopped.
__global__ void k_gm_setcond_batch(cudaGraphConditionalHandle h, const int* __restrict__ iflag, Bat bt) {
    int running = 0;
    for (int pb = threadIdx.x; pb < bt.np; pb += blockDim.x) {
        const long long off = bt.delta ? bt.delta[pb] : 0LL;
        if (bsh(iflag, off)[0] == 0) running = 1;
    }
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, running ? 1u : 0u);
}

cudaError_t launch_gm_setcond_batch(cudaGraphConditionalHandle h, const int* iflag, cudaStream_t s, const Bat& bt) {
    k_gm_setcond_batch<<<1, 128, 0, s>>>(h, iflag, bt);
    note_launch();
    return cudaGetLastError();
}

// Stop the GMRES of every problem the mask selects (problems that take no part in
// a batched Krylov solve must not run in its device-side loop).
__global__ void k_gm_stop(int* __restrict__ iflag, Bat bt) {
    const int pb = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (pb >= bt.np) return;
    long long off;
    if (!bat_enter(bt, pb, &off)) return;
    bsh(iflag, off)[0] = 1;
}

cudaError_t launch_gm_stop(int* iflag, cudaStream_t s, const Bat& bt) {
    k_gm_stop<<<(bt.np + 63) / 64, 64, 0, s>>>(iflag, bt);
    note_launch();
    return cudaGetLastError();
}

int gmres_dot_blocks(long long N) { return (int)((N + kDotChunk - 1) / kDotChunk); }
int gmres_dot_groups(int kmax) { return (kmax + 2 + kDotVec - 1) / kDotVec; }
int gmres_upd_blocks(long long N) { return (int)((N + 255) / 256); }

template <typename VT>
cudaError_t gmres_start(GmresDev& G, const double* b, double rtol, cudaStream_t s, int cap, const Bat& bt) {
    int np = 0;
    cudaError_t e = launch_sumsq(b, G.N, G.part_norm, &np, s, bt);
    if (e != cudaSuccess) return e;
    const int nb = gmres_upd_blocks(G.N) < 1024 ? gmres_upd_blocks(G.N) : 1024;
    const int c = (cap > 0 && cap < G.kmax) ? cap : G.kmax;
    k_gm_start<VT><<<dim3(nb, bt.np), 256, 0, s>>>(gmres_basis<VT>(G), b, G.N, G.part_norm, np, rtol, G.scal, G.gv,
                                                   G.kmax, c, G.iflag, G.jdev, G.H, bt);
    note_launch();
    return cudaGetLastError();
}

template <typename VT, bool VEC>
static void arnoldi_launch(GmresDev& G, cudaStream_t s, const Bat& bt) {
    const int nch = gmres_dot_blocks(G.N);
    const int bu = (int)((G.N + upd_elems<VT>() - 1) / upd_elems<VT>());
    const dim3 gd(nch, gmres_dot_groups(G.kmax), bt.np);
    const dim3 gu(bu, bt.np);
    VT* V = gmres_basis<VT>(G);
    k_gm_dots2<VT, VEC><<<gd, 256, 0, s>>>(V, G.jdev, G.N, G.part_dots, G.kmax, G.iflag, nullptr, G.hsum,
                                             G.counter, bt);
    note_launch();
    k_gm_update1<VT, VEC><<<gu, 256, 0, s>>>(V, G.jdev, G.N, G.hsum, G.kmax, G.H, G.scal, G.reo, G.force, G.iflag,
                                             bt);
    note_launch();
    k_gm_dots2<VT, VEC><<<gd, 256, 0, s>>>(V, G.jdev, G.N, G.part_dots, G.kmax, G.iflag, G.reo, G.hsum, G.counter,
                                             bt);
    note_launch();
    const size_t upd2_smem = (size_t)(4 * G.kmax + 4) * sizeof(double) + (size_t)(G.kmax + 2) * sizeof(VT);
    k_gm_update2<VT, VEC><<<gu, 256, upd2_smem, s>>>(V, G.jdev, G.N, G.hsum, G.kmax, G.H, G.cs, G.sn, G.gv,
                                                     G.scal, G.iflag, G.reo, G.counter2, G.jdev, bt);
    note_launch();
}

template <typename VT>
cudaError_t gmres_arnoldi(GmresDev& G, cudaStream_t s, const Bat& bt) {
    // float4 access needs every basis vector 16-byte aligned: N a multiple of 4
    if (sizeof(VT) == 4 && G.N % 4 == 0) arnoldi_launch<VT, true>(G, s, bt);
    else arnoldi_launch<VT, false>(G, s, bt);
    return cudaGetLastError();
}


__global__ void k_gm_setj(int* __restrict__ jdev, int* __restrict__ iflag, unsigned int* __restrict__ counter, int j,
                          int kmax) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *jdev = j;
        iflag[0] = iflag[1] = iflag[2] = iflag[3] = 0;
        iflag[4] = kmax;
        *counter = 0u;
    }
}

template <typename VT>
cudaError_t gmres_timed_step(GmresDev& G, int j, cudaStream_t s) {
    if (j < 0 || j >= G.kmax) return cudaErrorInvalidValue;
    k_gm_setj<<<1, 32, 0, s>>>(G.jdev, G.iflag, G.counter2, j, G.kmax);
    note_launch();
    return gmres_arnoldi<VT>(G, s, Bat{});
}

template <typename VT>
cudaError_t gmres_finish(GmresDev& G, double* x, cudaStream_t s, const Bat& bt) {
    const size_t tri = (size_t)G.kmax * (G.kmax + 1) / 2 * sizeof(double);
    const int use_smem = tri <= 200 * 1024;
    k_gm_backsolve<<<bt.np, 256, use_smem ? tri : 0, s>>>(G.H, G.gv, G.iflag, G.kmax, G.y, use_smem, bt);
    note_launch();
    k_gm_combine<VT><<<dim3((unsigned)((G.N + 255) / 256), bt.np), 256, 0, s>>>(gmres_basis<VT>(G), G.y, G.iflag,
                                                                               G.N, x, bt);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t gmres_start<double>(GmresDev&, const double*, double, cudaStream_t, int, const Bat&);
template cudaError_t gmres_start<float>(GmresDev&, const double*, double, cudaStream_t, int, const Bat&);
template cudaError_t gmres_arnoldi<double>(GmresDev&, cudaStream_t, const Bat&);
template cudaError_t gmres_arnoldi<float>(GmresDev&, cudaStream_t, const Bat&);
template cudaError_t gmres_timed_step<double>(GmresDev&, int, cudaStream_t);
template cudaError_t gmres_timed_step<float>(GmresDev&, int, cudaStream_t);
template cudaError_t gmres_finish<double>(GmresDev&, double*, cudaStream_t, const Bat&);
template cudaError_t gmres_finish<float>(GmresDev&, double*, cudaStream_t, const Bat&);

// ---- vector blocks of the flexible GMRES on G (host-driven outer loop) ---------
// part[v * nchunks + c] = sum over chunk c (kFgChunk elements) of V_v . w, v < nv
constexpr int kFgChunk = 2048;

__global__ void __launch_bounds__(256)
    k_mdot(const double* __restrict__ V, long long ld, const double* __restrict__ w, long long N, double* __restrict__ part) {
    __shared__ double sh[32];
    const long long e0 = (long long)blockIdx.x * kFgChunk;
    const double* v = V + (long long)blockIdx.y * ld;
    double acc = 0.0;
    for (int t = threadIdx.x; t < kFgChunk; t += blockDim.x) {
        const long long e = e0 + t;
        if (e < N) acc += v[e] * w[e];
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// w += sgn * sum_{v < nv} h[v] V_v, in order of v
__global__ void k_maxpy(double* __restrict__ w, const double* __restrict__ V, long long ld, const double* __restrict__ h,
                        int nv, long long N, double sgn) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    double acc = 0.0;
    for (int v = 0; v < nv; ++v) acc += h[v] * V[(long long)v * ld + e];
    w[e] += sgn * acc;
}

int fg_chunks(long long N) { return (int)((N + kFgChunk - 1) / kFgChunk); }

cudaError_t launch_mdot(const double* V, long long ld, int nv, const double* w, long long N, double* part,
                        cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    k_mdot<<<dim3((unsigned)fg_chunks(N), (unsigned)nv), 256, 0, s>>>(V, ld, w, N, part);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_maxpy(double* w, const double* V, long long ld, const double* h, int nv, long long N, double sgn,
                         cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    k_maxpy<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(w, V, ld, h, nv, N, sgn);
    note_launch();
    return cudaGetLastError();
}

// ---- iterative A_alpha^{-1}: block-Jacobi preconditioner and helpers -----------
__device__ __forceinline__ long long pcg_dof(const PcgGeo& pg, int t, const int* coord, int l) {
    // 1D interior index per axis: vertex v -> v; bubble b of cell c -> (m - 1) + c nbub + b
    long long I = 0, stride = 1;
    int rl = l;
    for (int j = 0; j < pg.d; ++j) {
        int i1;
        if ((t >> j) & 1) {
            const int b = rl % pg.nbub;
            rl /= pg.nbub;
            i1 = pg.m[j] - 1 + coord[j] * pg.nbub + b;
        } else {
            i1 = coord[j];
        }
        I += (long long)i1 * stride;
        stride *= pg.n1[j];
    }
    return I;
}

// one block per entity: gather its residual entries, multiply by the type's inverse block
__global__ void __launch_bounds__(128) k_ainv_blocks(PcgGeo pg, double ainv, const double* __restrict__ r,
                                                     double* __restrict__ z) {
    extern __shared__ double smp[];
    const long long ent = blockIdx.x;
    const int ntyp = 1 << pg.d;
    int t = 1;
    while (t + 1 < ntyp && ent >= pg.eoff[t + 1]) ++t;
    long long e = ent - pg.eoff[t];
    int coord[kMaxDim] = {0, 0, 0};
    for (int j = 0; j < pg.d; ++j) {
        const long long ext = ((t >> j) & 1) ? pg.m[j] : pg.nv[j];
        coord[j] = (int)(e % ext);
        e /= ext;
    }
    const int nb = pg.bsize[t];
    double* rs = smp;
    long long* idx = reinterpret_cast<long long*>(smp + pg.bmax);
    for (int l = threadIdx.x; l < nb; l += blockDim.x) {
        const long long I = pcg_dof(pg, t, coord, l);
        idx[l] = I;
        rs[l] = r[I];
    }
    __syncthreads();
    const double* Bi = pg.Binv + pg.boff[t];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nb; ++k) acc += Bi[(size_t)i * nb + k] * rs[k];
        z[idx[i]] = ainv * acc;
    }
}

cudaError_t launch_ainv_blocks(const PcgGeo& pg, double alpha, const double* r, double* z, cudaStream_t s) {
    const long long ne = pg.eoff[1 << pg.d] - pg.eoff[1];
    if (ne <= 0) return cudaSuccess;
    const size_t smem = (size_t)pg.bmax * (sizeof(double) + sizeof(long long));
    k_ainv_blocks<<<(unsigned)ne, 128, smem, s>>>(pg, 1.0 / alpha, r, z);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_vertex_move(PcgGeo pg, const double* __restrict__ src, double* __restrict__ dst, long long nc,
                              int gather) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int coord[kMaxDim] = {0, 0, 0};
    long long e = c;
    for (int j = 0; j < pg.d; ++j) {
        coord[j] = (int)(e % pg.nv[j]);
        e /= pg.nv[j];
    }
    const long long I = pcg_dof(pg, 0, coord, 0);
    if (gather) dst[c] = src[I];
    else dst[I] = src[c];
}

cudaError_t launch_vertex_gather(const PcgGeo& pg, const double* r, double* rc, long long nc, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    k_vertex_move<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(pg, r, rc, nc, 1);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_vertex_scatter(const PcgGeo& pg, const double* zc, double* z, long long nc, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    k_vertex_move<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(pg, zc, z, nc, 0);
    note_launch();
    return cudaGetLastError();
}

// ---- overlapping cell patches (two-level additive Schwarz) -----------------------
// local dof list of cell c along one axis: [left hat if c >= 1, right hat if c + 1 <= m - 1,
// bubbles]; returns the count and the number of hats
__device__ __forceinline__ int cell_nh(int m, int c) { return (c >= 1 ? 1 : 0) + (c + 1 <= m - 1 ? 1 : 0); }
__device__ __forceinline__ int cell_dof_1d(int m, int nbub, int c, int pos) {
    const int nh = cell_nh(m, c);
    if (pos < nh) return (pos == 0 && c >= 1) ? c - 1 : c;     // left hat: vertex c; right hat: vertex c + 1
    return m - 1 + c * nbub + (pos - nh);
}

__global__ void __launch_bounds__(128) k_cells_solve(PcgGeo pg, const double* __restrict__ r) {
    extern __shared__ double smc[];
    const long long cell = blockIdx.x;
    int c[kMaxDim] = {0, 0, 0}, n1d[kMaxDim] = {1, 1, 1};
    long long e = cell;
    int cls = 0, nb = 1;
    for (int j = 0; j < pg.d; ++j) {
        c[j] = (int)(e % pg.m[j]);
        e /= pg.m[j];
        const int code = (c[j] >= 1 ? 1 : 0) | (c[j] + 1 <= pg.m[j] - 1 ? 2 : 0);
        cls |= code << (2 * j);
        n1d[j] = cell_nh(pg.m[j], c[j]) + pg.nbub;
        nb *= n1d[j];
    }
    double* rs = smc;
    for (int l = threadIdx.x; l < nb; l += blockDim.x) {
        long long I = 0, stride = 1;
        int rl = l;
        for (int j = 0; j < pg.d; ++j) {
            const int pos = rl % n1d[j];
            rl /= n1d[j];
            I += (long long)cell_dof_1d(pg.m[j], pg.nbub, c[j], pos) * stride;
            stride *= pg.n1[j];
        }
        rs[l] = r[I];
    }
    __syncthreads();
    const double* Bi = pg.Cinv + pg.coff[cls];
    double* Y = pg.Y + cell * (long long)pg.cmax;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nb; ++k) acc += Bi[(size_t)i * nb + k] * rs[k];
        Y[i] = acc;
    }
}

cudaError_t launch_cells_solve(const PcgGeo& pg, long long ncells, const double* r, cudaStream_t s) {
    k_cells_solve<<<(unsigned)ncells, 128, (size_t)pg.cmax * sizeof(double), s>>>(pg, r);
    note_launch();
    return cudaGetLastError();
}

// every interior dof sums the block solutions of the (up to 2^d) cells that hold it, in
// the binary order of the choices per axis, plus the coarse correction at vertex dofs
__global__ void k_cells_gather(PcgGeo pg, double ainv, const double* __restrict__ zc, double* __restrict__ z,
                               long long n) {
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    int cc[kMaxDim][2], pp[kMaxDim][2], nch[kMaxDim];
    long long e = I;
    bool vertex = true;
    long long vidx = 0, vstride = 1;
    for (int j = 0; j < pg.d; ++j) {
        const int i1 = (int)(e % pg.n1[j]);
        e /= pg.n1[j];
        const int m = pg.m[j];
        if (i1 < m - 1) {
            const int v = i1 + 1;                         // interior vertex v: right hat of cell v-1, left of v
            cc[j][0] = v - 1; pp[j][0] = (v - 1 >= 1) ? 1 : 0;
            cc[j][1] = v;     pp[j][1] = 0;
            nch[j] = 2;
            vidx += (long long)i1 * vstride;
            vstride *= pg.nv[j];
        } else {
            const int q = i1 - (m - 1), cell = q / pg.nbub;
            cc[j][0] = cell;
            pp[j][0] = cell_nh(m, cell) + q % pg.nbub;
            nch[j] = 1;
            vertex = false;
        }
    }
    double acc = 0.0;
    const int ncomb = 1 << pg.d;
    for (int sel = 0; sel < ncomb; ++sel) {
        bool ok = true;
        long long cell = 0, cstride = 1, l = 0, lstride = 1;
        for (int j = 0; j < pg.d; ++j) {
            const int bj = (sel >> j) & 1;
            if (bj >= nch[j]) { ok = false; break; }
            cell += (long long)cc[j][bj] * cstride;
            cstride *= pg.m[j];
            l += (long long)pp[j][bj] * lstride;
            lstride *= cell_nh(pg.m[j], cc[j][bj]) + pg.nbub;
        }
        if (ok) acc += pg.Y[cell * (long long)pg.cmax + l];
    }
    double v = ainv * acc;
    if (vertex && zc) v += zc[vidx];
    z[I] = v;
}

cudaError_t launch_cells_gather(const PcgGeo& pg, double alpha, const double* zc, double* z, long long n,
                                cudaStream_t s) {
    k_cells_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pg, 1.0 / alpha, zc, z, n);
    note_launch();
    return cudaGetLastError();
}

// ---- vertex-star patches -------------------------------------------------------
// 1D interior index of position `pos` of the star of patch q (interior vertex v = q + 1)
// along an axis with m cells: [bubbles of cell v-1, hat v, bubbles of cell v]; on a
// one-cell axis the patch is that cell's bubbles
__device__ __forceinline__ int star_dof_1d(int m, int nbub, int q, int pos) {
    if (m < 2) return m - 1 + pos;
    const int v = q + 1;
    if (pos < nbub) return m - 1 + (v - 1) * nbub + pos;
    if (pos == nbub) return v - 1;
    return m - 1 + v * nbub + (pos - nbub - 1);
}

// one pass of a box fast diagonalisation along axis ax: out[.., a, ..] = sum_k W(a, k) in[.., k, ..],
// W = V^T (fwd: V[k][a]) or V (V[a][k])
__device__ __forceinline__ void box_pass(const double* in, double* out, const double* V, bool fwd, const int* ext,
                                         int d, int ax, int tot) {
    int stride = 1;
    for (int j = 0; j < ax; ++j) stride *= ext[j];
    const int n = ext[ax];
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int a = (e / stride) % n;
        const int base = e - a * stride;
        double acc = 0.0;
        if (fwd)
            for (int k = 0; k < n; ++k) acc += V[k * n + a] * in[base + k * stride];
        else
            for (int k = 0; k < n; ++k) acc += V[a * n + k] * in[base + k * stride];
        out[e] = acc;
    }
    (void)d;
}

__global__ void __launch_bounds__(256) k_stars_solve(PcgGeo pg, const double* __restrict__ r) {
    extern __shared__ double sms[];
    const int d = pg.d;
    int q[kMaxDim] = {0, 0, 0};
    long long e = blockIdx.x;
    for (int j = 0; j < d; ++j) {
        q[j] = (int)(e % pg.np_[j]);
        e /= pg.np_[j];
    }
    int ext[kMaxDim] = {1, 1, 1}, tot = 1;
    for (int j = 0; j < d; ++j) { ext[j] = pg.ns[j]; tot *= ext[j]; }
    double* b0 = sms;
    double* b1 = sms + tot;
    for (int l = threadIdx.x; l < tot; l += blockDim.x) {
        long long I = 0, stride = 1;
        int rl = l;
        for (int j = 0; j < d; ++j) {
            const int pos = rl % ext[j];
            rl /= ext[j];
            I += (long long)star_dof_1d(pg.m[j], pg.nbub, q[j], pos) * stride;
            stride *= pg.n1[j];
        }
        b0[l] = r[I];
    }
    __syncthreads();
    double *in = b0, *out = b1;
    for (int ax = 0; ax < d; ++ax) {
        box_pass(in, out, pg.Vs[ax], true, ext, d, ax, tot);
        __syncthreads();
        double* t = in; in = out; out = t;
    }
    for (int l = threadIdx.x; l < tot; l += blockDim.x) {
        int rl = l;
        double lsum = 0.0;
        for (int j = 0; j < d; ++j) {
            lsum += pg.lams[j][rl % ext[j]];
            rl /= ext[j];
        }
        in[l] /= lsum;
    }
    __syncthreads();
    for (int ax = 0; ax < d; ++ax) {
        box_pass(in, out, pg.Vs[ax], false, ext, d, ax, tot);
        __syncthreads();
        double* t = in; in = out; out = t;
    }
    double* Y = pg.Ys + (long long)blockIdx.x * tot;
    for (int l = threadIdx.x; l < tot; l += blockDim.x) Y[l] = in[l];
}

cudaError_t launch_stars_solve(const PcgGeo& pg, const double* r, cudaStream_t s) {
    long long npatch = 1, tot = 1;
    for (int j = 0; j < pg.d; ++j) { npatch *= pg.np_[j]; tot *= pg.ns[j]; }
    k_stars_solve<<<(unsigned)npatch, 256, (size_t)(2 * tot) * sizeof(double), s>>>(pg, r);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_stars_gather(PcgGeo pg, double ainv, const double* __restrict__ zc, double* __restrict__ z,
                               long long n) {
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    int qq[kMaxDim][2], pp[kMaxDim][2], nch[kMaxDim];
    long long e = I, vidx = 0, vstride = 1;
    bool vertex = true;
    for (int j = 0; j < pg.d; ++j) {
        const int i1 = (int)(e % pg.n1[j]);
        e /= pg.n1[j];
        const int m = pg.m[j], nb = pg.nbub;
        if (m < 2) {                                  // one cell: the single patch's bubbles
            qq[j][0] = 0; pp[j][0] = i1 - (m - 1); nch[j] = 1;
            vertex = false;
        } else if (i1 < m - 1) {                      // hat of interior vertex v = i1 + 1: centre of patch v
            qq[j][0] = i1; pp[j][0] = nb; nch[j] = 1;
            vidx += (long long)i1 * vstride;
            vstride *= pg.nv[j];
        } else {                                      // bubble b of cell c: stars of vertices c and c + 1
            const int qb = i1 - (m - 1), c = qb / nb, b = qb % nb;
            nch[j] = 0;
            if (c >= 1) { qq[j][nch[j]] = c - 1; pp[j][nch[j]] = nb + 1 + b; ++nch[j]; }
            if (c + 1 <= m - 1) { qq[j][nch[j]] = c; pp[j][nch[j]] = b; ++nch[j]; }
            vertex = false;
        }
    }
    double acc = 0.0;
    for (int sel = 0; sel < (1 << pg.d); ++sel) {
        bool ok = true;
        long long patch = 0, pstride = 1, l = 0, lstride = 1;
        for (int j = 0; j < pg.d; ++j) {
            const int bj = (sel >> j) & 1;
            if (bj >= nch[j]) { ok = false; break; }
            patch += (long long)qq[j][bj] * pstride;
            pstride *= pg.np_[j];
            l += (long long)pp[j][bj] * lstride;
            lstride *= pg.ns[j];
        }
        if (ok) acc += pg.Ys[patch * lstride + l];
    }
    double v = ainv * acc;
    if (vertex && zc) v += zc[vidx];
    z[I] = v;
}

cudaError_t launch_stars_gather(const PcgGeo& pg, double alpha, const double* zc, double* z, long long n,
                                cudaStream_t s) {
    k_stars_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pg, 1.0 / alpha, zc, z, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_aapply(const Geo<double>& g, double alpha, const double* x, double* y, cudaStream_t s) {
    if (g.d == 2)
        k_urow<2, double, double, double, true, false, false><<<utile_grid<2>(g.n1), 256,
                                                                urow_smem<2>(g, true, false), s>>>(
            g, alpha, x, 0.0, (const double*)nullptr, (const double*)nullptr, nullptr, nullptr, nullptr, nullptr, y,
            nullptr, Bat{}, 0);
    else
        k_urow<3, double, double, double, true, false, false><<<utile_grid<3>(g.n1), 256,
                                                                urow_smem<3>(g, true, false), s>>>(
            g, alpha, x, 0.0, (const double*)nullptr, (const double*)nullptr, nullptr, nullptr, nullptr, nullptr, y,
            nullptr, Bat{}, 0);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, long long n,
                      double* __restrict__ part) {
    __shared__ double sh[32];
    double v = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v += a[i] * b[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

cudaError_t launch_dot(const double* a, const double* b, long long n, double* part, int* nparts, cudaStream_t s) {
    int nb = (int)((n + 255) / 256);
    if (nb > 1024) nb = 1024;
    if (nb < 1) nb = 1;
    k_dot<<<nb, 256, 0, s>>>(a, b, n, part);
    note_launch();
    *nparts = nb;
    return cudaGetLastError();
}

template <typename F>
static void allow_big_smem(F* kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void configure_kernels() {
    configure_tiles<float>();
    configure_tiles<double>();
    // per-cell kernels of high degrees (one cell's coefficients and Gauss values)
    allow_big_smem(k_eval);
    allow_big_smem(k_project);
    // tiled u-row kernels (stencil tile + staged value boxes) and cell operators
    allow_big_smem(k_urow<2, double, double, double, true, true, true>);
    allow_big_smem(k_urow<3, double, double, double, true, true, true>);
    allow_big_smem(k_urow<2, double, double, double, false, true, false>);
    allow_big_smem(k_urow<3, double, double, double, false, true, false>);
    allow_big_smem(k_urow<2, double, double, double, true, false, false>);
    allow_big_smem(k_urow<3, double, double, double, true, false, false>);
    allow_big_smem(k_ainv_blocks);
    allow_big_smem(k_cells_solve);
    allow_big_smem(k_stars_solve);
    allow_big_smem(k_urow<2, float, float, float, false, true, false>);
    allow_big_smem(k_urow<3, float, float, float, false, true, false>);
    allow_big_smem(k_urow<2, float, float, double, false, true, false>);
    allow_big_smem(k_urow<3, float, float, double, false, true, false>);
    allow_big_smem(k_cellop<2, double, double, double, double>);
    allow_big_smem(k_cellop<3, double, double, double, double>);
    allow_big_smem(k_cellop<2, float, float, float, double>);
    allow_big_smem(k_cellop<3, float, float, float, double>);
    allow_big_smem(k_cellop<2, float, float, float, float>);
    allow_big_smem(k_cellop<3, float, float, float, float>);
    cudaFuncSetAttribute(k_gemm_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
    cudaFuncSetAttribute(k_gemm_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
    cudaFuncSetAttribute(k_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor_warp<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor_warp<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor_warp<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor_warp<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);
    cudaFuncSetAttribute(k_factor_warp<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmemMax);

    cudaFuncSetAttribute(k_gm_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_newton_fused<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_newton_fused<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// ---- SIMT FMA throughput probe ------------------------------------------------
// Eight independent FMA chains per thread (enough to cover the pipe latency with
// 8 warps per SM scheduler), x <- x * a + b with |a| < 1 so nothing overflows; the
// sum is stored only under a condition that never holds, which keeps the chains live.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    T sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += x[k];
    if (sum == (T)-12345.0) out[0] = sum;
}

cudaError_t measure_fma_peak(int elem, int sm_count, cudaStream_t s, double* tflops) {
    const int blocks = sm_count * 8, threads = 256;
    const int iters = elem == 4 ? 32768 : 1024;
    void* out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, 16, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        if (elem == 4) k_fma_peak<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-6f);
        else k_fma_peak<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-6);
        note_launch();
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.f) best = std::min(best, ms);     // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaStreamSynchronize(s);
}

// ============================================================ instantiations
template cudaError_t launch_factor<double>(const Geo<double>&, const double*, double, double, double*, double*,
                                           int*, double*, cudaStream_t, const Bat&);
template cudaError_t launch_factor<float>(const Geo<float>&, const float*, double, double, float*, double*, int*,
                                          float*, cudaStream_t, const Bat&);
template cudaError_t launch_precond<double, double, double>(const Geo<double>&, const double*, const double*,
                                                            double*, cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_precond<float, float, float>(const Geo<float>&, const float*, const float*, float*,
                                                         cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_precond<float, double, float>(const Geo<float>&, const float*, const double*, float*,
                                                          cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_precond<float, double, double>(const Geo<float>&, const float*, const double*,
                                                           double*, cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_bapply<double, double, double>(const Geo<double>&, const double*, double*, cudaStream_t,
                                                           const int*, const Bat&);
template cudaError_t launch_bapply<float, float, float>(const Geo<float>&, const float*, float*, cudaStream_t,
                                                        const int*, const Bat&);
template cudaError_t launch_bapply<float, double, float>(const Geo<float>&, const double*, float*, cudaStream_t,
                                                         const int*, const Bat&);
template cudaError_t launch_btapply<double, double, double>(const Geo<double>&, const double*, double*,
                                                            cudaStream_t, const Bat&);
template cudaError_t launch_btapply<float, float, float>(const Geo<float>&, const float*, float*, cudaStream_t,
                                                         const Bat&);
template cudaError_t launch_fdm<double>(const Geo<double>&, const double*, double, const double*, double*, double*,
                                        double*, cudaStream_t, const int*, const Bat&, double);
template cudaError_t launch_fdm<float>(const Geo<float>&, const double*, double, const float*, float*, float*,
                                       float*, cudaStream_t, const int*, const Bat&, double);
template cudaError_t launch_schur_rest<double, double>(const Geo<double>&, const double*, double, const double*,
                                                       const double*, double*, cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_schur_rest<float, float>(const Geo<float>&, const float*, double, const float*,
                                                    const float*, float*, cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_schur_rest<float, double>(const Geo<float>&, const float*, double, const float*,
                                                      const float*, double*, cudaStream_t, IterCtl, const Bat&);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t, const Bat&);
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t, const Bat&);
template cudaError_t launch_sub_scaled<double>(const double*, double, const double*, double*, long long,
                                               cudaStream_t, const Bat&);
template cudaError_t launch_sub_scaled<float>(const double*, double, const float*, double*, long long,
                                              cudaStream_t, const Bat&);
template cudaError_t launch_copy<double>(const double*, double*, long long, cudaStream_t, const Bat&);
template cudaError_t launch_copy<float>(const float*, float*, long long, cudaStream_t, const Bat&);
template cudaError_t launch_copy<int>(const int*, int*, long long, cudaStream_t, const Bat&);

}  // namespace hpg
