// A_alpha^{-1} by fast diagonalisation (Section 4.4's inverse, applied as the tensor
// product of the 1D generalised eigenvectors) on the 5th-generation tensor cores, fed
// by the Tensor Memory Accelerator.
//
// Each of the 2d passes contracts one axis with a dense n1 x n1 matrix (V^T forward,
// V backward).  A pass is the GEMM  D[r][a] = sum_k X[r][k] W[a][k]  where k runs over
// the contracted axis (the fastest of the pass's input layout) and r over the others.
// The output is written with a as its slowest index, so the next axis becomes the
// fastest: after d passes the axes are back in their natural order (2D: [i1][i0] ->
// [a0][i1] -> [a1][a0]).  Between passes the tensors live in a workspace in "sliced"
// form, [k / 4][r][k % 4] (16-byte slices of four consecutive k, zero-padded, rows padded
// to the 128-row tile), split into a TF32-exact high part (the FP32 value with its 13 low
// mantissa bits cleared) and the FP32 remainder.  That layout is a plain 3D tensor for
// TMA whose box lands in shared memory as the no-swizzle K-major core-matrix layout of
// tcgen05.mma, so every operand tile is one bulk tensor copy (runs of 1 KB).
//
// Per CTA (128 threads): warp 0 issues the TMA loads of a ring of stages (A high and
// remainder: 128 rows, B high and remainder: the pass's matrix; 16 k each), warp 1 issues
// the MMAs (kind::tf32, M = 128, N = BN, K = 8; three products per step: hi*hi + hi*lo +
// lo*hi, FP32 accumulation in TMEM) and commits each stage back to the producer; then
// all four warps read the accumulator with tcgen05.ld and write the next pass's sliced
// parts (the last forward pass scales by 1 / (alpha (sum of eigenvalues + shift)); the
// last backward pass writes the natural FP32 output).  Every
// mbarrier wait is a bounded spin; on time-out the tile is written as NaN (which the
// solver's finiteness checks report), in-flight copies and products are waited for once
// more (bounded) and TMEM is released.
#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "device.h"

namespace hpg {

namespace {

constexpr int kTBM = 128;      // rows per CTA tile (the MMA's M)
constexpr int kTBK = 16;       // k per stage (4 slices)
constexpr int kTNS = 8;        // most stages in the ring (as many as fit 192 KB)
constexpr int kTSl = kTBK / 4; // slices per stage
constexpr int kTRbA = 64;      // rows per innermost TMA run of the A operand (1 KB runs)

struct TmaPassArgs {
    const CUtensorMap* mA;     // input maps of problem 0 (high at +0, remainder at +1); problem pb at + pb * mA_stride
    int mA_stride;
    const CUtensorMap* mBh;    // the pass's matrix, high and remainder parts
    const CUtensorMap* mBl;
    int M, N, nch;             // rows, columns (n1 of the axis), stages of k
    int BN, tcols;             // N tile (= the B box's rows), TMEM columns
    int rb;                    // rows per innermost TMA run of the B tile
    int ns;                    // stages in the ring (<= kTNS)
    int lbo_a, lbo_b;          // bytes between k-adjacent core matrices in shared memory
    int mode;                  // 0: sliced out, 1: the same scaled by the eigenvalues, 2: natural FP32 out
    float* ohi;                // sliced output parts of problem 0 (problem pb at + pb * ws_stride floats)
    float* olo;
    long long ws_stride;
    int F;                     // fastest extent of the output layout
    long long Rn;              // rows of the output layout (padded to a multiple of the M tile)
    float* y;                  // natural output of problem 0 (mode 2; other problems by Bat byte offsets)
    const float* lam[kMaxDim];
    int d, n1[kMaxDim];
    double shift;
    const double* alpha_dev;
    double alpha_host;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory descriptor: start, leading (k-direction) and stride (8-row
// direction) byte offsets, no swizzle, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Bounded spin on an mbarrier phase with the non-blocking test (a suspended try_wait
// wakes up late: each hand-off between the producer and the MMA warp then costs
// microseconds); about 0.1 s at most.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
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

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// TF32-exact high part (13 low mantissa bits cleared) and the exact FP32 remainder
__device__ __forceinline__ void split_hl(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

__global__ void __launch_bounds__(128, 1) k_fdm_tma(TmaPassArgs p, const int* skip, Bat bt) {
    extern __shared__ unsigned char tsm_raw[];
    __shared__ __align__(8) uint64_t full[kTNS];
    __shared__ __align__(8) uint64_t empty[kTNS];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tbase;
    __shared__ int s_fail, s_issued, s_consumed;
    const int pb = (int)blockIdx.z;
    long long off;
    if (!bat_enter(bt, pb, &off)) return;
    skip = bsh(skip, off);
    if (skip && *skip) return;
    const double* adev = bsh(p.alpha_dev, off);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int BN = p.BN, NS = p.ns;
    // stage: [A high][A remainder][B high][B remainder], each a TMA box
    const uint32_t a_bytes = kTBM * kTBK * 4, b_bytes = (uint32_t)BN * kTBK * 4;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    const uint32_t st0 = (saddr(tsm_raw) + 1023u) & ~1023u;
    const int m0 = (int)blockIdx.y * kTBM, n0 = (int)blockIdx.x * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tbase)),
                     "r"(p.tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const CUtensorMap* mAh = p.mA + (size_t)pb * p.mA_stride;
    const CUtensorMap* mAl = mAh + 1;
    if (warp == 0 && lane == 0) {
        // producer: one bulk tensor copy per operand part and stage
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mAh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mAl)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(p.mBh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(p.mBl)) : "memory");
        int c = 0;
        for (; c < p.nch; ++c) {
            const int s = c % NS;
            if (c >= NS && !bar_wait(saddr(&empty[s]), (uint32_t)(((c / NS) - 1) & 1))) {
                atomicExch(&s_fail, 1);
                break;
            }
            const uint32_t sb = st0 + (uint32_t)s * stage_bytes;
            const uint32_t fb = saddr(&full[s]);
            bar_expect_tx(fb, stage_bytes);
            tma_load3(sb, mAh, 0, m0 / kTRbA, c * kTSl, fb);
            tma_load3(sb + a_bytes, mAl, 0, m0 / kTRbA, c * kTSl, fb);
            tma_load3(sb + 2 * a_bytes, p.mBh, 0, n0 / p.rb, c * kTSl, fb);
            tma_load3(sb + 2 * a_bytes + b_bytes, p.mBl, 0, n0 / p.rb, c * kTSl, fb);
        }
        atomicExch(&s_issued, c);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: kind::tf32, A and B K-major, D in FP32 (TMEM)
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(kTBM >> 4) << 24);
        int c = 0;
        for (; c < p.nch; ++c) {
            const int s = c % NS;
            if (!bar_wait(saddr(&full[s]), (uint32_t)((c / NS) & 1))) {
                atomicExch(&s_fail, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sb = st0 + (uint32_t)s * stage_bytes;
            const uint32_t ah = sb, al = sb + a_bytes, bh = sb + 2 * a_bytes, bl = bh + b_bytes;
#pragma unroll
            for (int kk = 0; kk < kTBK / 8; ++kk) {
                const uint32_t oa = (uint32_t)kk * 2 * (uint32_t)p.lbo_a, ob = (uint32_t)kk * 2 * (uint32_t)p.lbo_b;
                const uint64_t dah = sdesc(ah + oa, p.lbo_a, 128), dal = sdesc(al + oa, p.lbo_a, 128);
                const uint64_t dbh = sdesc(bh + ob, p.lbo_b, 128), dbl = sdesc(bl + ob, p.lbo_b, 128);
                mma_tf32(tmem, dah, dbh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            mma_commit(saddr(&empty[s]));
        }
        atomicExch(&s_consumed, c);
        mma_commit(saddr(&done));   // completes when every product issued above has landed
    }
    __syncwarp();
    bool ok = bar_wait(saddr(&done), 0);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool good = __syncthreads_and(ok && *((volatile int*)&s_fail) == 0) != 0;
    // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile in its TMEM lanes
    const int r = m0 + warp * 32 + lane;
    const bool rok = r < p.M;
    float ainv = 1.0f, part = 0.0f;
    if (p.mode == 1) {
        ainv = (float)(1.0 / (adev ? *adev : p.alpha_host));
        // the rows of the last forward pass are (a_{d-2}, ..., a_0), a_0 fastest
        long long t = rok ? r : 0;
        for (int i = 0; i + 1 < p.d; ++i) {
            part += p.lam[i][t % p.n1[i]];
            t /= p.n1[i];
        }
        part += (float)p.shift;
    }
    float* ohi = p.ohi + (size_t)pb * p.ws_stride;
    float* olo = p.olo + (size_t)pb * p.ws_stride;
    float* y = bsh(p.y, off);
    // the next pass's sliced parts (or, on the last pass, the natural output): consecutive
    // lanes write consecutive rows of one column; after a timed-out wait every row of the
    // tile is written as NaN (no TMEM read)
    const long long MF = p.mode != 2 ? (long long)p.M / p.F : 0;
    const int rf = (p.mode != 2 && rok) ? r % p.F : 0;
    const long long rq = (p.mode != 2 && rok) ? r / p.F : 0;
    for (int j0 = 0; j0 < BN; j0 += 16) {
        uint32_t v[16];
        if (good) {
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = 0x7fc00000u;
        }
        if (!rok) continue;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int n = n0 + j0 + jj;
            if (n >= p.N) break;
            float val = __uint_as_float(v[jj]);
            if (p.mode == 2) {
                y[(long long)n * p.M + r] = val;
                continue;
            }
            if (p.mode == 1) val = val * ainv / (part + p.lam[p.d - 1][n]);
            const long long addr = ((long long)(rf >> 2) * p.Rn + (long long)n * MF + rq) * 4 + (rf & 3);
            float h, l;
            split_hl(val, h, l);
            ohi[addr] = h;
            olo[addr] = l;
        }
    }
    if (!good && tid == 0) {
        // one more bounded wait for copies and products still in flight
        bar_wait(saddr(&done), 0);
        const int is = *((volatile int*)&s_issued), cs = *((volatile int*)&s_consumed);
        for (int c = cs; c < is; ++c) bar_wait(saddr(&full[c % NS]), (uint32_t)((c / NS) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tcols));
}

// natural FP32 input -> sliced hi/lo parts of workspace buffer 0 (layout of the pass along axis 0)
__global__ void k_fdm_tma_split(const float* __restrict__ x, float* ws, long long ws_stride, long long wsz, int n10,
                                long long Rp0, long long total, const int* skip, Bat bt) {
    const int pb = (int)blockIdx.y;
    long long off;
    if (!bat_enter(bt, pb, &off)) return;
    skip = bsh(skip, off);
    if (skip && *skip) return;
    x = bsh(x, off);
    float* hi = ws + (size_t)pb * ws_stride;
    float* lo = hi + wsz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % n10);
        const long long q = i / n10;
        const long long addr = ((long long)(f >> 2) * Rp0 + q) * 4 + (f & 3);
        float h, l;
        split_hl(x[i], h, l);
        hi[addr] = h;
        lo[addr] = l;
    }
}

// N tile of a variant: 64, 128 or 256 columns (at most n1 rounded up to 16), or 32 (variant 3:
// more, smaller CTAs)
int tma_bn(int variant, int n1) {
    const int r16 = (n1 + 15) / 16 * 16;
    if (variant == 3) return std::min(32, r16);
    if (r16 <= 64) return r16;
    const int cap = variant == 0 ? 64 : (variant == 1 ? 128 : 256);
    const int r64 = (n1 + 63) / 64 * 64;
    return std::min(cap, r64);
}

// rows per innermost TMA run of a B tile of bn rows (a divisor of bn and of the padded rows)
int tma_rb(int bn) { return bn % 64 == 0 ? 64 : 16; }

int pow2_cols(int bn) {
    int c = 32;
    while (c < bn) c <<= 1;
    return c;
}

size_t tma_stage_bytes(int bn) { return 2 * (size_t)kTBM * kTBK * 4 + 2 * (size_t)bn * kTBK * 4; }
// stages in about 96 KB (two CTAs per SM), at least 2 and at most kTNS
int tma_stages(int bn) {
    return (int)std::max<size_t>(2, std::min<size_t>(kTNS, (96 * 1024) / tma_stage_bytes(bn)));
}
size_t tma_smem(int bn) { return 1024 + (size_t)tma_stages(bn) * tma_stage_bytes(bn); }

}  // namespace

int fdm_tma_variants() { return 4; }

cudaError_t launch_fdm_tma(const FdmTma& t, int variant, const double* alpha_dev, double alpha, const float* x,
                           float* y, cudaStream_t s, const int* skip, const Bat& bt, double shift) {
    if (!t.ready || t.np != bt.np || variant < 0 || variant >= fdm_tma_variants()) return cudaErrorInvalidValue;
    const int d = t.d;
    {
        const long long total = t.R[0] * t.n1[0];
        const unsigned gx = (unsigned)std::min<long long>((total + 255) / 256, 2048);
        k_fdm_tma_split<<<dim3(gx, (unsigned)bt.np), 256, 0, s>>>(x, t.ws, 4 * t.wsz, t.wsz, t.n1[0], t.Rp[0], total,
                                                                  skip, bt);
        note_kernel_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const CUtensorMap* mA = static_cast<const CUtensorMap*>(t.mA);
    const CUtensorMap* mB = static_cast<const CUtensorMap*>(t.mB);
    for (int pass = 0; pass < 2 * d; ++pass) {
        const int ax = pass % d, fb = pass < d ? 0 : 1, in = pass % 2, out = 1 - in;
        TmaPassArgs a{};
        a.mA = mA + (size_t)((ax * 2 + in) * 2);
        a.mA_stride = 4 * d;
        a.mBh = mB + (size_t)(((variant * d + ax) * 2 + fb) * 2);
        a.mBl = a.mBh + 1;
        a.M = (int)t.R[ax];
        a.N = t.n1[ax];
        a.nch = t.Cp[ax] / kTSl;
        a.BN = tma_bn(variant, t.n1[ax]);
        a.tcols = pow2_cols(a.BN);
        a.rb = tma_rb(a.BN);
        a.ns = tma_stages(a.BN);
        a.lbo_a = kTBM * 16;
        a.lbo_b = a.BN * 16;
        a.mode = pass == 2 * d - 1 ? 2 : (pass == d - 1 ? 1 : 0);
        a.ohi = t.ws + (size_t)out * 2 * t.wsz;
        a.olo = a.ohi + t.wsz;
        a.ws_stride = 4 * t.wsz;
        a.F = t.n1[(ax + 1) % d];
        a.Rn = t.Rp[(ax + 1) % d];
        a.y = y;
        for (int j = 0; j < kMaxDim; ++j) {
            a.lam[j] = t.lam[j];
            a.n1[j] = t.n1[j];
        }
        a.d = d;
        a.shift = shift;
        a.alpha_dev = alpha_dev;
        a.alpha_host = alpha;
        dim3 grid((unsigned)((a.N + a.BN - 1) / a.BN), (unsigned)((a.M + kTBM - 1) / kTBM), (unsigned)bt.np);
        k_fdm_tma<<<grid, 128, tma_smem(a.BN), s>>>(a, skip, bt);
        note_kernel_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------ host set-up
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// a sliced tensor [slices][rows][4] floats at base, described with rb rows per innermost
// element run (4 rb floats, rb a divisor of rows and of box_rows) so that TMA moves
// runs of 16 rb bytes; box {4 rb, box_rows / rb, kTSl}.  The box lands in shared memory
// as [slice][box_rows][4], the same bytes as with 16-byte runs.
bool encode_sliced(CUtensorMap* m, const float* base, long long rows, int slices, int box_rows, int rb) {
    EncodeTiledFn f = encode_fn();
    if (!f || rows % rb != 0 || box_rows % rb != 0) return false;
    cuuint64_t dims[3] = {(cuuint64_t)(4 * rb), (cuuint64_t)(rows / rb), (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)rb * 16, (cuuint64_t)rows * 16};
    cuuint32_t box[3] = {(cuuint32_t)(4 * rb), (cuuint32_t)(box_rows / rb), (cuuint32_t)kTSl};
    cuuint32_t es[3] = {1, 1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool fdm_tma_setup(FdmTma& t, const HostProblem& H, const float* const* lam, int np,
                   const std::function<void*(size_t)>& alloc, cudaStream_t s, const FdmTma* consts, std::string* why) {
    t = FdmTma{};
    const int d = H.d;
    t.d = d;
    t.np = np;
    long long tot = 1;
    for (int j = 0; j < d; ++j) {
        t.n1[j] = H.dir[j].n1;
        tot *= t.n1[j];
    }
    t.wsz = 0;
    for (int j = 0; j < d; ++j) {
        t.R[j] = tot / t.n1[j];
        t.Rp[j] = (t.R[j] + kTBM - 1) / kTBM * kTBM;          // rows padded to the M tile
        t.C[j] = (t.n1[j] + 3) / 4;
        t.Cp[j] = (t.C[j] + kTSl - 1) / kTSl * kTSl;          // slices padded to the stage depth
        t.wsz = std::max<long long>(t.wsz, 4LL * t.Cp[j] * t.Rp[j]);
        t.lam[j] = lam[j];
    }
    t.wsz = (t.wsz + 63) / 64 * 64;    // 256-byte aligned buffers
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_fdm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem(256));
    if (attr != cudaSuccess) {
        if (why) *why = "shared-memory opt-in refused";
        return false;
    }
    if (!encode_fn()) {
        if (why) *why = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    // the pass matrices: sliced high parts and remainders of V^T (forward) and V (backward),
    // rows padded so that every variant's N tile is one in-bounds box; shared by a group
    if (consts) {
        t.mB = consts->mB;
    } else {
        const int nv = fdm_tma_variants();
        std::vector<CUtensorMap> mb((size_t)nv * d * 4);
        for (int j = 0; j < d; ++j) {
            const int n = t.n1[j], Cp = t.Cp[j];
            const int np_rows = (n + 255) / 256 * 256;   // a multiple of every variant's N tile
            const std::vector<double>& V = H.dir[j].V;   // row-major V[k][a]
            for (int fb = 0; fb < 2; ++fb) {
                std::vector<float> hi((size_t)Cp * np_rows * 4, 0.0f), lo((size_t)Cp * np_rows * 4, 0.0f);
                for (int row = 0; row < n; ++row)
                    for (int k = 0; k < n; ++k) {
                        // forward W[a][k] = V[k][a]; backward W[a][k] = V[a][k]
                        const float x = (float)(fb == 0 ? V[(size_t)k * n + row] : V[(size_t)row * n + k]);
                        uint32_t bits;
                        std::memcpy(&bits, &x, 4);
                        bits &= 0xFFFFE000u;
                        float h;
                        std::memcpy(&h, &bits, 4);
                        const size_t at = ((size_t)(k >> 2) * np_rows + row) * 4 + (k & 3);
                        hi[at] = h;
                        lo[at] = x - h;
                    }
                float* dh = static_cast<float*>(alloc(hi.size() * sizeof(float)));
                float* dl = static_cast<float*>(alloc(lo.size() * sizeof(float)));
                if (!dh || !dl) {
                    if (why) *why = "device allocation failed";
                    return false;
                }
                cudaMemcpyAsync(dh, hi.data(), hi.size() * sizeof(float), cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(dl, lo.data(), lo.size() * sizeof(float), cudaMemcpyHostToDevice, s);
                cudaStreamSynchronize(s);
                for (int v = 0; v < nv; ++v) {
                    const int bn = tma_bn(v, n), rb = tma_rb(bn);
                    if (!encode_sliced(&mb[(size_t)(((v * d + j) * 2 + fb) * 2) + 0], dh, np_rows, Cp, bn, rb) ||
                        !encode_sliced(&mb[(size_t)(((v * d + j) * 2 + fb) * 2) + 1], dl, np_rows, Cp, bn, rb)) {
                        if (why) *why = "tensor map of a pass matrix rejected";
                        return false;
                    }
                }
            }
        }
        void* dmb = alloc(mb.size() * sizeof(CUtensorMap));
        if (!dmb) {
            if (why) *why = "device allocation failed";
            return false;
        }
        cudaMemcpyAsync(dmb, mb.data(), mb.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s);
        t.mB = dmb;
    }
    // workspace: np x [buffer 0 high, remainder, buffer 1 high, remainder], zeroed once (the
    // padding of the last slice of every row is never written)
    t.ws = static_cast<float*>(alloc((size_t)np * 4 * t.wsz * sizeof(float)));
    if (!t.ws) {
        if (why) *why = "device allocation failed";
        return false;
    }
    cudaMemsetAsync(t.ws, 0, (size_t)np * 4 * t.wsz * sizeof(float), s);
    std::vector<CUtensorMap> ma((size_t)np * d * 4);
    for (int pb = 0; pb < np; ++pb)
        for (int j = 0; j < d; ++j)
            for (int b = 0; b < 2; ++b)
                for (int hl = 0; hl < 2; ++hl) {
                    const float* base = t.ws + ((size_t)pb * 4 + (size_t)b * 2 + hl) * t.wsz;
                    if (!encode_sliced(&ma[(size_t)pb * d * 4 + (size_t)(j * 2 + b) * 2 + hl], base, t.Rp[j],
                                       t.Cp[j], kTBM, kTRbA)) {
                        if (why) *why = "tensor map of the workspace rejected";
                        return false;
                    }
                }
    void* dma = alloc(ma.size() * sizeof(CUtensorMap));
    if (!dma) {
        if (why) *why = "device allocation failed";
        return false;
    }
    cudaMemcpyAsync(dma, ma.data(), ma.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s);
    t.mA = dma;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        if (why) *why = "upload failed";
        return false;
    }
    t.ready = true;
    return true;
}

}  // namespace hpg
