// KZ: the 2D matvec on the tcgen05 tensor cores with an FP64-class result, by the Ozaki scheme
// (error-free splitting of both factors into fixed-point digit slices whose products and short
// sums are exact in the tensor core's FP32 accumulator: Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 59 (2012); on tensor cores: Mukunoki, Ozaki, Ogita and Imamura, ICCS 2020).
//
// Structure used.  On the uniform n x n grid (point i = i1 n + i2) the off-diagonal entry of A
// depends only on the lattice offsets through the per-offset table, A_ij = t(|i1 - j1|, |i2 - j2|)
// (Eq. e:a_2d; t(0, 0) is the diagonal, added separately in FP64).  With d1 = i1 - j1,
//     y[i1][i2] = sum_d1 sum_j2 T_d1[i2][j2] x[i1 - d1][j2],   T_d1[i2][j2] = t(|d1|, |i2 - j2|),
// so for each d1 the product is a GEMM of the Toeplitz matrix T_d1 with the grid rows shifted by
// d1: a dense contraction with K = n per d1 and 2n - 1 values of d1.
//
// Digits.  Both factors are scaled by a power of two (sigma_t = 2^ceil(log2 max |t|), sigma_x the
// same for x) and cut into D = 6 signed integer digits, v / sigma = d_0 2^-7 + d_1 2^-16 + ... +
// d_5 2^-52 (|d_0| <= 128, |d_k| <= 256 for k >= 1), each exactly a BF16 number.  The product is
// the sum over digit pairs (a, b) with a + b <= 5 (21 pairs) at level a + b; pairs of one level
// share one FP32 accumulator.  Over a window of 128 source columns the level-0 and level-1 sums
// are integers below 2^21 and 2^23, so the tensor core adds them exactly, and level 2 stays below
// 2^24; levels 3-5 are integers in their own units too (their sums stay below 2^24 for any input
// whose digits are not all of one sign and maximal).  After each window the six accumulators are
// read and added into a 64-bit integer per output in units of 2^-F of a level-0 product: levels
// 0-2 exactly, each of levels 3-5 rounded to the unit.  F is the largest value for which no sum
// can overflow: every output is at most 2^14 (sum_j |t_ij|) / sigma_t level-0 units, and that row
// sum is bounded once per problem from the table (F is 34 at 128^2, 30 at 512^2, 29 at 1024^2).  The
// result differs from the exact product by the dropped pairs, the last-digit truncation and one
// rounding of each of levels 3-5 to 2^-F per window: ~1e-17 of sum |A_ij x_j|.
//
// Tile.  A CTA owns 128 target points of one grid line segment (M = 128 values of i2) for 32
// consecutive lines (i1), one block of 128 source columns j2, and a range of d1.  Per d1 (one
// window) it
//   * loads the A operand with one TMA tensor copy: the six digit planes of a 248-row strip of the
//     window table (built once per problem; row p holds 8 consecutive table values along the
//     Toeplitz diagonal), which the MMAs of all 8 K-steps read through shifted shared-memory
//     descriptors (MMA row m is target i2_0 + 127 - m, so the tile entry depends on m + k);
//   * loads the B operand (the six digit planes of the 32 source rows i1 - d1 over the 128
//     columns, pre-split once per matvec) with one TMA tensor copy (3D map: runs of 32 rows x 8
//     values x planes x column groups, which lands directly in the canonical K-major layout);
//   * issues, per K-step, one MMA per A digit a with the B digit planes 0..5-a side by side
//     (N = 32 (6 - a)) into TMEM columns from level a on: digit pair (a, b) lands in level a + b.
// Operands are triple-buffered and the TMEM accumulators double-buffered (2 x 192 columns):
// later windows' operands land and window w - 1's accumulators are read while window w's MMAs run.
// Waits are bounded: a CTA that waits too long records an error code, drains, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "iedd_internal.cuh"

namespace {

constexpr int kZM = 128;                     // i2 per tile (MMA M)
constexpr int kZC = 32;                      // grid lines i1 per tile (N per digit plane)
constexpr int kZK = 128;                     // source columns j2 per window (8 K-steps of 16)
constexpr int kZD = 6;                       // digits per factor
constexpr int kZWin = kZK + kZM - 8;        // strip rows (window-table rows per window): 248
constexpr int kZStages = 3;                  // operand stages
constexpr int kTopBits = 7, kDigBits = 9;
constexpr uint32_t kStripPlane = kZWin * 16u;                  // bytes per digit plane (3968)
constexpr uint32_t kStripBytes = kZD * kStripPlane;            // 23808
constexpr uint32_t kBRows = kZD * kZC;                         // B rows: 6 planes x 32 lines
constexpr uint32_t kBGroup = kBRows * 16u;                     // bytes per 8-column group (3072)
constexpr uint32_t kBBytes = (kZK / 8) * kBGroup;              // 49152
constexpr uint32_t kStageBytes = kStripBytes + kBBytes;        // 72960 (a multiple of 128)
constexpr int kZSmem = kZStages * (int)kStageBytes;            // 218880
constexpr long long kSpinLimit = 1LL << 24;
constexpr int kZMinF = 2 * kDigBits;         // levels 0-2 need units down to 2^-18

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; base offset 0, no swizzle
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kZM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase), "r"(1000u)
        : "memory");
    return ok != 0;
}

// non-blocking probe: one shared-memory round trip, cheaper than try_wait on a phase that has
// already completed
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (long long i = 0; i < kSpinLimit / 8; ++i)
        if (mbar_try(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// the six digits of v in [-1, 1] (exact FP64 steps: scalings by powers of two, rint, subtraction)
__device__ __forceinline__ void digits6(double v, float (&d)[kZD]) {
    double w = v * (double)(1 << kTopBits);
#pragma unroll
    for (int k = 0; k < kZD; ++k) {
        const double r = rint(w);
        d[k] = (float)r;
        w = (w - r) * (double)(1 << kDigBits);
    }
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {  // exact: |v| <= 256 is an integer
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// power-of-two scale sigma >= max |v| from the bits of max |v| (a non-negative double)
__device__ __forceinline__ double scale_of(unsigned long long maxbits) {
    const double m = __longlong_as_double((long long)maxbits);
    if (!(m > 0.0)) return 1.0;
    int e;
    frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
    return ldexp(1.0, e);
}

__global__ void absmax_kernel(const double *__restrict__ v, long long count, unsigned long long *__restrict__ out) {
    double m = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// An upper bound of max_i sum_{j != i} |A_ij| from the per-offset table: sum over the offsets
// (d1, d2) != 0 of |t(d1, d2)| times the number of sign combinations (at most 4).  One CTA, a
// fixed summation order (deterministic).
__global__ void __launch_bounds__(1024) rowsum_bound_kernel(const double *__restrict__ t64, int n, double *__restrict__ out) {
    __shared__ double sh[32];
    const long long T = (long long)n * n;
    double s = 0.0;
    for (long long q = threadIdx.x; q < T; q += blockDim.x) {
        const int d1 = (int)(q % n), d2 = (int)(q / n);
        if (q != 0) s += fabs(t64[q]) * ((d1 > 0 ? 2.0 : 1.0) * (d2 > 0 ? 2.0 : 1.0));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) out[0] = t;
    }
}

// Window table of the A operand.  With v_d(p) = t(d, |n - 1 - p|) (0 outside the table and at
// t(0, 0), the diagonal), row p of plane a for offset d holds digit a of v_d(p), ..., v_d(p + 7):
// out[(d D + a) 2n + p] (16 bytes), p < 2n.  A run of 248 consecutive rows is the Toeplitz strip of
// one window (see kz_matvec_tc), so a window's A operand is one TMA copy.  One thread per (d, p).
__global__ void window_table_kernel(const double *__restrict__ t64, int n, const unsigned long long *__restrict__ maxbits,
                                    uint4 *__restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = 2 * n;
    if (e >= (long long)n * rows) return;
    const int d = (int)(e / rows), p = (int)(e % rows);
    const double sig = scale_of(*maxbits);
    uint32_t w[kZD][4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        float d0[kZD], d1[kZD];
        const int q0 = abs(n - 1 - (p + k)), q1 = abs(n - 1 - (p + k + 1));
        const long long e0 = (long long)d * n + q0, e1 = (long long)d * n + q1;
        digits6(q0 < n && e0 != 0 ? t64[e0] / sig : 0.0, d0);
        digits6(q1 < n && e1 != 0 ? t64[e1] / sig : 0.0, d1);
#pragma unroll
        for (int a = 0; a < kZD; ++a) w[a][k >> 1] = (uint32_t)bf16_bits(d0[a]) | ((uint32_t)bf16_bits(d1[a]) << 16);
    }
#pragma unroll
    for (int a = 0; a < kZD; ++a)
        out[((long long)d * kZD + a) * rows + p] = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
}

// x digits in the B-operand source layout: [8-column group][plane][row + 32][8 values], rows
// -32..n+31 (rows outside the grid are zero).  One thread per (row, group): six 16-byte chunks.
__global__ void x_digits_kernel(const double *__restrict__ x, int n, const unsigned long long *__restrict__ maxbits,
                                uint4 *__restrict__ out) {
    const int groups = n >> 3, rows = n + 64;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)groups * rows) return;
    const int g = (int)(e / rows), rr = (int)(e % rows), r = rr - 32;
    const double sig = scale_of(*maxbits);
    uint32_t w[kZD][4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        float d0[kZD], d1[kZD];
        const bool in = r >= 0 && r < n;
        digits6(in ? x[(long long)r * n + 8 * g + k] / sig : 0.0, d0);
        digits6(in ? x[(long long)r * n + 8 * g + k + 1] / sig : 0.0, d1);
#pragma unroll
        for (int a = 0; a < kZD; ++a) w[a][k >> 1] = (uint32_t)bf16_bits(d0[a]) | ((uint32_t)bf16_bits(d1[a]) << 16);
    }
#pragma unroll
    for (int a = 0; a < kZD; ++a) out[((long long)g * kZD + a) * rows + rr] = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
}

// One CTA: target points i2 in [128 bx, +128) of lines i1 in [32 by, +32), source columns
// j2 in [128 kb, +128), d1 in its share of [i1_0 - n + 1, i1_0 + 31].  Writes the CTA's integer
// partial sums (units 2^-F of a level-0 product) to part[z][i].
//
// MMA row m is target i2_0 + 127 - m, so that the A tile entry (m, k) of a window, t(|d1|,
// |i2_0 + 127 - kb - (m + k)|), depends on m + k alone and rises with both: the tile of K-step s
// is the window-table strip seen from row 16 s, and its second 8-column half is the same strip
// 8 rows further on (core-matrix strides of 128 bytes in both directions).
//
// Warp roles, handing over through mbarriers (no block-wide barrier inside the window loop):
//   warp 0      one lane issues a window's 48 MMAs once its operands are in place (full[stage])
//               and its accumulator set has been read (aempty[set]); commits them to
//               sfree[stage] and afull[set];
//   warp 1      one lane: once the stage is free (sfree), the two TMA copies of the window
//               (strip, B operand), completing full[stage] (expect_tx); copies run up to two
//               windows ahead;
//   warps 2-5   read a finished window's accumulator set (TMEM lane quarter warp & 3, all 32
//               lines), release it (aempty[set]) and add it into the 64-bit sums.
// Window w uses operand stage w % kZStages (its (w / kZStages)-th use, so waits take parity
// (w / kZStages) & 1) and accumulator set w & 1 (parity (w >> 1) & 1).  No barrier can run two
// phases ahead of a waiter (each role's next use waits for the consumer of the previous one).
// Every wait is bounded: a role that gives up sets the shared abort flag, which ends the other
// roles' waits.
__global__ void __launch_bounds__(192, 1)
kz_matvec_tc(const __grid_constant__ CUtensorMap wmap, const __grid_constant__ CUtensorMap xmap, int n, int dsplit,
             int F, long long *__restrict__ part, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char zsm[];  // kZStages x [strip | B]
    __shared__ __align__(8) uint64_t full[kZStages], sfree[kZStages], afull[2], aempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i2_0 = blockIdx.x * kZM, i1_0 = blockIdx.y * kZC;
    const int kb = (blockIdx.z / dsplit) * kZK, ds = blockIdx.z % dsplit;
    const long long N = (long long)n * n;
    const int dn = n + kZC - 1, per = (dn + dsplit - 1) / dsplit;
    const int d_begin = i1_0 - n + 1 + ds * per;
    const int T = max(0, min(per, dn - ds * per));
    const int R0 = n - kZM - i2_0 + kb;  // first window-table row of the strip, in [0, 2n - 256]

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < kZStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[st])), "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sfree[st])), "r"(1u));
        }
        for (int st = 0; st < 2; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull[st])), "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&aempty[st])), "r"(4u));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t smem0 = smem_u32(zsm);

    // bounded wait for a phase of a barrier; false (and the abort flag set) if it ran out or if
    // another role gave up
    auto wait_bar = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (mbar_test(smem_u32(bar), parity)) return true;
        for (long long i = 0; i < kSpinLimit / 8; ++i) {
            if (mbar_try(smem_u32(bar), parity)) return true;
            if (abort_flag) return false;
        }
        abort_flag = 1;
        return false;
    };
    // the same for a whole warp: lane 0 waits, the result is broadcast
    auto warp_wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        int ok = 1;
        if (lane == 0) ok = wait_bar(bar, parity) ? 1 : 0;
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    long long acc[32];  // warps 2-5: lines i1_0 + c (c < 32) at MMA row 32 (warp & 3) + lane
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0;

    if (warp == 0) {
        // ---- MMA issue (one lane) ----
        if (lane == 0) {
            uint32_t idesc[kZD];
#pragma unroll
            for (int a = 0; a < kZD; ++a) idesc[a] = idesc_bf16((kZD - a) * kZC);
            int issued = 0;
            for (int w = 0; w < T; ++w) {
                const int sb = w % kZStages, set = w & 1;
                if (!wait_bar(&full[sb], (uint32_t)(w / kZStages) & 1u)) break;
                if (w >= 2 && !wait_bar(&aempty[set], ((uint32_t)(w >> 1) & 1u) ^ 1u)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t strip = smem0 + sb * kStageBytes, bop = strip + kStripBytes;
                const uint64_t a0 = make_desc(strip, 128u, 128u), b0 = make_desc(bop, kBGroup, 128u);
                const uint32_t dt = tmem + set * 256u;
#pragma unroll 1
                for (int s = 0; s < kZK / 16; ++s) {
                    const uint64_t bd = b0 + (uint64_t)((2u * s * kBGroup) >> 4);
#pragma unroll
                    for (int a = 0; a < kZD; ++a) {
                        const uint64_t ad = a0 + (uint64_t)((a * kStripPlane + (uint32_t)s * 256u) >> 4);
                        mma_bf16(dt + (uint32_t)(a * kZC), ad, bd, idesc[a], (s > 0 || a > 0) ? 1u : 0u);
                    }
                }
                mma_commit(smem_u32(&sfree[sb]));
                mma_commit(smem_u32(&afull[set]));
                issued = w + 1;
            }
            // every MMA issued has completed before the accumulators are freed (commit tracks
            // all earlier MMAs of this thread); this wait ignores the abort flag (still bounded)
            if (issued > 0 && !mbar_wait(smem_u32(&afull[(issued - 1) & 1]), (uint32_t)((issued - 1) >> 1) & 1u))
                abort_flag = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- operands of a window: the strip (six planes of 248 window-table rows) and the B
        // operand (six digit planes of the 32 source lines over the 128 columns) ----
        int issued = 0;
        for (int w = 0; w < T; ++w) {
            const int sb = w % kZStages;
            if (w >= kZStages && !warp_wait(&sfree[sb], ((uint32_t)(w / kZStages) & 1u) ^ 1u)) break;
            if (lane == 0) {
                const uint32_t bar = smem_u32(&full[sb]), dst = smem0 + sb * kStageBytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageBytes)
                             : "memory");
                // strip: box (8 values, 248 rows, 6 planes) at (0, R0, |d1| x 6)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                    ::"r"(dst), "l"(reinterpret_cast<uint64_t>(&wmap)), "r"(0), "r"(R0), "r"(abs(d_begin + w) * kZD),
                    "r"(bar)
                    : "memory");
                // B: box (32 rows x 8 values, 6 planes, 16 groups) at ((first source row + 32) x 8,
                // 0, kb / 8): the padded rows keep every coordinate inside the tensor, and x is a
                // whole number of 16-byte rows
                const int r0 = i1_0 - (d_begin + w);  // first source line, in [-31, n - 1]
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                    ::"r"(dst + kStripBytes), "l"(reinterpret_cast<uint64_t>(&xmap)), "r"((r0 + 32) * 8), "r"(0),
                    "r"(kb >> 3), "r"(bar)
                    : "memory");
            }
            __syncwarp();
            issued = w + 1;
        }
        // no copy may still be landing when the CTA ends (waits that ignore the abort flag, bounded;
        // an earlier window's copies completed before its stage was reused)
        if (lane == 0)
            for (int w = max(0, issued - kZStages); w < issued; ++w)
                if (!mbar_wait(smem_u32(&full[w % kZStages]), (uint32_t)(w / kZStages) & 1u)) abort_flag = 1;
        __syncwarp();
    } else {
        // ---- accumulator reads and exact sums (TMEM lane quarter warp & 3, all 32 lines) ----
        const int q4 = warp & 3;
        const long long w1 = 1LL << (F - kDigBits);
        const long long w2 = 1LL << (F - 2 * kDigBits);
        // levels 3, 4, 5 are integers in units of 2^-27, 2^-36, 2^-45 of level 0.  Level 3 (< 2^25)
        // converts exactly to int32 and is shifted to units of 2^-F (rounded to the unit instead
        // when F < 27); levels 4 and 5 are joined in FP32 in level-4 units (a rounding of <= 2^-39
        // level-0 units, below the unit 2^-F for F <= 38), scaled by 2^(F - 36) and rounded to the
        // unit (|value| < 2^31 for F <= 36).  All conversions are 32-bit.
        const int sh3 = F - 3 * kDigBits;
        const float s3 = __int_as_float((127 + (sh3 < 0 ? sh3 : 0)) << 23);
        const float s4 = __int_as_float((127 + F - 4 * kDigBits) << 23);
        for (int w = 0; w < T; ++w) {
            const int set = w & 1;
            if (!warp_wait(&afull[set], (uint32_t)(w >> 1) & 1u)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = tmem + ((uint32_t)(32 * q4) << 16) + set * 256u;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const uint32_t cb = base + 16u * hh;
                uint32_t v3[16], v4[16], v5[16];
                tmem_ld16(cb + 3 * kZC, v3);
                tmem_ld16(cb + 4 * kZC, v4);
                tmem_ld16(cb + 5 * kZC, v5);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const long long l3 = (long long)__float2int_rn(__uint_as_float(v3[c]) * s3) << (sh3 > 0 ? sh3 : 0);
                    const int l45 = __float2int_rn(fmaf(__uint_as_float(v5[c]), 0x1p-9f, __uint_as_float(v4[c])) * s4);
                    acc[16 * hh + c] += l3 + l45;
                }
                uint32_t v0[16], v1[16], v2[16];
                tmem_ld16(cb + 0 * kZC, v0);
                tmem_ld16(cb + 1 * kZC, v1);
                tmem_ld16(cb + 2 * kZC, v2);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (hh == 1) {  // every read of this set is complete: release it to the MMA lane
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&aempty[set])) : "memory");
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int a0 = __float2int_rn(__uint_as_float(v0[c]));  // exact integers
                    const int a1 = __float2int_rn(__uint_as_float(v1[c]));
                    const int a2 = __float2int_rn(__uint_as_float(v2[c]));
                    const int wv = a0 * (1 << kDigBits) + a1;             // < 2^31
                    acc[16 * hh + c] += (long long)wv * w1 + (long long)a2 * w2;  // exact
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!abort_flag) {
        if (warp >= 2) {
            long long *outp = part + (long long)blockIdx.z * N;
            const int i2 = i2_0 + (kZM - 1) - (32 * (warp & 3) + lane);
#pragma unroll
            for (int c = 0; c < 32; ++c) outp[(long long)(i1_0 + c) * n + i2] = acc[c];
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
}

// y = diag x + (sum of the CTAs' integer partials) sigma_t sigma_x 2^-(14 + F)
__global__ void kz_combine_kernel(const long long *__restrict__ part, int nparts, long long N, const double *__restrict__ x,
                                  double *__restrict__ y, double diag, const unsigned long long *__restrict__ tmax,
                                  const unsigned long long *__restrict__ xmax, int F) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    long long s = 0;
    for (int z = 0; z < nparts; ++z) s += part[(long long)z * N + i];
    const double scale = ldexp(scale_of(*tmax) * scale_of(*xmax), -(2 * kTopBits + F));
    y[i] = fma(diag, x[i], (double)s * scale);
}

}  // namespace

// The exact tensor-core 2D matvec applies to n a multiple of 128 with n <= 4096 (F >= 24).
bool tc_exact_supported(const ie_problem *p) { return p->dim == 2 && p->n % kZM == 0 && p->n <= 4096; }

// d1 splits per (tile, column block): the smallest modelled time ceil(CTAs / SMs) x (windows + 2)
static int kz_dsplit(int n, int sms) {
    const long long base = (long long)(n / kZM) * (n / kZC) * (n / kZK);
    const int dn = n + kZC - 1;
    int best = 1;
    long long best_cost = -1;
    for (int ds = 1; ds <= 64 && ds <= dn; ++ds) {
        const long long waves = (base * ds + sms - 1) / sms;
        const long long cost = waves * ((dn + ds - 1) / ds + 2);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = ds; }
    }
    return best;
}

int prepare_tc_exact(const ie_problem *p_) {
    ie_problem *p = const_cast<ie_problem *>(p_);
    if (p->d_zt_win) return IE_OK;
    IE_TRY_CUDA(cudaFuncSetAttribute(kz_matvec_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kZSmem));
    const long long T = (long long)p->n * p->n;
    IE_TRY_CUDA(cudaMalloc(&p->d_zt_max, sizeof(unsigned long long)));
    IE_TRY_CUDA(cudaMemset(p->d_zt_max, 0, sizeof(unsigned long long)));
    // max |t| over the off-diagonal table entries (entry 0 is the diagonal)
    absmax_kernel<<<std::max(1, (int)std::min<long long>(1024, (T - 1 + 255) / 256)), 256>>>(p->d_table64 + 1, T - 1,
                                                                                          p->d_zt_max);
    IE_LAUNCHED();
    // window table: n offsets x 6 planes x 2n rows of 16 bytes (192 n^2 bytes)
    const long long rows = 2 * T;
    IE_TRY_CUDA(cudaMalloc(&p->d_zt_win, sizeof(uint4) * kZD * rows));
    window_table_kernel<<<(unsigned)((rows + 255) / 256), 256>>>(p->d_table64, p->n, p->d_zt_max,
                                                                 static_cast<uint4 *>(p->d_zt_win));
    IE_LAUNCHED();
    // fraction bits F of the int64 sums: every output is at most 2^14 S / sigma_t level-0 units
    // (S = the row-sum bound, |x| <= sigma_x), so F <= 62 - 14 - log2(S / sigma_t) keeps every sum,
    // partial or total, below 2^62; one bit of margin more, and at most 36 (the 32-bit conversion
    // of the joined levels 4-5 in the accumulator warps)
    double *d_s = nullptr;
    IE_TRY_CUDA(cudaMalloc(&d_s, sizeof(double)));
    rowsum_bound_kernel<<<1, 1024>>>(p->d_table64, p->n, d_s);
    IE_LAUNCHED();
    double S = 0.0;
    unsigned long long tmax_bits = 0;
    IE_TRY_CUDA(cudaMemcpy(&S, d_s, sizeof(double), cudaMemcpyDeviceToHost));
    IE_TRY_CUDA(cudaMemcpy(&tmax_bits, p->d_zt_max, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    cudaFree(d_s);
    double tmax = 0.0;
    std::memcpy(&tmax, &tmax_bits, sizeof(double));
    int e = 0;
    std::frexp(tmax, &e);
    const double sigma_t = std::ldexp(1.0, e);
    const double ratio = S > 0.0 && sigma_t > 0.0 ? S / sigma_t : 1.0;
    p->zt_F = std::max(kZMinF, std::min(36, (int)std::floor(48.0 - std::log2(ratio)) - 1));
    IE_TRY_CUDA(cudaDeviceSynchronize());
    return IE_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no libcuda link)
void *tensor_map_encode_fn() {
    static void *fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = f;
    }
    return fn;
}
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encode_fn());
}

int launch_matvec_tc_exact(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy, int nrhs,
                           cudaStream_t s) {
    if (!tc_exact_supported(p)) {
        ie_set_error("ie_matvec: the exact tensor-core matvec needs a 2D grid with n a multiple of 128, n <= 4096");
        return IE_ERR_ARG;
    }
    if (!p->d_zt_win) {
        ie_set_error("ie_matvec: the exact tensor-core matvec was not prepared for this problem");
        return IE_ERR_ARG;
    }
    const int n = p->n;
    const long long N = p->N;
    const int ds = kz_dsplit(n, p->sm_count);
    const int F = p->zt_F;
    const int nparts = (n / kZK) * ds;
    DevBuf xd, part, mx;
    IE_TRY(xd.alloc(sizeof(uint4) * (size_t)kZD * (n / 8) * (n + 64), s));
    IE_TRY(part.alloc(sizeof(long long) * (size_t)nparts * N, s));
    IE_TRY(mx.alloc(sizeof(unsigned long long), s));
    // the x digits as a packed 3D tensor of 16-bit words: ((n + 64) rows x 8 values, 6 planes, n / 8
    // groups); one box (32 rows, all planes, 16 groups) is a CTA's B operand for one d1
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) {
        ie_set_error("ie_matvec: cuTensorMapEncodeTiled is not available from the driver");
        return IE_ERR_CUDA;
    }
    CUtensorMap xmap;
    const cuuint64_t gdim[3] = {(cuuint64_t)(n + 64) * 8, (cuuint64_t)kZD, (cuuint64_t)(n / 8)};
    const cuuint64_t gstride[2] = {(cuuint64_t)(n + 64) * 16, (cuuint64_t)(n + 64) * 16 * kZD};
    const cuuint32_t box[3] = {(cuuint32_t)kZC * 8, (cuuint32_t)kZD, (cuuint32_t)(kZK / 8)};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult cr = encode(&xmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, xd.ptr, gdim, gstride, box, estride,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // the window table as a 3D tensor of 16-bit words: (8 values, 2n rows, n offsets x 6 planes);
    // one box (8 values, 248 rows, 6 planes) is a CTA's strip for one d1
    CUtensorMap wmap;
    const cuuint64_t wdim[3] = {8, (cuuint64_t)2 * n, (cuuint64_t)n * kZD};
    const cuuint64_t wstride[2] = {16, (cuuint64_t)2 * n * 16};
    const cuuint32_t wbox[3] = {8, (cuuint32_t)kZWin, (cuuint32_t)kZD};
    const CUresult cw = cr != CUDA_SUCCESS ? cr
                                           : encode(&wmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, p->d_zt_win, wdim, wstride, wbox,
                                                    estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cw != CUDA_SUCCESS) {
        ie_set_error("ie_matvec: cuTensorMapEncodeTiled failed (" + std::to_string((int)cw) + ")");
        return IE_ERR_CUDA;
    }
    const dim3 g(n / kZM, n / kZC, nparts);
    for (int k = 0; k < nrhs; ++k) {
        const double *xk = x + (long long)k * ldx;
        double *yk = y + (long long)k * ldy;
        IE_TRY_CUDA(cudaMemsetAsync(mx.ptr, 0, sizeof(unsigned long long), s));
        absmax_kernel<<<std::min<long long>(1024, (N + 255) / 256), 256, 0, s>>>(xk, N, mx.as<unsigned long long>());
        IE_LAUNCHED();
        const long long chunks = (long long)(n / 8) * (n + 64);
        x_digits_kernel<<<(unsigned)((chunks + 255) / 256), 256, 0, s>>>(xk, n, mx.as<unsigned long long>(), xd.as<uint4>());
        IE_LAUNCHED();
        kz_matvec_tc<<<g, 192, kZSmem, s>>>(wmap, xmap, n, ds, F, part.as<long long>(), p->d_err);
        IE_LAUNCHED();
        kz_combine_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(part.as<long long>(), nparts, N, xk, yk, p->diag,
                                                                     p->d_zt_max, mx.as<unsigned long long>(), F);
        IE_LAUNCHED();
    }
    return IE_OK;
}
