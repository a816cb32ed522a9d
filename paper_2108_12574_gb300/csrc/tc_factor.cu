// Mixed-precision subdomain factor on the tensor cores: A_i = L_i L_i^T and the explicit symmetric
// inverse M_i = A_i^{-1} = W_i^T W_i (W_i = L_i^{-1}) for every block at once, FP32 storage, the
// bulk of the flops as tcgen05 BF16 MMAs on exact three-part splits of the FP32 operands (the
// exact subdomain solver of Sec. 4.3, Eq. e:ai).
//
// Blocks are cut into tiles of P = 128 rows (the last one ragged, a multiple of 32).  Per block,
// in phases (a phase's tasks are independent of each other; phase p needs phases < p done):
//   for each panel k0:
//     DIAG       Cholesky of the diagonal tile in shared memory (32-wide blocked, 32 x 32
//                diagonal sub-tiles in one warp's registers), its triangular inverse Tinv in place
//                (kept per tile), and the diagonal tile of W^T (= Tinv^T, zero below its diagonal)
//     PANEL      L_21 = A_21 Tinv^T                                 (GEMM tasks, in place)
//     TRAILING   A_22 -= L_21 L_21^T over the lower tiles            (GEMM tasks)
//   then W by tile rows i = 1, 2, ...: G_ij = sum_{k=j}^{i-1} L_ik W_kj (stored transposed), then
//   W_ij = -Tinv_i G_ij (stored transposed, in W^T); finally M_ab = sum_k W_ka W_kb for the lower
//   tiles a >= b, written to (a, b) and mirrored to (b, a) from the same values, so M_i is exactly
//   symmetric; M_i replaces L_i in the pool.
//
// KP factor_persistent  ONE launch for all blocks: a grid of CTAs resident on every SM takes tasks
//                       (DIAG or GEMM) from one list in order (an atomic counter) and, before each,
//                       waits until every task of the earlier phases of its block is done (a
//                       per-block counter of finished tasks, release/acquire ordering; bounded
//                       wait).  The list is ordered by (phase + skew, block), largest blocks first,
//                       so every task's dependencies come earlier in it: a CTA only ever waits for
//                       tasks that running CTAs have taken, and nothing deadlocks whatever the
//                       number of resident CTAs.  The skew staggers the blocks' phases, so the
//                       CUDA-core DIAG tasks of some blocks run beside the GEMM tasks of others.
//                       CTAs per SM and the skew are chosen by the autotuner (every choice runs
//                       the same arithmetic per task: results are bitwise the same).
// GEMM task             C (<= 128 x 128) = s_old C + s_acc A B^T, A: m x k and B: n x k row-major
//                       FP32 with k contiguous (k a multiple of 32).  Per 16-wide chunk the threads
//                       copy A and B into a ring of three raw shared-memory slots with cp.async (L2
//                       only; two chunks ahead; each thread later reads back exactly the 16-byte
//                       pieces it copied, so the ring needs no block barrier), split each FP32
//                       value v exactly into three BF16 parts v = v0 + v1 + v2 and store the
//                       parts as three planes in the canonical K-major no-swizzle layout (8-row x
//                       16-byte core matrices); one thread issues six tcgen05.mma.kind::f16 (M =
//                       128, N = n rounded up to 16, K = 16) for the part products a_p b_q with
//                       p + q <= 2 (weights down to 2^-18; every BF16 product is exact in FP32, the
//                       dropped ones weigh <= 2^-26, so each product is FP32-accurate: three TF32
//                       products would give only ~2^-21) into an FP32 accumulator in tensor memory;
//                       same MMA time as three TF32 products, since BF16 runs at twice the TF32
//                       rate; two operand stages, tcgen05.commit to per-stage mbarriers, bounded
//                       waits.  The epilogue stages the accumulator in shared memory (tcgen05.ld
//                       32x32b) and writes C row-wise and / or the transposed CT column-wise, both
//                       coalesced.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "iedd_internal.cuh"

namespace {

constexpr int kP = 128;                 // tile rows
constexpr int kGK = 16;                 // K per operand chunk
constexpr uint32_t kGLBO = 128;         // bytes between core matrices along K (8 BF16 values each)
constexpr uint32_t kGSBO = (kGK / 8) * 128;  // bytes between 8-row groups
constexpr int kGOp = kP * kGK / 2;      // 32-bit words of one BF16 operand plane (128 x 16)
constexpr int kGStage = 6 * kGOp;       // A planes 0..2, B planes 0..2 (24 KB)
constexpr int kGPlaneBytes = 2 * kGStage * 4;  // two plane stages (48 KB)
constexpr int kGF4 = kP * kGK / 4 / 256;  // float4 per thread per operand and chunk (2)
constexpr int kGRawRow = kGK * 4 + 16;  // raw FP32 row stride in shared memory (80 bytes: the
                                        // 16-byte reads of eight consecutive rows hit distinct banks)
constexpr int kGRawOp = kP * kGRawRow;  // one raw operand chunk (10 KB)
constexpr int kGRawStages = 3;          // raw chunks in flight (cp.async, L2 -> shared memory)
constexpr int kGSmem = kGPlaneBytes + kGRawStages * 2 * kGRawOp;  // 108 KB: two CTAs per SM
constexpr int kTS = kP + 1;             // diagonal-kernel tile row stride (floats)
constexpr int kES = kP / 2 + 1;         // epilogue half-tile row stride (floats)
constexpr long long kGSpin = 1LL << 24; // non-blocking mbarrier polls before giving up
// kind::f16: D FP32 (bit 4), A and B BF16 (bits 7, 10), K-major both, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t gidesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kP >> 4) << 24);
}

struct GemmTask {
    const float *A, *B;  // operand origins: A rows 0..m-1, B rows 0..n-1, k contiguous
    float *C, *CT;       // outputs (either may be null)
    int lda, ldb, ldc, ldct;
    int m, n, k;         // m, n <= 128; k a multiple of 32
    float s_old, s_acc;  // C = s_old C + s_acc acc (C is not read when s_old == 0); CT^T = s_acc acc
    int diag;            // diagonal tile: C only where r >= c, CT only where c < r
    int pad_;
};

__device__ __forceinline__ uint32_t gsmem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// v = b0 + b1 + b2 exactly (three BF16 numbers of 8 significant bits each cover FP32's 24): each
// part is the round-to-nearest BF16 of what the earlier parts leave, and every remainder is exact
// in FP32.  Two values at a time (packed conversions): p_q holds part q of x (low half) and of y
// (high half).
__device__ __forceinline__ void bf16x3_pair(float x, float y, uint32_t &p0, uint32_t &p1, uint32_t &p2) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p0) : "f"(y), "f"(x));
    float rx = x - __uint_as_float(p0 << 16), ry = y - __uint_as_float(p0 & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p1) : "f"(ry), "f"(rx));
    rx -= __uint_as_float(p1 << 16);
    ry -= __uint_as_float(p1 & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p2) : "f"(ry), "f"(rx));
}

__device__ __forceinline__ uint64_t gdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kGLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kGSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // tcgen05 descriptor version; base offset 0, no swizzle
    return d;
}

__device__ __forceinline__ void gmma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// one suspending probe (the thread may sleep up to ~1 us while the phase is pending)
__device__ __forceinline__ bool gbar_try(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase), "r"(1000u)
        : "memory");
    return ok != 0;
}

// bounded wait (a few seconds at most); false if the limit ran out
__device__ __forceinline__ bool gbar_wait(uint32_t bar, uint32_t phase) {
    for (long long i = 0; i < kGSpin / 8; ++i)
        if (gbar_try(bar, phase)) return true;
    return false;
}

// One operand chunk (128 rows x 16 columns, 512 float4) copied from global memory into a raw
// shared-memory slot with cp.async (L2 only: other CTAs of the persistent factor write these tiles
// between tasks); element e = tid + 256 u: row (e / 32) * 8 + e % 8, float4 column (e / 8) % 4.
// Rows past rows_valid are zero-filled (source size 0).
__device__ __forceinline__ void chunk_issue(const float *src, int ld, int rows_valid, int c0, int tid,
                                            uint32_t raw) {
#pragma unroll
    for (int u = 0; u < kGF4; ++u) {
        const int e = tid + 256 * u;
        const int r = (e >> 5) * 8 + (e & 7), k4 = (e >> 3) & 3;
        const bool ok = r < rows_valid;
        const float *g = src + (ok ? (long long)r * ld + c0 + 4 * k4 : 0);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(raw + (uint32_t)(r * kGRawRow + 16 * k4)),
                     "l"(g), "r"(ok ? 16 : 0)
                     : "memory");
    }
}

// The same elements back from the raw slot (the thread reads the float4s it copied itself)
__device__ __forceinline__ void chunk_read(const unsigned char *raw, int tid, float4 (&v)[kGF4]) {
#pragma unroll
    for (int u = 0; u < kGF4; ++u) {
        const int e = tid + 256 * u;
        const int r = (e >> 5) * 8 + (e & 7), k4 = (e >> 3) & 3;
        v[u] = *reinterpret_cast<const float4 *>(raw + r * kGRawRow + 16 * k4);
    }
}

// The three BF16 planes of one operand chunk in the canonical K-major layout: plane q holds part
// q of every value; row r's 16 values are two core-matrix rows of 8 (16 bytes each), a float4 of
// thread data is half of one (8 bytes).
__device__ __forceinline__ void chunk_store(const float4 (&v)[kGF4], uint32_t *planes, int tid) {
#pragma unroll
    for (int u = 0; u < kGF4; ++u) {
        const int e = tid + 256 * u;
        const int r = (e >> 5) * 8 + (e & 7), k4 = (e >> 3) & 3;
        const uint32_t off = (uint32_t)(((r >> 3) * kGSBO + (k4 >> 1) * kGLBO + (r & 7) * 16 + (k4 & 1) * 8) >> 2);
        uint32_t p0, p1, p2, q0, q1, q2;
        bf16x3_pair(v[u].x, v[u].y, p0, p1, p2);
        bf16x3_pair(v[u].z, v[u].w, q0, q1, q2);
        *reinterpret_cast<uint2 *>(planes + off) = make_uint2(p0, q0);
        *reinterpret_cast<uint2 *>(planes + kGOp + off) = make_uint2(p1, q1);
        *reinterpret_cast<uint2 *>(planes + 2 * kGOp + off) = make_uint2(p2, q2);
    }
}

// Per-CTA state of the GEMM tasks kept across the tasks of the persistent kernel
struct GemmCta {
    uint32_t tmem;     // 128 TMEM columns (the accumulator)
    uint64_t *mbar;    // two stage barriers
    uint32_t ph[2];    // their next parities
    int *abort_flag;   // shared: a bounded wait ran out
};

// One GEMM task (all 256 threads).  Returns with every MMA it issued complete.
__device__ void gemm_task(const GemmTask &t, uint32_t *gsm, GemmCta &c) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = t.k / kGK;
    const uint32_t idesc = gidesc((t.n + 15) & ~15);
    int pending[2] = {0, 0};
    unsigned char *raw0 = reinterpret_cast<unsigned char *>(gsm) + kGPlaneBytes;
    const uint32_t raw0_s = gsmem_u32(raw0);
    auto raw_of = [&](int ch) { return (uint32_t)((ch % kGRawStages) * 2 * kGRawOp); };
    // prologue: chunks 0 and 1 in flight; every chunk index gets one commit group (empty past the
    // end), so that "all but the newest group" is always the chunk about to be converted
    for (int ch = 0; ch < 2; ++ch) {
        if (ch < nch) {
            chunk_issue(t.A, t.lda, t.m, ch * kGK, tid, raw0_s + raw_of(ch));
            chunk_issue(t.B, t.ldb, t.n, ch * kGK, tid, raw0_s + raw_of(ch) + kGRawOp);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int ch = 0; ch < nch; ++ch) {
        const int st = ch & 1;
        uint32_t *Ap = gsm + st * kGStage, *Bp = Ap + 3 * kGOp;
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this thread's copies of chunk ch
        if (pending[st]) {  // the plane stage's previous MMAs must be done before it changes;
                            // one thread waits, the barrier below releases the others
            if (tid == 0 && !gbar_wait(gsmem_u32(&c.mbar[st]), c.ph[st])) *c.abort_flag = 1;
            c.ph[st] ^= 1u;
            pending[st] = 0;
        }
        __syncthreads();  // every copy of chunk ch landed; every read of raw slot (ch + 2) % 3 done
        if (*c.abort_flag) break;
        float4 va[kGF4], vb[kGF4];
        chunk_read(raw0 + raw_of(ch), tid, va);
        chunk_read(raw0 + raw_of(ch) + kGRawOp, tid, vb);
        if (ch + 2 < nch) {
            chunk_issue(t.A, t.lda, t.m, (ch + 2) * kGK, tid, raw0_s + raw_of(ch + 2));
            chunk_issue(t.B, t.ldb, t.n, (ch + 2) * kGK, tid, raw0_s + raw_of(ch + 2) + kGRawOp);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        chunk_store(va, Ap, tid);
        chunk_store(vb, Bp, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // the six BF16 part products of weight >= 2^-16 relative (a_p b_q with p + q <= 2), one
            // K = 16 MMA each: every product is exact in the FP32 accumulator
            const uint32_t a0 = gsmem_u32(Ap), b0 = gsmem_u32(Bp), pl = (uint32_t)kGOp * 4u;
            gmma(c.tmem, gdesc(a0), gdesc(b0), idesc, ch > 0 ? 1u : 0u);
            gmma(c.tmem, gdesc(a0), gdesc(b0 + pl), idesc, 1u);
            gmma(c.tmem, gdesc(a0 + pl), gdesc(b0), idesc, 1u);
            gmma(c.tmem, gdesc(a0), gdesc(b0 + 2 * pl), idesc, 1u);
            gmma(c.tmem, gdesc(a0 + pl), gdesc(b0 + pl), idesc, 1u);
            gmma(c.tmem, gdesc(a0 + 2 * pl), gdesc(b0), idesc, 1u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             gsmem_u32(&c.mbar[st]))
                         : "memory");
        }
        pending[st] = 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy in flight past the task
    for (int st = 0; st < 2; ++st) {  // drain (bounded, one thread; waits even after an abort so
                                      // that no MMA is in flight when the CTA moves on)
        if (pending[st]) {
            if (tid == 0 && !gbar_wait(gsmem_u32(&c.mbar[st]), c.ph[st])) *c.abort_flag = 1;
            c.ph[st] ^= 1u;
            pending[st] = 0;
        }
    }
    __syncthreads();
    if (*c.abort_flag || nch == 0) return;
    // accumulator -> shared half tile T[r][cl] (64 columns per pass, stride kES): warp w reads TMEM
    // lanes 32 (w % 4) .., columns 64 pass + 32 (w / 4) ..; then C row-wise, CT column-wise
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float *T = reinterpret_cast<float *>(gsm);
    const int q = warp & 3, h = warp >> 2;
    for (int pass = 0; pass < 2; ++pass) {
        const int cbase = 64 * pass;
        if (cbase >= t.n) break;  // uniform
        {
            uint32_t v[32];
            const uint32_t taddr = c.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cbase + 32 * h);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float *row = T + (32 * q + lane) * kES + 32 * h;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) row[cc] = __uint_as_float(v[cc]);
        }
        __syncthreads();
        if (t.C) {
            // 16 elements per batch: their old values are loaded together before any store (the
            // compiler cannot overlap a load with an earlier store through the same pointer)
            for (int e0 = 0; e0 < kP * 64; e0 += 256 * 16) {
                float old[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = e0 + tid + 256 * i, r = e >> 6, cc = cbase + (e & 63);
                    const bool in = r < t.m && cc < t.n && (!t.diag || r >= cc);
                    old[i] = (in && t.s_old != 0.f) ? __ldcg(t.C + (long long)r * t.ldc + cc) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = e0 + tid + 256 * i, r = e >> 6, cl = e & 63, cc = cbase + cl;
                    if (r < t.m && cc < t.n && (!t.diag || r >= cc))
                        t.C[(long long)r * t.ldc + cc] = fmaf(t.s_acc, T[r * kES + cl], t.s_old * old[i]);
                }
            }
        }
        if (t.CT) {
            for (int e = tid; e < kP * 64; e += 256) {
                const int cl = e >> 7, r = e & (kP - 1), cc = cbase + cl;
                if (r < t.m && cc < t.n && (!t.diag || cc < r))
                    t.CT[(long long)cc * t.ldct + r] = t.s_acc * T[r * kES + cl];
            }
        }
        __syncthreads();
    }
    // the next task's MMAs overwrite the accumulator only after every thread has read it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// X = L^{-1} of the lower-triangular 32 x 32 tile L (row stride ld) into X (row stride 33, zero
// above the diagonal), all 256 threads: warp w takes columns 4w .. 4w + 3 and runs their chains
// down the column together (lane = row, entries shuffled down).
__device__ __forceinline__ void tile_inverse32(const float *L, int ld, float *X) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float lrow[32];
    float dii = 1.f;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        lrow[c] = c <= lane ? L[lane * ld + c] : 0.f;
        if (c == lane) dii = lrow[c];
    }
    const float rdii = 1.f / dii;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q) X[lane * 33 + 4 * warp + q] = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 4 * warp + q;
            if (k >= j) {
                const float mine = lane == k ? (k == j ? rdii : -acc[q] * rdii) : 0.f;
                const float xk = __shfl_sync(0xffffffffu, mine, k);
                if (lane == k) X[k * 33 + j] = xk;
                if (lane > k) acc[q] = fmaf(lrow[k], xk, acc[q]);
            }
        }
    }
}

// The diagonal tile of panel k0 of block b, in one 128 x 129 shared tile D: the block's entries,
// then L_kk (written back), then Tinv = L_kk^{-1} in place.  Per 32-column step: one warp factors
// the 32 x 32 diagonal sub-tile in registers, all warps invert it (X11, kept in Xd for the final
// inverse), the rows below become L21 = A21 X11^T (a product, no divisions or dependency chains),
// and the trailing lower part is updated.  Xd: 4 x 32 x 33 floats after D.
__device__ void diag_task(float *__restrict__ pool, float *__restrict__ wt, float *__restrict__ tinv,
                          const long long *__restrict__ loff, const long long *__restrict__ toff,
                          const int *__restrict__ npad, int b, int k0, int *__restrict__ info, float *D, int *bad) {
    const int np = npad[b], pk = min(kP, np - k0), nt = pk / 32;
    float *A = pool + loff[b] + (long long)k0 * np + k0;
    float *Xd = D + kP * kTS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kRows = (kP - 32) * 32 / 256;  // outputs per thread below a 32-column block (12)
    if (tid == 0) *bad = -1;
    // the tile's lower part into D, 16 loads in flight per thread (the compiler cannot overlap
    // loads with stores through pointers that may alias)
    for (int e0 = 0; e0 < kP * kP; e0 += 256 * 16) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = e0 + tid + 256 * i, r = e >> 7, c = e & (kP - 1);
            v[i] = (r < pk && c <= r) ? __ldcg(A + (long long)r * np + c) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = e0 + tid + 256 * i;
            D[(e >> 7) * kTS + (e & (kP - 1))] = v[i];
        }
    }
    __syncthreads();
    for (int kk = 0; kk < nt; ++kk) {
        const int c0 = kk * 32, r0 = c0 + 32, rest = pk - r0;
        // the 32 x 32 diagonal sub-tile in one warp's registers (lane = row): right-looking,
        // column j's entries shuffled to the lanes that update with them
        if (warp == 0) {
            float row[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) row[c] = c <= lane ? D[(c0 + lane) * kTS + c0 + c] : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float piv = __shfl_sync(0xffffffffu, row[j], j);
                if (!(piv > 0.f)) {  // uniform: every lane holds the same pivot
                    if (lane == 0 && *bad < 0) *bad = c0 + j;
                    piv = 1.f;
                }
                const float djj = sqrtf(piv);
                const float lij = lane > j ? row[j] / djj : (lane == j ? djj : 0.f);
                if (lane >= j) row[j] = lij;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    if (c > j) {  // compile-time after unrolling
                        const float lcj = __shfl_sync(0xffffffffu, lij, c);
                        if (c <= lane) row[c] = fmaf(-lij, lcj, row[c]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c <= lane) D[(c0 + lane) * kTS + c0 + c] = row[c];
        }
        __syncthreads();
        float *X11 = Xd + kk * 32 * 33;
        tile_inverse32(D + c0 * kTS + c0, kTS, X11);
        __syncthreads();
        if (rest > 0) {
            // L21 = A21 X11^T: thread column c = lane, rows r0 + warp + 8 i
            float u[kRows];
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int r = r0 + warp + 8 * i;
                float acc = 0.f;
                if (r < pk) {
#pragma unroll 8
                    for (int t2 = 0; t2 < 32; ++t2) acc = fmaf(D[r * kTS + c0 + t2], X11[lane * 33 + t2], acc);
                }
                u[i] = acc;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int r = r0 + warp + 8 * i;
                if (r < pk) D[r * kTS + c0 + lane] = u[i];
            }
            __syncthreads();
            // trailing lower part: D[i][c] -= sum_t D[i][c0 + t] D[c][c0 + t], r0 <= c <= i < pk
            // (warp: rows i = r0 + warp + 8 s; lane: columns c = r0 + lane + 32 q)
            for (int i = r0 + warp; i < pk; i += 8) {
                for (int c = r0 + lane; c <= i; c += 32) {
                    float sum = 0.f;
#pragma unroll 8
                    for (int t2 = 0; t2 < 32; ++t2) sum = fmaf(D[i * kTS + c0 + t2], D[c * kTS + c0 + t2], sum);
                    D[i * kTS + c] -= sum;
                }
            }
            __syncthreads();
        }
    }
    // L_kk back to the pool (lower part)
    for (int e = tid; e < pk * pk; e += 256) {
        const int r = e / pk, c = e % pk;
        if (c <= r) A[(long long)r * np + c] = D[r * kTS + c];
    }
    __syncthreads();
    // D := L_kk^{-1} in place, 32-column blocks from the last one back: with L = [L11 0; L21 L22]
    // and X22 = L22^{-1} already in place, X21 = -X22 (L21 X11) with X11 from Xd, each product
    // formed in registers before it overwrites its operand
    for (int jb = nt - 1; jb >= 0; --jb) {
        const int c0 = jb * 32, r0 = c0 + 32, rest = pk - r0;
        const float *X11 = Xd + jb * 32 * 33;
        if (rest > 0) {
            // thread: column c = lane, rows r0 + warp + 8 i
            float u[kRows];
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int r = r0 + warp + 8 * i;
                float acc = 0.f;
                if (r < pk) {
                    for (int t2 = lane; t2 < 32; ++t2) acc = fmaf(D[r * kTS + c0 + t2], X11[t2 * 33 + lane], acc);
                }
                u[i] = acc;  // (L21 X11)[r][c]
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int r = r0 + warp + 8 * i;
                if (r < pk) D[r * kTS + c0 + lane] = u[i];
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int r = r0 + warp + 8 * i;
                float acc = 0.f;
                if (r < pk) {
                    for (int k = r0; k <= r; ++k) acc = fmaf(D[r * kTS + k], D[k * kTS + c0 + lane], acc);
                }
                u[i] = -acc;  // (-X22 U)[r][c]
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int r = r0 + warp + 8 * i;
                if (r < pk) D[r * kTS + c0 + lane] = u[i];
            }
        }
        // X11 into the diagonal block (L11 is no longer needed)
        for (int e = tid; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            D[(c0 + r) * kTS + c0 + c] = X11[r * 33 + c];
        }
        __syncthreads();
    }
    // Tinv (128 x 128, zero outside pk x pk) and the diagonal tile of W^T (Tinv^T, zero below)
    float *Tb = tinv + toff[b] + (long long)(k0 / kP) * kP * kP;
    float *Wb = wt + loff[b] + (long long)k0 * np + k0;
    for (int e = tid; e < kP * kP; e += 256) {
        const int r = e >> 7, c = e & (kP - 1);
        Tb[e] = (r < pk && c <= r) ? D[r * kTS + c] : 0.f;
        if (r < pk && c < pk) Wb[(long long)r * np + c] = c >= r ? D[c * kTS + r] : 0.f;
    }
    __syncthreads();
    if (tid == 0 && *bad >= 0 && info[b] < 0) info[b] = k0 + *bad;
}

// One entry of the persistent factor's task list
struct FTask {
    GemmTask g;    // kind 0
    int kind;      // 0 GEMM, 1 DIAG
    int block;
    int need;      // finished tasks of this block required first (all of its earlier phases)
    int k0;        // DIAG: first row of the diagonal tile
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr long long kDepSpin = 1LL << 26;  // polls (~1 us each at most) of a block's counter

__global__ void __launch_bounds__(256, 2)
factor_persistent(const FTask *__restrict__ tasks, int ntasks, int *__restrict__ next, int *__restrict__ done,
                  float *__restrict__ pool, float *__restrict__ wt, float *__restrict__ tinv,
                  const long long *__restrict__ loff, const long long *__restrict__ toff,
                  const int *__restrict__ npad, int *__restrict__ info, int *__restrict__ err) {
    extern __shared__ __align__(1024) uint32_t gsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, cur, bad;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gsmem_u32(&tmem_base)),
                     "r"((uint32_t)kP));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < 2; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gsmem_u32(&mbar[st])), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    GemmCta c;
    c.tmem = tmem_base;
    c.mbar = mbar;
    c.ph[0] = c.ph[1] = 0u;
    c.abort_flag = &abort_flag;
    for (;;) {
        if (tid == 0) {
            int t = atomicAdd(next, 1);
            if (t < ntasks) {
                // wait (bounded) until the block's earlier phases are done; give up if another
                // CTA has recorded an error
                const FTask &ft = tasks[t];
                long long i = 0;
                while (ld_acquire(done + ft.block) < ft.need) {
                    if (ld_acquire(err) != 0) { t = ntasks; break; }
                    if (++i > kDepSpin) { atomicExch(err, 2); t = ntasks; break; }
                    __nanosleep(256);
                }
            }
            cur = t;
        }
        __syncthreads();
        const int t = cur;
        if (t >= ntasks) break;
        const FTask &ft = tasks[t];
        if (ft.kind == 1) {
            diag_task(pool, wt, tinv, loff, toff, npad, ft.block, ft.k0, info, reinterpret_cast<float *>(gsm), &bad);
        } else {
            gemm_task(ft.g, gsm, c);
        }
        __syncthreads();
        if (abort_flag) {
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        if (tid == 0) {
            __threadfence();  // this task's writes before the count that releases its dependants
            atomicAdd(done + ft.block, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"((uint32_t)kP));
    }
}

}  // namespace

constexpr int kDiagSmem = (kP * kTS + 4 * 32 * 33) * (int)sizeof(float);
constexpr int kFSmem = kDiagSmem > kGSmem ? kDiagSmem : kGSmem;

int prepare_tc_factor() {
    IE_TRY_CUDA(cudaFuncSetAttribute(factor_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmem));
    return IE_OK;
}

namespace {

// The task list of the persistent factor for a given skew: each block's phases (DIAG, PANEL and
// TRAILING per panel; then G and W per tile row of W; then M), ordered by (phase + rank % skew,
// rank), rank = the block's place in decreasing size order.  A task's `need` is the number of
// tasks of its block in the phases before its own.
void build_plan(const std::vector<int> &npad, const std::vector<long long> &loff, const std::vector<int> &order,
                float *pool, float *W, float *T, float *G, const std::vector<long long> &toff,
                const std::vector<long long> &goff, int skew, std::vector<FTask> &out) {
    const int nb = (int)npad.size();
    // per block: its tasks in phase order and the first task of every phase
    std::vector<std::vector<FTask>> bt((size_t)nb);
    std::vector<std::vector<int>> first((size_t)nb);
    size_t total = 0;
    int max_levels = 0;
    for (int b = 0; b < nb; ++b) {
        const int np = npad[(size_t)b];
        std::vector<FTask> &tl = bt[(size_t)b];
        std::vector<int> &ph = first[(size_t)b];
        float *P_ = pool + loff[(size_t)b], *W_ = W + loff[(size_t)b], *G_ = G + goff[(size_t)b];
        auto T_ = [&](int i) { return T + toff[(size_t)b] + (long long)i * kP * kP; };
        int open = 0;  // tasks since the phase began
        auto begin = [&]() { open = 0; ph.push_back((int)tl.size()); };
        auto close_phase = [&]() {
            if (open == 0) ph.pop_back();  // an empty phase
        };
        auto need = [&]() { return ph.back(); };  // every task of the earlier phases
        auto gemm = [&](const float *A, int lda, const float *B, int ldb, int m, int n, int k, float *C, int ldc,
                        float *CT, int ldct, float s_old, float s_acc, int diag) {
            FTask t{};
            t.kind = 0; t.block = b; t.need = need(); t.k0 = 0;
            t.g.A = A; t.g.B = B; t.g.C = C; t.g.CT = CT;
            t.g.lda = lda; t.g.ldb = ldb; t.g.ldc = ldc; t.g.ldct = ldct;
            t.g.m = m; t.g.n = n; t.g.k = k; t.g.s_old = s_old; t.g.s_acc = s_acc; t.g.diag = diag; t.g.pad_ = 0;
            tl.push_back(t);
            ++open;
        };
        for (int k0 = 0; k0 < np; k0 += kP) {
            const int pk = std::min(kP, np - k0);
            begin();
            FTask d{};
            d.kind = 1; d.block = b; d.need = need(); d.k0 = k0;
            tl.push_back(d);
            ++open;
            close_phase();
            begin();
            for (int r0 = k0 + pk; r0 < np; r0 += kP) {  // panel: L_21 = A_21 Tinv^T, in place
                float *a = P_ + (long long)r0 * np + k0;
                gemm(a, np, T_(k0 / kP), kP, std::min(kP, np - r0), pk, pk, a, np, nullptr, 0, 0.f, 1.f, 0);
            }
            close_phase();
            begin();
            for (int ra = k0 + pk; ra < np; ra += kP)  // trailing: A_22 -= L_21 L_21^T, lower tiles
                for (int rb = k0 + pk; rb <= ra; rb += kP)
                    gemm(P_ + (long long)ra * np + k0, np, P_ + (long long)rb * np + k0, np, std::min(kP, np - ra),
                         std::min(kP, np - rb), pk, P_ + (long long)ra * np + rb, np, nullptr, 0, 1.f, -1.f, 0);
            close_phase();
        }
        const int nt = (np + kP - 1) / kP;
        for (int i = 1; i < nt; ++i) {  // W = L^{-1} by tile rows (W^T stored)
            const int ri = i * kP, mi = std::min(kP, np - ri);
            begin();
            for (int j = 0; j < i; ++j) {
                const int rj = j * kP;
                gemm(P_ + (long long)ri * np + rj, np, W_ + (long long)rj * np + rj, np, mi, kP, ri - rj, nullptr, 0,
                     G_ + (long long)rj * kP, kP, 0.f, 1.f, 0);
            }
            close_phase();
            begin();
            for (int j = 0; j < i; ++j) {
                const int rj = j * kP;
                gemm(T_(i), kP, G_ + (long long)rj * kP, kP, mi, kP, mi, nullptr, 0, W_ + (long long)rj * np + ri, np,
                     0.f, -1.f, 0);
            }
            close_phase();
        }
        begin();
        for (int ra = 0; ra < np; ra += kP)  // M = W^T W into the pool: lower tiles a >= b, mirrored
            for (int rb = 0; rb <= ra; rb += kP)
                gemm(W_ + (long long)ra * np + ra, np, W_ + (long long)rb * np + ra, np, std::min(kP, np - ra),
                     std::min(kP, np - rb), np - ra, P_ + (long long)ra * np + rb, np, P_ + (long long)rb * np + ra, np,
                     0.f, 1.f, ra == rb ? 1 : 0);
        close_phase();
        ph.push_back((int)tl.size());  // sentinel: the end of the last phase
        total += tl.size();
        max_levels = std::max(max_levels, (int)ph.size() - 1);
    }
    // emit by (phase + rank % skew, rank): every task's dependencies come before it
    out.clear();
    out.reserve(total);
    for (int key = 0; key < max_levels + skew; ++key)
        for (int r = 0; r < nb; ++r) {
            const int b = order[(size_t)r], l = key - r % skew;
            const std::vector<int> &ph = first[(size_t)b];
            if (l < 0 || l + 1 >= (int)ph.size()) continue;
            for (int i = ph[(size_t)l]; i < ph[(size_t)l + 1]; ++i) out.push_back(bt[(size_t)b][(size_t)i]);
        }
}

// candidates of the factor's autotuner: CTAs per SM x skew
constexpr int kFactorCand[][2] = {{2, 1}, {2, 2}, {2, 4}, {1, 2}};
constexpr int kFactorNCand = (int)(sizeof(kFactorCand) / sizeof(kFactorCand[0]));

}  // namespace

// L and then M in f->d_pool (FP32, already holding the gathered lower blocks); synchronizes.  One
// launch of the persistent kernel; with the autotuner on, the first factor of a shape times every
// candidate (CTAs per SM, skew) on a copy of the gathered blocks and keeps the fastest.
int launch_factor_tc(dd_factor_t *f, const std::vector<int> &npad, const std::vector<long long> &loff,
                     cudaStream_t s) {
    const int nb = f->nblocks;
    if (nb == 0) return IE_OK;
    IE_TRY(prepare_tc_factor());
    float *pool = (float *)f->d_pool;
    std::vector<long long> toff((size_t)nb + 1, 0), goff((size_t)nb + 1, 0);
    long long sum_np = 0;
    for (int b = 0; b < nb; ++b) {
        const int nt = (npad[(size_t)b] + kP - 1) / kP;
        toff[(size_t)b + 1] = toff[(size_t)b] + (long long)nt * kP * kP;
        goff[(size_t)b + 1] = goff[(size_t)b] + (long long)npad[(size_t)b] * kP;
        sum_np += npad[(size_t)b];
    }
    std::vector<int> order((size_t)nb);
    for (int b = 0; b < nb; ++b) order[(size_t)b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return npad[(size_t)a] > npad[(size_t)b]; });
    DevBuf wt, tinv, gbuf, dtoff, derr, dnext, ddone;
    IE_TRY(wt.alloc(sizeof(float) * (size_t)f->pool_elems, s));
    IE_TRY(tinv.alloc(sizeof(float) * (size_t)toff.back(), s));
    IE_TRY(gbuf.alloc(sizeof(float) * (size_t)goff.back(), s));
    IE_TRY(dtoff.alloc(sizeof(long long) * toff.size(), s));
    IE_TRY(derr.alloc(sizeof(int), s));
    IE_TRY(dnext.alloc(sizeof(int), s));
    IE_TRY(ddone.alloc(sizeof(int) * (size_t)nb, s));
    IE_TRY_CUDA(cudaMemcpyAsync(dtoff.ptr, toff.data(), sizeof(long long) * toff.size(), cudaMemcpyHostToDevice, s));
    IE_TRY_CUDA(cudaMemsetAsync(derr.ptr, 0, sizeof(int), s));
    float *W = wt.as<float>(), *T = tinv.as<float>(), *G = gbuf.as<float>();
    const int sms = f->prob->sm_count;

    // IEDD_FACTOR_SCHEDULE="c,s" fixes the schedule (c CTAs per SM, skew s) instead of the tuner's
    int force_ctas = 0, force_skew = 0;
    if (const char *env = std::getenv("IEDD_FACTOR_SCHEDULE")) {
        if (std::sscanf(env, "%d,%d", &force_ctas, &force_skew) != 2 || force_ctas < 1 || force_ctas > 2 ||
            force_skew < 1 || force_skew > 64)
            force_ctas = force_skew = 0;
    }
    auto run = [&](int ctas, const std::vector<FTask> &tasks, DevBuf &dtasks) -> int {
        IE_TRY_CUDA(cudaMemsetAsync(dnext.ptr, 0, sizeof(int), s));
        IE_TRY_CUDA(cudaMemsetAsync(ddone.ptr, 0, sizeof(int) * (size_t)nb, s));
        const int grid = std::max(1, std::min((int)tasks.size(), sms * ctas));
        factor_persistent<<<grid, 256, kFSmem, s>>>(dtasks.as<FTask>(), (int)tasks.size(), dnext.as<int>(),
                                                    ddone.as<int>(), pool, W, T, f->d_loff, dtoff.as<long long>(),
                                                    f->d_npad, f->d_info, derr.as<int>());
        IE_LAUNCHED();
        return IE_OK;
    };
    auto upload = [&](const std::vector<FTask> &tasks, DevBuf &dtasks) -> int {
        IE_TRY(dtasks.alloc(sizeof(FTask) * std::max<size_t>(tasks.size(), 1), s));
        IE_TRY_CUDA(cudaMemcpyAsync(dtasks.ptr, tasks.data(), sizeof(FTask) * tasks.size(), cudaMemcpyHostToDevice, s));
        return IE_OK;
    };

    const std::string key = "factor/nb" + std::to_string(nb) + "/max" + std::to_string(f->max_pad) + "/sum" +
                            std::to_string(sum_np);
    int cand = 1;  // default: two CTAs per SM, skew 2
    int tuned = -1;
    // tuning runs every candidate once: only where a factor is cheap (not the dense CBD colour
    // blocks, whose factor takes seconds)
    double work = 0.0;
    for (int b = 0; b < nb; ++b) work += (double)npad[(size_t)b] * npad[(size_t)b] * npad[(size_t)b];
    const bool tune = force_ctas == 0 && autotune_enabled() && !ie_capturing() && work < 2e12 && !tune_get(key, &tuned);
    if (tuned >= 0) cand = tuned;
    if (tune) {
        // time every candidate on a copy of the gathered blocks (the factor works in place)
        DevBuf saved;
        IE_TRY(saved.alloc(sizeof(float) * (size_t)f->pool_elems, s));
        IE_TRY_CUDA(cudaMemcpyAsync(saved.ptr, pool, sizeof(float) * (size_t)f->pool_elems, cudaMemcpyDeviceToDevice, s));
        cudaEvent_t e0, e1;
        IE_TRY_CUDA(cudaEventCreate(&e0));
        IE_TRY_CUDA(cudaEventCreate(&e1));
        float best = -1.f;
        std::string detail;
        for (int c = 0; c < kFactorNCand; ++c) {
            std::vector<FTask> tasks;
            build_plan(npad, loff, order, pool, W, T, G, toff, goff, kFactorCand[c][1], tasks);
            DevBuf dtasks;
            IE_TRY(upload(tasks, dtasks));
            IE_TRY_CUDA(cudaMemcpyAsync(pool, saved.ptr, sizeof(float) * (size_t)f->pool_elems, cudaMemcpyDeviceToDevice, s));
            IE_TRY_CUDA(cudaEventRecord(e0, s));
            IE_TRY(run(kFactorCand[c][0], tasks, dtasks));
            IE_TRY_CUDA(cudaEventRecord(e1, s));
            IE_TRY_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            IE_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            detail += (c ? ", " : "") + std::to_string(kFactorCand[c][0]) + "x" + std::to_string(kFactorCand[c][1]) + ":" +
                      std::to_string(ms).substr(0, 6) + "ms";
            if (best < 0.f || ms < best) { best = ms; cand = c; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tune_put(key, cand, "CTAs/SM x skew: " + detail);
        IE_TRY_CUDA(cudaMemcpyAsync(pool, saved.ptr, sizeof(float) * (size_t)f->pool_elems, cudaMemcpyDeviceToDevice, s));
        IE_TRY_CUDA(cudaMemsetAsync(f->d_info, 0xFF, sizeof(int) * (size_t)nb, s));
        IE_TRY_CUDA(cudaMemsetAsync(derr.ptr, 0, sizeof(int), s));
    }
    const int ctas = force_ctas ? force_ctas : kFactorCand[cand][0];
    const int skew = force_ctas ? force_skew : kFactorCand[cand][1];
    std::vector<FTask> tasks;
    build_plan(npad, loff, order, pool, W, T, G, toff, goff, skew, tasks);
    DevBuf dtasks;
    IE_TRY(upload(tasks, dtasks));
    IE_TRY(run(ctas, tasks, dtasks));
    int herr = 0;
    IE_TRY_CUDA(cudaMemcpyAsync(&herr, derr.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    IE_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        ie_set_error(herr == 2 ? "dd_factor: a task of the persistent factor timed out waiting for its block"
                               : "dd_factor: a tensor-core GEMM timed out waiting for its MMAs");
        return IE_ERR_TIMEOUT;
    }
    return IE_OK;
}

// ---------------------------------------------------------------------------------------------
// The batched apply on the tensor cores: per block, per 128-row tile of M_i, per group of up to
// 128 right-hand sides one GEMM task C^T = M_i[rows, :] X_i^T (X_i: the block's scaled FP32 right-
// hand sides, K = the padded block size), run by the persistent kernel with no dependencies.  The
// task list is written on the device (the call may be captured in a CUDA graph).
// ---------------------------------------------------------------------------------------------
namespace {

__global__ void apply_tasks_kernel(const int *__restrict__ npad, const int *__restrict__ nb,
                                   const long long *__restrict__ loff, const long long *__restrict__ xoff,
                                   const long long *__restrict__ tile_off, const float *pool, const float *xh, float *tmp,
                                   long long xtotal, int nrhs, int ngroups, FTask *__restrict__ tasks) {
    const int b = blockIdx.x;
    const int np = npad[b], n = nb[b];
    const int tiles = (n + kP - 1) / kP;
    for (int e = threadIdx.x; e < tiles * ngroups; e += blockDim.x) {
        const int i = e / ngroups, g = e % ngroups;
        const int r0 = i * kP, c0 = g * kP;
        FTask t{};
        t.kind = 0; t.block = 0; t.need = 0; t.k0 = 0;
        t.g.A = pool + loff[b] + (long long)r0 * np;
        t.g.lda = np;
        t.g.B = xh + (long long)c0 * xtotal + xoff[b];
        t.g.ldb = (int)xtotal;
        t.g.C = nullptr;
        t.g.ldc = 0;
        t.g.CT = tmp + (long long)c0 * xtotal + xoff[b] + r0;
        t.g.ldct = (int)xtotal;
        t.g.m = min(kP, n - r0);
        t.g.n = min(kP, nrhs - c0);
        t.g.k = np;
        t.g.s_old = 0.f;
        t.g.s_acc = 1.f;
        t.g.diag = 0;
        t.g.pad_ = 0;
        tasks[(tile_off[b] + i) * ngroups + g] = t;
    }
}

__device__ __forceinline__ double pow2_exp(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// zbuf[k][offs[b] + j] = tmp[k][xoff[b] + j] 2^e(b, k) (exact: two power-of-two factors)
__global__ void apply_widen_kernel(const float *__restrict__ tmp, const int *__restrict__ nb,
                                   const long long *__restrict__ offs, const long long *__restrict__ xoff,
                                   const int *__restrict__ xexp, long long xtotal, long long total, int nblocks,
                                   double *__restrict__ zbuf) {
    const int b = blockIdx.x, k = blockIdx.y;
    const int n = nb[b], e = xexp[(long long)k * nblocks + b], e1 = e / 2;
    const double s1 = pow2_exp(e1), s2 = pow2_exp(e - e1);
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        zbuf[(long long)k * total + offs[b] + j] = ((double)tmp[(long long)k * xtotal + xoff[b] + j] * s1) * s2;
}

}  // namespace

int launch_apply_tc(const dd_factor_t *f, const float *xh, const int *xe, int nrhs, double *zbuf, cudaStream_t s) {
    const int nb = f->nblocks;
    if (nb == 0 || nrhs < 1) return IE_OK;
    if (!f->d_tile_off) {
        ie_set_error("dd_apply: the tensor-core apply tables are missing");
        return IE_ERR_ARG;
    }
    IE_TRY(prepare_tc_factor());
    const int ngroups = (nrhs + kP - 1) / kP;
    const long long ntasks = (long long)f->ntiles * ngroups;
    DevBuf tmp, tasks, ctr;
    IE_TRY(tmp.alloc(sizeof(float) * (size_t)f->xtotal * nrhs, s));
    IE_TRY(tasks.alloc(sizeof(FTask) * (size_t)std::max<long long>(ntasks, 1), s));
    IE_TRY(ctr.alloc(sizeof(int) * 2, s));  // next, done (one counter: no dependencies)
    IE_TRY_CUDA(cudaMemsetAsync(ctr.ptr, 0, sizeof(int) * 2, s));
    apply_tasks_kernel<<<nb, 128, 0, s>>>(f->d_npad, f->d_n, f->d_loff, f->d_xoff, f->d_tile_off,
                                          (const float *)f->d_pool, xh, tmp.as<float>(), f->xtotal, nrhs, ngroups,
                                          tasks.as<FTask>());
    IE_LAUNCHED();
    int *c = ctr.as<int>();
    const int grid = (int)std::max<long long>(1, std::min<long long>(ntasks, (long long)f->prob->sm_count * 2));
    // a GEMM that gives up waiting for its MMAs records it in the problem's error word, which
    // pcg_solve reports (the tensor-core matvec uses the same word)
    factor_persistent<<<grid, 256, kFSmem, s>>>(tasks.as<FTask>(), (int)ntasks, c, c + 1, nullptr, nullptr, nullptr,
                                                f->d_loff, nullptr, f->d_npad, f->d_info, f->prob->d_err);
    IE_LAUNCHED();
    apply_widen_kernel<<<dim3(nb, nrhs), 256, 0, s>>>(tmp.as<float>(), f->d_n, f->part->d_offs, f->d_xoff, xe, f->xtotal,
                                                      f->part->total, nb, zbuf);
    IE_LAUNCHED();
    return IE_OK;
}
