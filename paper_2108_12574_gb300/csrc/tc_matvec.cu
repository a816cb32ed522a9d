// The batched-RHS matvecs on the 5th-generation tensor cores (tcgen05, sm_103a): K1w (below)
// for grids of n = 32, 64 or a multiple of 128, whose tiles come from the exact per-offset table,
// and K1t for the other sizes.
//
// K1t.  For a batch of right-hand sides the matvec is a dense contraction: a CTA owns 128 target rows
// and 64 right-hand sides; for each chunk of 32 source points it evaluates the 128 x 32 entry
// tile E (SFU rsqrt / log2, as K1), split into TF32 high and low parts, while a bulk
// asynchronous copy (cp.async.bulk, mbarrier complete_tx) brings the matching 64 x 32 slice of
// x, split once per matvec by xsplit_kernel.  One thread issues 12 tcgen05.mma.kind::tf32
// (M = 128, N = 64, K = 8; 3xTF32: E_hi x_hi + E_hi x_lo + E_lo x_hi) into an FP32 accumulator in
// tensor memory (64 TMEM columns).  Two operand stages let the CTA build chunk c + 1 while the
// MMAs of chunk c run; every 8 chunks the accumulator is read (tcgen05.ld 32x32b) and added to a
// compensated (TwoSum) FP32 pair per output, which keeps the sum at FP32-entry accuracy.
// Completion is tracked with tcgen05.commit on per-stage mbarriers, with bounded waits: a CTA
// that waits too long records an error code, frees its TMEM and returns.
//
// Shared-memory operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, element (r, k) at (r / 8) * SBO + (k / 4) * LBO + (r % 8) * 16 + (k % 4) * 4 bytes,
// LBO = 128 (next 4 K elements), SBO = 1024 (next 8 rows, K = 32 per chunk).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>

#include "iedd_internal.cuh"

namespace {

constexpr int kTM = 128, kTN = 64, kTK = 32;
constexpr uint32_t kLBO = 128, kSBO = (kTK / 4) * 128;
constexpr long long kSpinLimit = 1LL << 24;  // non-blocking mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; base offset 0, no swizzle
    return d;
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major, N = 64 (or 128), M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
constexpr uint32_t kIdesc128 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((2 * kTN) >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                         uint32_t idesc = kIdesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// one suspending probe: the thread may sleep up to ~1 us in hardware while the phase is pending
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

// bounded wait for the given phase of the barrier; false if the limit ran out (a few seconds)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (long long i = 0; i < kSpinLimit / 8; ++i)
        if (mbar_try(bar, phase)) return true;
    return false;
}

// x pre-split for the tensor-core matvec: for right-hand-side group g (64 columns) and source
// chunk c (32 points) one 16 KB record: the 64 x 32 TF32 high parts, then the low parts, both
// in the core-matrix layout of a K-major B operand.  One pass over x per matvec.
__global__ void xsplit_kernel(const double *__restrict__ x, long long ldx, int nrhs, long long N, int nchunks,
                              uint32_t *__restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (g, c, slot)
    const long long per = (long long)kTN * kTK;
    const long long rec = e / per;
    if (rec >= (long long)nchunks * ((nrhs + kTN - 1) / kTN)) return;
    const int slot = (int)(e % per);
    const int g = (int)(rec / nchunks), c = (int)(rec % nchunks);
    // slot -> core matrix cm and position l inside it (the layout order of the record)
    const int cm = slot >> 5, l = slot & 31;
    const int col = (cm / (kTK / 4)) * 8 + (l >> 2);   // right-hand side within the group
    const int k = (cm % (kTK / 4)) * 4 + (l & 3);       // source within the chunk
    const long long j = (long long)c * kTK + k;
    const int r = g * kTN + col;
    const float v = (j < N && r < nrhs) ? (float)x[(long long)r * ldx + j] : 0.f;
    const uint32_t hi = to_tf32(v);
    const uint32_t lo = to_tf32(v - __uint_as_float(hi));
    uint32_t *o = out + rec * 2 * per;
    o[slot] = hi;
    o[per + slot] = lo;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void two_sum_acc(float v, float &hi, float &lo) {
    const float s = __fadd_rn(hi, v);
    const float bp = __fsub_rn(s, hi);
    const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
    hi = s;
    lo = __fadd_rn(lo, er);
}

constexpr int kStage = 2 * kTM * kTK + 2 * kTN * kTK;  // uint32 words per operand stage (48 KB)
constexpr int kStages = 2;                             // operand stages (96 KB, two CTAs per SM)
constexpr int kFlush = 256 / kTK;                      // chunks accumulated in TMEM between flushes

// K1t serves the grids K1w does not take (n not 32, 64 or a multiple of 128): its entries come
// from the SFU as in K1.  Pipeline (one CTA = 128 rows x 64 right-hand sides x a range of chunks,
// two CTAs per SM): two operand stages; chunk c's entries are built while chunk c - 1's MMAs run.
// A stage is reused only after the commit of its previous MMAs was waited for (by one thread, with
// a suspending try_wait; the block barrier releases the others).
template <int DIM>
__global__ void __launch_bounds__(256, 2)
k1t_matvec_tc(const float4 *__restrict__ coord, const uint32_t *__restrict__ xsplit, int nrhs, long long N,
              int chunks_per_split, int nchunks, double *__restrict__ partial, int *__restrict__ err) {
    extern __shared__ __align__(128) uint32_t opnd[];  // kStages x [A hi | A lo | B hi | B lo]
    __shared__ float4 rc[kTM];
    __shared__ __align__(8) uint64_t mbar_mma[kStages];
    __shared__ __align__(8) uint64_t mbar_ld[kStages];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long row0 = (long long)blockIdx.x * kTM;
    const int grp = blockIdx.z;
    const int rhs0 = grp * kTN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar_mma[st])), "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar_ld[st])), "r"(1u));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (tid < kTM) {
        const long long i = row0 + tid;
        rc[tid] = i < N ? coord[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    // epilogue ownership: warp w reads TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..
    const int q = warp & 3, h = warp >> 2;
    float ahi[32], alo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) { ahi[c] = 0.f; alo[c] = 0.f; }

    const int k0 = blockIdx.y * chunks_per_split;
    const int k1 = min(k0 + chunks_per_split, nchunks);
    // per stage: phase parities, and whether a commit (MMAs) or a copy (B) is outstanding; the
    // flags are uniform over the block, only thread 0 waits
    uint32_t ph_mma[kStages], ph_ld[kStages];
    int pend_mma[kStages], pend_ld[kStages];
#pragma unroll
    for (int st = 0; st < kStages; ++st) { ph_mma[st] = 0u; ph_ld[st] = 0u; pend_mma[st] = 0; pend_ld[st] = 0; }
    int since_flush = 0;

    auto wait_mma = [&](int st) {  // the stage's last MMAs have completed (bounded, thread 0)
        if (pend_mma[st]) {
            if (tid == 0 && !mbar_wait(smem_u32(&mbar_mma[st]), ph_mma[st])) abort_flag = 1;
            ph_mma[st] ^= 1u;
            pend_mma[st] = 0;
        }
    };
    auto issue_b = [&](int c) {  // B operand of chunk c (pre-split x) into its stage, thread 0
        const int st = (c - k0) % kStages;
        if (tid == 0) {
            const uint32_t *src = xsplit + ((long long)grp * nchunks + c) * (2LL * kTN * kTK);
            bulk_g2s(smem_u32(opnd + st * kStage + 2 * kTM * kTK), src, (uint32_t)(2 * kTN * kTK * sizeof(uint32_t)),
                     smem_u32(&mbar_ld[st]));
        }
        pend_ld[st] = 1;
    };
    auto flush = [&](void) {
        // all MMAs issued so far have completed (caller waited); read and add to (hi, lo)
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 32; ++c) two_sum_acc(__uint_as_float(v[c]), ahi[c], alo[c]);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };
    // element e = tid + 256 it of a part in core-matrix order (RG = kTK / 4 core-matrix columns per
    // row group) is row (64 / RG) it + 8 (warp / RG) + lane / 4 of source column 4 (warp % RG) + lane % 4
    constexpr int RG = kTK / 4, kRowStep = 64 / RG, kIters = kTM * kTK / 256;
    const int kk = 4 * (warp % RG) + (lane & 3);
    const int rbase = 8 * (warp / RG) + (lane >> 2);
    for (int ch = k0; ch < k1; ++ch) {  // abort_flag is acted on only after a barrier (uniform exit)
        const int ci = ch - k0, st = ci % kStages;
        uint32_t *Ahi = opnd + st * kStage, *Alo = Ahi + kTM * kTK, *Bv = Ahi + 2 * kTM * kTK;
        wait_mma(st);  // the stage's previous MMAs (chunk ch - 2) are done before its operands change
        __syncthreads();
        if (abort_flag) break;
        if (since_flush == kFlush) {
            for (int s2 = 0; s2 < kStages; ++s2) wait_mma(s2);
            __syncthreads();
            if (abort_flag) break;
            flush();
            __syncthreads();
            since_flush = 0;
        }
        issue_b(ch);
        // A operand of chunk ch
        const long long j = (long long)ch * kTK + kk;
        {
            const float4 b = j < N ? coord[j] : make_float4(1e6f, 1e6f, 1e6f, 0.f);
#pragma unroll 4
            for (int it = 0; it < kIters; ++it) {
                const float4 a = rc[kRowStep * it + rbase];
                const float dx = a.x - b.x, dy = a.y - b.y;
                float v;
                if (DIM == 2) {
                    v = __log2f(fmaf(dx, dx, fmaf(dy, dy, 0x1p-30f)));
                } else {
                    const float dz = a.z - b.z;
                    v = rsqrtf(fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), 1.0f));
                }
                const uint32_t hi = to_tf32(v);
                Ahi[tid + 256 * it] = hi;
                Alo[tid + 256 * it] = to_tf32(v - __uint_as_float(hi));
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0) {
            const bool ok = mbar_wait(smem_u32(&mbar_ld[st]), ph_ld[st]);
            if (!ok) {
                abort_flag = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ahi_ = smem_u32(Ahi), alo_ = smem_u32(Alo);
                const uint32_t bhi = smem_u32(Bv), blo = bhi + kTN * kTK * 4;
#pragma unroll
                for (int s = 0; s < kTK / 8; ++s) {
                    const uint32_t koff = (uint32_t)s * 2 * kLBO;
                    mma_tf32(tmem, make_desc(ahi_ + koff), make_desc(bhi + koff), (since_flush > 0 || s > 0) ? 1u : 0u);
                    mma_tf32(tmem, make_desc(ahi_ + koff), make_desc(blo + koff), 1u);
                    mma_tf32(tmem, make_desc(alo_ + koff), make_desc(bhi + koff), 1u);
                }
                mma_commit(smem_u32(&mbar_mma[st]));
            }
        }
        ph_ld[st] ^= 1u;
        pend_ld[st] = 0;
        pend_mma[st] = 1;
        ++since_flush;
    }
    // drain (bounded): outstanding MMAs and any B copies still in flight after an early exit
    for (int st = 0; st < kStages; ++st) {
        wait_mma(st);
        if (pend_ld[st]) {
            if (tid == 0 && !mbar_wait(smem_u32(&mbar_ld[st]), ph_ld[st])) abort_flag = 1;
            pend_ld[st] = 0;
        }
    }
    __syncthreads();
    if (!abort_flag && since_flush > 0) flush();
    if (!abort_flag) {
        const long long i = row0 + 32 * q + lane;
        if (i < N) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int r = rhs0 + 32 * h + c;
                if (r < nrhs) partial[((long long)blockIdx.y * nrhs + r) * N + i] = (double)ahi[c] + (double)alo[c];
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTN));
    }
}

// K1w: the batched matvec for grids whose lines tile the 256-row blocks (n = 32, 64 or a multiple
// of 128), with exact table entries split into TF32 high / low words and 3xTF32 products (hi hi,
// hi lo, lo hi).  The B record's low rows follow its high rows at the same stride, so per K-step
// one N = 128 MMA gives hi hi (level 0, columns 0-63) and hi lo (level 1, columns 64-127) and a
// second adds lo hi to level 1.
//
// A CTA owns a block of 256 targets (two M = 128 tiles sharing every B record: the copies, not the
// MMAs, bound this kernel, and the B record is two thirds of them) and 64 right-hand sides.
//
// A operand from a Toeplitz strip.  The block holds nb = 256 / Lb grid lines of Lb = min(n, 256)
// targets; block row mb (tile mb / 128, MMA row mb % 128) is line q = mb % nb, target f0 + Lb - 1
// - mb / nb along it (reversed), so against the chunk's 32 sources j = fj + k of one source line
// the entry depends on (mb / nb) + k only: t(.., |f0 + Lb - 1 - fj - (mb / nb + k)|).  The strip
// table (built once per problem) holds, per plane, per slow-axis offset and per row rho, the 4
// consecutive entries t(.., |n - 1 - rho - k'|), k' < 4, of every signed offset along the
// interleaved axis (the mid axis in 3D, the slow axis in 2D, on which the block's nb lines are
// consecutive).  One 4D TMA copy brings rows rho0 .. rho0 + Lb + 27 of the nb consecutive offsets
// into shared memory as [row][line][4 entries] (one line, n >= 256: a bulk copy per plane of its
// contiguous rows), so block row mb of K-group g sits at 16 ((mb / nb + 4 g) nb + mb % nb) = 16 mb
// + 64 nb g bytes: K-major descriptors with SBO = 128 and LBO = 64 nb read each tile's 128 x 8
// operand of a K-step straight from the strip (core matrices overlap).  A chunk's strip is
// 2 x 16 nb (Lb + 28) bytes (<= 15 KB) for 256 targets.
//
// Roles: warp 0 issues the MMAs (one lane), warp 1 the copies (one lane: the strip, the pre-split
// B record by a bulk copy, all completing one mbarrier), warps 2-9 fold finished accumulator sets
// (levels 0 + 1, FP32 over 8 chunks) into running (high, low) sums kept in tensor memory (one tile
// and TMEM lane quarter each).  Seven operand stages; one accumulator set per tile (TMEM: tile t
// at columns 256 t: the set, then the high and the low running sums), so the MMAs of a window
// wait for the fold of the previous one; mbarriers hand over; every wait is bounded.
constexpr int kWStages = 7, kWThreads = 320, kWWin = 8, kWBM = 256, kWFold = 8;
constexpr int kWStripMax = 2 * 8 * (32 + 28) * 16;             // strip bytes, both planes, at most (nb = 8)
constexpr int kWBBytes = 2 * kTN * kTK * (int)sizeof(uint32_t); // B record: 16 KB
constexpr int kWStage = kWStripMax + kWBBytes;                  // 31,744 bytes (248 x 128)
constexpr int kWSmem = kWStages * kWStage;                      // 222,208 bytes
constexpr long long kStripCap = 1LL << 30;                      // largest strip table (bytes)

__device__ __forceinline__ uint64_t make_desc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void tmem_ld16w(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16w(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// Strip table entries: plane pl (0: TF32 high, 1: low) of the entry at lattice offset (fast
// |n - 1 - rho - k'|, interleaved axis |qq - (n - 1)|, slow o in 3D), 0 outside the grid; Q = R =
// 2n values of qq and rho (the last one padding).  Layout [pl][o][rho][qq][k'] when a block holds
// several lines (the TMA box interleaves them), [pl][o][qq][rho][k'] when it holds one (each plane
// of a chunk's strip is then one contiguous run, fetched by a bulk copy).
__global__ void tc_strip_kernel(const uint2 *__restrict__ tab, int dim, int n, int interleaved, uint4 *__restrict__ strip) {
    const long long Q = 2LL * n, R = 2LL * n, O = dim == 3 ? n : 1;
    const long long rows = 2 * O * R * Q;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows) return;
    const int qq = interleaved ? (int)(e % Q) : (int)((e / R) % Q);
    const int rho = interleaved ? (int)((e / Q) % R) : (int)(e % R);
    const int o = (int)((e / (Q * R)) % O), pl = (int)(e / (Q * R * O));
    const int di = abs(qq - (n - 1));
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int df = abs(n - 1 - rho - k);
        v[k] = 0u;
        if (df < n && di < n) {
            const uint2 t = tab[dim == 3 ? ((long long)o * n + di) * n + df : (long long)di * n + df];
            v[k] = pl ? t.y : t.x;
        }
    }
    strip[e] = make_uint4(v[0], v[1], v[2], v[3]);
}

template <int DIM>
__global__ void __launch_bounds__(kWThreads, 1)
k1w_matvec_tc(const __grid_constant__ CUtensorMap smap, const unsigned char *__restrict__ strip,
              const uint32_t *__restrict__ xsplit, int nrhs, long long N, int chunks_per_split, int nchunks,
              double *__restrict__ partial, int *__restrict__ err, int n, int Lb) {
    extern __shared__ __align__(128) unsigned char wsm[];  // kWStages x [strip hi | strip lo | pad | B hi | B lo]
    __shared__ __align__(8) uint64_t full[kWStages], mdone[kWStages], afull, aempty;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long blk0 = (long long)blockIdx.x * kWBM;
    const int grp = blockIdx.z;
    const int k0 = blockIdx.y * chunks_per_split;
    const int T = max(0, min(chunks_per_split, nchunks - k0));
    const int nb = kWBM / Lb;
    const uint32_t plane_bytes = (uint32_t)(16 * nb * (Lb + 28));

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < kWStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[st])), "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mdone[st])), "r"(1u));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull)), "r"(1u));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&aempty)), "r"((uint32_t)kWFold));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    auto wait_bar = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (long long i = 0; i < kSpinLimit / 8; ++i) {
            if (mbar_try(smem_u32(bar), parity)) return true;
            if (abort_flag) return false;
        }
        abort_flag = 1;
        return false;
    };
    auto warp_wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        int ok = 1;
        if (lane == 0) ok = wait_bar(bar, parity) ? 1 : 0;
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    if (warp == 0) {
        // ---- MMA issue (one lane): per chunk 4 K-steps x 2 tiles x (hi [hi | lo], lo hi) ----
        if (lane == 0) {
            const uint32_t lbo_a = 64u * (uint32_t)nb;
            int issued = 0;
            for (int c = 0; c < T; ++c) {
                const int st = c % kWStages, f = c / kWWin;
                const uint32_t spar = (uint32_t)(c / kWStages) & 1u;
                if (!wait_bar(&full[st], spar)) break;
                // a window's first MMAs overwrite the accumulators: the previous fold must be done
                if (c % kWWin == 0 && f >= 1 && !wait_bar(&aempty, (uint32_t)(f - 1) & 1u)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ahi = smem_u32(wsm + st * kWStage), alo = ahi + plane_bytes;
                const uint32_t bhi = ahi + kWStripMax;
#pragma unroll
                for (int s = 0; s < kTK / 8; ++s) {
                    const uint64_t db = make_desc(bhi + (uint32_t)s * 2 * kLBO);
                    const uint32_t acc = (c % kWWin == 0 && s == 0) ? 0u : 1u;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const uint32_t toff = (uint32_t)t * (16u * kTM) + 2u * s * lbo_a;  // tile t's rows
                        const uint32_t dt = tmem + (uint32_t)t * 256u;
                        mma_tf32(dt, make_desc2(ahi + toff, lbo_a, 128u), db, acc, kIdesc128);
                        mma_tf32(dt + kTN, make_desc2(alo + toff, lbo_a, 128u), db, 1u);
                    }
                }
                mma_commit(smem_u32(&mdone[st]));
                if (c % kWWin == kWWin - 1 || c == T - 1) mma_commit(smem_u32(&afull));
                issued = c + 1;
            }
            if (issued > 0 && !mbar_wait(smem_u32(&mdone[(issued - 1) % kWStages]), (uint32_t)((issued - 1) / kWStages) & 1u))
                abort_flag = 1;  // (a wait that ignores the abort flag: the TMEM must be idle)
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- operands of a chunk: the strip (several lines: one TMA copy of the 4D box (4 nb,
        // Lb + 28, 1, 2); one line: a bulk copy per plane) and the B record ----
        if (lane == 0) {
            // the block's first target: slow, mid (3D) and fast coordinates
            const int f0 = (int)(blk0 % n);
            const int i_mid = DIM == 3 ? (int)((blk0 / n) % n) : 0;
            const int i_slow = DIM == 3 ? (int)(blk0 / ((long long)n * n)) : (int)(blk0 / n);
            const uint32_t bytes = 2u * plane_bytes + (uint32_t)kWBBytes;
            int issued = 0;
            for (int c = 0; c < T; ++c) {
                const int st = c % kWStages;
                const uint32_t spar = (uint32_t)(c / kWStages) & 1u;
                if (c >= kWStages && !wait_bar(&mdone[st], spar ^ 1u)) break;
                const long long j0 = (long long)(k0 + c) * kTK;  // the chunk's first source
                const int fj = (int)(j0 % n);
                const long long tj = j0 / n;
                const int mj = DIM == 3 ? (int)(tj % n) : 0;
                const int sj = DIM == 3 ? (int)(tj / n) : (int)tj;
                const int o = DIM == 3 ? abs(i_slow - sj) : 0;
                const int q0 = (DIM == 3 ? i_mid - mj : i_slow - sj) + (n - 1);
                const int rho0 = n - f0 - Lb + fj;
                const uint32_t bar = smem_u32(&full[st]), dst = smem_u32(wsm + st * kWStage);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
                if (nb > 1) {
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(&smap)), "r"(4 * q0), "r"(rho0), "r"(o), "r"(0), "r"(bar)
                        : "memory");
                } else {
                    const long long O = DIM == 3 ? n : 1;
                    for (int pl = 0; pl < 2; ++pl) {
                        const unsigned char *src = strip + ((((long long)pl * O + o) * (2 * n) + q0) * (2 * n) + rho0) * 16;
                        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                         dst + (uint32_t)pl * plane_bytes),
                                     "l"(src), "r"(plane_bytes), "r"(bar)
                                     : "memory");
                    }
                }
                const uint32_t *src = xsplit + ((long long)grp * nchunks + k0 + c) * (2LL * kTN * kTK);
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                 dst + (uint32_t)kWStripMax),
                             "l"(src), "r"((uint32_t)kWBBytes), "r"(bar)
                             : "memory");
                issued = c + 1;
            }
            // no copy may still be landing when the CTA ends (waits that ignore the abort flag)
            for (int c = max(0, issued - kWStages); c < issued; ++c)
                if (!mbar_wait(smem_u32(&full[c % kWStages]), (uint32_t)(c / kWStages) & 1u)) abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ---- tile t's accumulator set into running (high, low) sums in TMEM columns 256 t + 128 ..
        // and 256 t + 192 .. ----
        const int q4 = warp & 3, t = (warp - 2) >> 2;
        const uint32_t lanes = (uint32_t)(32 * q4) << 16, col0 = (uint32_t)t * 256u;
        {
            uint32_t z[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = 0u;
#pragma unroll
            for (int b = 0; b < kTN / 16; ++b) {
                tmem_st16w(tmem + lanes + col0 + 128u + 16u * b, z);
                tmem_st16w(tmem + lanes + col0 + 192u + 16u * b, z);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        const int nwin = (T + kWWin - 1) / kWWin;
        for (int f = 0; f < nwin; ++f) {
            if (!warp_wait(&afull, (uint32_t)f & 1u)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int b = 0; b < kTN / 16; ++b) {
                uint32_t a[16], a1[16], h[16], l[16];
                tmem_ld16w(tmem + lanes + col0 + 16u * b, a);
                tmem_ld16w(tmem + lanes + col0 + kTN + 16u * b, a1);
                tmem_ld16w(tmem + lanes + col0 + 128u + 16u * b, h);
                tmem_ld16w(tmem + lanes + col0 + 192u + 16u * b, l);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (b == kTN / 16 - 1) {  // every read of this set is complete: release it
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&aempty)) : "memory");
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    float hi = __uint_as_float(h[k]), lo = __uint_as_float(l[k]);
                    two_sum_acc(__uint_as_float(a[k]) + __uint_as_float(a1[k]), hi, lo);
                    h[k] = __float_as_uint(hi);
                    l[k] = __float_as_uint(lo);
                }
                tmem_st16w(tmem + lanes + col0 + 128u + 16u * b, h);
                tmem_st16w(tmem + lanes + col0 + 192u + 16u * b, l);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        // TMEM lane m of tile t is block row mb = 128 t + m: line mb % nb, target Lb - 1 - mb / nb
        const int mb = 128 * t + 32 * q4 + lane;
        const long long i = blk0 + (long long)(mb % nb) * Lb + (Lb - 1 - mb / nb);
        if (!abort_flag) {
#pragma unroll
            for (int b = 0; b < kTN / 16; ++b) {
                uint32_t h[16], l[16];
                tmem_ld16w(tmem + lanes + col0 + 128u + 16u * b, h);
                tmem_ld16w(tmem + lanes + col0 + 192u + 16u * b, l);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (i < N) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int r = grp * kTN + 16 * b + k;
                        if (r < nrhs)
                            partial[((long long)blockIdx.y * nrhs + r) * N + i] =
                                (double)__uint_as_float(h[k]) + (double)__uint_as_float(l[k]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(err, 1);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
}

}  // namespace

// y partials for nrhs >= 1 right-hand sides through the tensor cores; returns IE_ERR_TIMEOUT
// (after the launch completes) if a CTA gave up waiting for its MMAs.
int launch_matvec_tc(const ie_problem *p, const double *x, long long ldx, int nrhs, double *partial, int S, int cps,
                     int nchunks, int *d_err, cudaStream_t s) {
    const int rt = (int)((p->N + kTM - 1) / kTM);
    const int groups = (nrhs + kTN - 1) / kTN;
    DevBuf xs;
    const long long words = (long long)groups * nchunks * 2 * kTN * kTK;
    IE_TRY(xs.alloc(sizeof(uint32_t) * words, s));
    xsplit_kernel<<<(unsigned)((words / 2 + 255) / 256), 256, 0, s>>>(x, ldx, nrhs, p->N, nchunks, xs.as<uint32_t>());
    IE_LAUNCHED();
    const dim3 g(rt, S, groups);
    const size_t dsm = sizeof(uint32_t) * kStages * kStage;
    if (tc_toeplitz(p)) {
        const dim3 gw((unsigned)((p->N + kWBM - 1) / kWBM), S, groups);
        if (!p->d_tc_strip) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            IE_TRY_CUDA(cudaStreamIsCapturing(s, &cs));
            if (cs != cudaStreamCaptureStatusNone) {
                ie_set_error("ie_matvec: the first IE_TENSOR call on a problem builds its strip table and must not be captured");
                return IE_ERR_ARG;
            }
            IE_TRY(prepare_tc_strip(p));
        }
        auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encode_fn());
        if (!encode) {
            ie_set_error("ie_matvec: cuTensorMapEncodeTiled is not available from the driver");
            return IE_ERR_CUDA;
        }
        const int n = p->n, Lb = std::min(n, kWBM), nb = kWBM / Lb;
        CUtensorMap smap;
        std::memset(&smap, 0, sizeof(smap));
        if (nb > 1) {
            // the interleaved strip table [plane][slow offset][rho][signed interleaved offset x 4
            // entries] of TF32 words; a box is 4 nb words x (Lb + 28) rows x both planes
            const cuuint64_t O = p->dim == 3 ? (cuuint64_t)n : 1, Q = 2 * (cuuint64_t)n, R = 2 * (cuuint64_t)n;
            const cuuint64_t gdim[4] = {4 * Q, R, O, 2};
            const cuuint64_t gstride[3] = {Q * 16, R * Q * 16, O * R * Q * 16};
            const cuuint32_t box[4] = {(cuuint32_t)(4 * nb), (cuuint32_t)(Lb + 28), 1, 2};
            const cuuint32_t estride[4] = {1, 1, 1, 1};
            const CUresult cr = encode(&smap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, p->d_tc_strip, gdim, gstride, box, estride,
                                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (cr != CUDA_SUCCESS) {
                ie_set_error("ie_matvec: cuTensorMapEncodeTiled failed for the strip table (" + std::to_string((int)cr) + ")");
                return IE_ERR_CUDA;
            }
        }
        const unsigned char *strip = static_cast<const unsigned char *>(p->d_tc_strip);
        if (p->dim == 2)
            k1w_matvec_tc<2><<<gw, kWThreads, kWSmem, s>>>(smap, strip, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial,
                                                           d_err, n, Lb);
        else
            k1w_matvec_tc<3><<<gw, kWThreads, kWSmem, s>>>(smap, strip, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial,
                                                           d_err, n, Lb);
    } else if (p->dim == 2) {
        k1t_matvec_tc<2><<<g, 256, dsm, s>>>(p->d_coord, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial, d_err);
    } else {
        k1t_matvec_tc<3><<<g, 256, dsm, s>>>(p->d_coord, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial, d_err);
    }
    IE_LAUNCHED();
    return IE_OK;
}

// The strip-fed variant applies when n is a multiple of 32, 256 rows are whole lines (n = 32, 64,
// 128) or part of one (n a multiple of 256), and the strip table (128 n^3 bytes in 3D, 128 n^2 in
// 2D) is at most 1 GiB.
bool tc_toeplitz(const ie_problem *p) {
    const long long n = p->n;
    const long long bytes = 128LL * n * n * (p->dim == 3 ? n : 1);
    return p->d_table_tc && n % 32 == 0 && (n >= kWBM ? n % kWBM == 0 : kWBM % n == 0) && bytes <= kStripCap;
}

// The strip table of K1w (once per problem, on first use; synchronizes)
int prepare_tc_strip(const ie_problem *p_) {
    ie_problem *p = const_cast<ie_problem *>(p_);
    if (p->d_tc_strip || !tc_toeplitz(p)) return IE_OK;
    const long long n = p->n, rows = 2LL * (p->dim == 3 ? n : 1) * (2 * n) * (2 * n);
    IE_TRY_CUDA(cudaMalloc(&p->d_tc_strip, sizeof(uint4) * rows));
    tc_strip_kernel<<<(unsigned)((rows + 255) / 256), 256>>>(p->d_table_tc, p->dim, p->n, p->n < kWBM ? 1 : 0,
                                                              static_cast<uint4 *>(p->d_tc_strip));
    IE_LAUNCHED();
    IE_TRY_CUDA(cudaDeviceSynchronize());
    return IE_OK;
}

// Per |offset| q: the exact entry (FP64 table; 0 at q = 0, the diagonal being added in FP64) split
// into TF32 high and low words.
__global__ void tc_table_kernel(const double *__restrict__ t64, long long T, uint2 *__restrict__ out) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= T) return;
    const float v = q == 0 ? 0.f : (float)t64[q];
    const float r = q == 0 ? 0.f : (float)(t64[q] - (double)v);
    const uint32_t hi = to_tf32(v);
    // low word: the rest of the FP64 value below the TF32 high part
    out[q] = make_uint2(hi, to_tf32((v - __uint_as_float(hi)) + r));
}

int build_tc_table(ie_problem *p) {
    const long long T = p->N;
    IE_TRY_CUDA(cudaMalloc(&p->d_table_tc, sizeof(uint2) * T));
    tc_table_kernel<<<(unsigned)((T + 255) / 256), 256>>>(p->d_table64, T, p->d_table_tc);
    IE_LAUNCHED();
    return IE_OK;
}

// source splits of the warp-specialized kernel (one CTA per SM): the smallest modelled time
// ceil(CTAs / SMs) x (chunks per CTA + 8 for a CTA's setup and final write)
int tc_splits_toeplitz(long long tiles, int nchunks, int sms) {
    int best = 1;
    long long best_cost = -1;
    for (int s = 1; s <= 64 && s <= nchunks; ++s) {
        const long long cps = (nchunks + s - 1) / s;
        const long long cost = (tiles * s + sms - 1) / sms * (cps + 8);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = s; }
    }
    return best;
}

int tc_chunk() { return kTK; }
int tc_rows() { return kTM; }
int tc_block_rows() { return kWBM; }
int tc_cols() { return kTN; }

int prepare_tc() {
    const int dsm = (int)(sizeof(uint32_t) * kStages * kStage);
    IE_TRY_CUDA(cudaFuncSetAttribute(k1t_matvec_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1t_matvec_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1w_matvec_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1w_matvec_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem));
    return IE_OK;
}
