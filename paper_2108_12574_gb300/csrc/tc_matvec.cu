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
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

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

// K1w: the table-fed batched matvec with warp roles (n = 32, 64 or a multiple of 128).  The products are K1t's (A tiles of
// exact table entries split into TF32 high / low words, the same pre-split B operand: hi hi,
// hi lo and lo hi), but the B record's low rows follow its high rows at the same stride, so per
// K-step one N = 128 MMA gives hi hi (level 0, columns 0-63) and hi lo (level 1, columns 64-127)
// and a second adds lo hi to level 1: 8 MMAs per 32-source chunk instead of 12.  No block-wide
// barrier couples the roles: one lane issues the MMAs (warp 0), one the bulk copy of each chunk's
// B operand (warp 1), six warps write the A tiles (warps 2-7), and four warps fold finished
// accumulator sets (levels 0 + 1, FP32 over 8 chunks) into running (high, low) sums kept in
// tensor memory (warps 8-11, one TMEM lane quarter each).  Four operand stages, two accumulator
// sets of 128 columns; mbarriers hand over; every wait is bounded.
constexpr int kWStages = 4, kWThreads = 384, kWWin = 8, kWFillWarps = 6;
constexpr int kWSmem = kWStages * kStage * (int)sizeof(uint32_t);  // 192 KB
constexpr int kWSlots = 2;  // staged entries per fill thread (nl (Lr + 31) <= 252 <= 2 x 192)

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

template <int DIM>
__global__ void __launch_bounds__(kWThreads, 1)
k1w_matvec_tc(const float4 *__restrict__ coord, const uint32_t *__restrict__ xsplit, int nrhs, long long N,
              int chunks_per_split, int nchunks, double *__restrict__ partial, int *__restrict__ err,
              const uint2 *__restrict__ ttab, int n, int Lr) {
    extern __shared__ __align__(128) uint32_t opnd[];  // kWStages x [A hi | A lo | B hi | B lo]
    constexpr int kPer = kTM + kTK - 1;
    __shared__ uint2 tval[2][kTM / 32 * kPer];          // a chunk's distinct entries, double-buffered
    __shared__ int4 rline[kTM / 32];                    // slow, mid, fast coordinate of target line q
    __shared__ __align__(8) uint64_t sfull[kWStages], bfull[kWStages], mdone[kWStages], afull[2], aempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long row0 = (long long)blockIdx.x * kTM;
    const int grp = blockIdx.z;
    const int k0 = blockIdx.y * chunks_per_split;
    const int T = max(0, min(chunks_per_split, nchunks - k0));
    const int nl = kTM / Lr, per = Lr + kTK - 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < kWStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sfull[st])), "r"((uint32_t)kWFillWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bfull[st])), "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mdone[st])), "r"(1u));
        }
        for (int st = 0; st < 2; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull[st])), "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&aempty[st])), "r"(4u));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (tid < nl) {
        const float4 c = coord[row0 + (long long)tid * Lr];
        rline[tid] = DIM == 2 ? make_int4((int)c.x, 0, (int)c.y, 0) : make_int4((int)c.x, (int)c.y, (int)c.z, 0);
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
        // ---- MMA issue (one lane): per chunk 4 K-steps x (hi hi, hi lo, lo hi) ----
        if (lane == 0) {
            int issued = 0;
            for (int c = 0; c < T; ++c) {
                const int st = c % kWStages, f = c / kWWin, set = f & 1;
                const uint32_t spar = (uint32_t)(c / kWStages) & 1u, fpar = (uint32_t)(f >> 1) & 1u;
                if (!wait_bar(&sfull[st], spar) || !wait_bar(&bfull[st], spar)) break;
                if (c % kWWin == 0 && f >= 2 && !wait_bar(&aempty[set], fpar ^ 1u)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ahi = smem_u32(opnd + st * kStage), alo = ahi + kTM * kTK * 4;
                const uint32_t bhi = ahi + 2 * kTM * kTK * 4, blo = bhi + kTN * kTK * 4;
                const uint32_t dt = tmem + (uint32_t)set * (2 * kTN);
                (void)blo;
#pragma unroll
                for (int s = 0; s < kTK / 8; ++s) {
                    const uint32_t koff = (uint32_t)s * 2 * kLBO;
                    // [hi hi | hi lo] over the high then low rows of B, then lo hi into level 1
                    mma_tf32(dt, make_desc(ahi + koff), make_desc(bhi + koff), (c % kWWin == 0 && s == 0) ? 0u : 1u,
                             kIdesc128);
                    mma_tf32(dt + kTN, make_desc(alo + koff), make_desc(bhi + koff), 1u);
                }
                mma_commit(smem_u32(&mdone[st]));
                if (c % kWWin == kWWin - 1 || c == T - 1) mma_commit(smem_u32(&afull[set]));
                issued = c + 1;
            }
            if (issued > 0 && !mbar_wait(smem_u32(&mdone[(issued - 1) % kWStages]), (uint32_t)((issued - 1) / kWStages) & 1u))
                abort_flag = 1;  // (a wait that ignores the abort flag: the TMEM must be idle)
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- B operand: one bulk copy of the pre-split x per chunk ----
        int issued = 0;
        for (int c = 0; c < T; ++c) {
            const int st = c % kWStages;
            const uint32_t spar = (uint32_t)(c / kWStages) & 1u;
            if (c >= kWStages && !warp_wait(&mdone[st], spar ^ 1u)) break;
            if (lane == 0) {
                const uint32_t *src = xsplit + ((long long)grp * nchunks + k0 + c) * (2LL * kTN * kTK);
                bulk_g2s(smem_u32(opnd + st * kStage + 2 * kTM * kTK), src, (uint32_t)(2 * kTN * kTK * sizeof(uint32_t)),
                         smem_u32(&bfull[st]));
            }
            __syncwarp();
            issued = c + 1;
        }
        if (lane == 0)  // no copy may still be landing when the CTA ends
            for (int c = max(0, issued - kWStages); c < issued; ++c)
                if (!mbar_wait(smem_u32(&bfull[c % kWStages]), (uint32_t)(c / kWStages) & 1u)) abort_flag = 1;
        __syncwarp();
    } else if (warp < 2 + kWFillWarps) {
        // ---- A tiles (192 threads); every fill warp runs every chunk and every named barrier ----
        const int ft = tid - 64;
        int sq[kWSlots], stt[kWSlots];  // staged entry e = ft + 192 i: line and position
#pragma unroll
        for (int i = 0; i < kWSlots; ++i) {
            const int e = ft + 32 * kWFillWarps * i;
            sq[i] = e < nl * per ? e / per : -1;
            stt[i] = e < nl * per ? e - sq[i] * per : 0;
        }
        uint2 tv[kWSlots];
        // coordinates of the next chunk to fetch (chunks are fetched in order, 32 sources each)
        int fj, mj, sj;
        {
            const int j0 = k0 * kTK, tj = j0 / n;
            fj = j0 % n;
            mj = DIM == 2 ? 0 : tj % n;
            sj = DIM == 2 ? tj : tj / n;
        }
        auto fetch = [&](int c) {
#pragma unroll
            for (int i = 0; i < kWSlots; ++i) {
                tv[i] = make_uint2(0u, 0u);
                if (c < T && sq[i] >= 0) {
                    const int4 L = rline[sq[i]];
                    const int df = abs(L.z - fj - (kTK - 1) + stt[i]), dm = abs(L.y - mj), ds = abs(L.x - sj);
                    tv[i] = __ldg(ttab + (DIM == 2 ? (long long)ds * n + df : ((long long)ds * n + dm) * n + df));
                }
            }
            fj += kTK;  // the next chunk
            if (fj >= n) {
                fj = 0;
                if (DIM == 2) {
                    ++sj;
                } else if (++mj >= n) {
                    mj = 0;
                    ++sj;
                }
            }
        };
        auto stage_tv = [&](int buf) {
#pragma unroll
            for (int i = 0; i < kWSlots; ++i)
                if (sq[i] >= 0) tval[buf][sq[i] * per + stt[i]] = tv[i];
        };
        fetch(0);
        stage_tv(0);
        fetch(1);
        const int lgL = __ffs(Lr) - 1;
        for (int c = 0; c < T; ++c) {
            const int st = c % kWStages;
            const uint32_t spar = (uint32_t)(c / kWStages) & 1u;
            bool ok = !abort_flag;
            if (ok && c >= kWStages) ok = warp_wait(&mdone[st], spar ^ 1u);
            asm volatile("bar.sync 1, 192;" ::: "memory");  // tval[c & 1] is complete
            if (ok) {
                uint32_t *Ahi = opnd + st * kStage, *Alo = Ahi + kTM * kTK;
                const uint2 *tb = tval[c & 1];
                // unit u = (column group g, row r): the 4 sources 4g..4g+3 of row r, one 16-byte
                // core-matrix row in each of the hi and lo planes
                for (int u = ft; u < kTM * (kTK / 4); u += 32 * kWFillWarps) {
                    const int g = u >> 7, r = u & (kTM - 1);
                    const int base = (r >> lgL) * per + (r & (Lr - 1)) + (kTK - 1) - 4 * g;
                    const uint2 w0 = tb[base], w1 = tb[base - 1], w2 = tb[base - 2], w3 = tb[base - 3];
                    const int off = (r >> 3) * (kSBO / 4) + g * (kLBO / 4) + (r & 7) * 4;
                    *reinterpret_cast<uint4 *>(Ahi + off) = make_uint4(w0.x, w1.x, w2.x, w3.x);
                    *reinterpret_cast<uint4 *>(Alo + off) = make_uint4(w0.y, w1.y, w2.y, w3.y);
                }
            }
            stage_tv((c + 1) & 1);  // the buffer was last read in chunk c - 1, before this barrier
            fetch(c + 2);
            if (ok) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&sfull[st])) : "memory");
            }
        }
    } else {
        // ---- accumulator sets into running (high, low) sums in TMEM columns 128.. and 192.. ----
        const int q4 = warp & 3;
        const uint32_t lanes = (uint32_t)(32 * q4) << 16;
        {
            uint32_t z[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = 0u;
#pragma unroll
            for (int b = 0; b < kTN / 16; ++b) {
                tmem_st16w(tmem + lanes + 256u + 16u * b, z);
                tmem_st16w(tmem + lanes + 320u + 16u * b, z);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        const int nwin = (T + kWWin - 1) / kWWin;
        for (int f = 0; f < nwin; ++f) {
            const int set = f & 1;
            if (!warp_wait(&afull[set], (uint32_t)(f >> 1) & 1u)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int b = 0; b < kTN / 16; ++b) {
                uint32_t a[16], a1[16], h[16], l[16];
                tmem_ld16w(tmem + lanes + (uint32_t)set * (2 * kTN) + 16u * b, a);
                tmem_ld16w(tmem + lanes + (uint32_t)set * (2 * kTN) + kTN + 16u * b, a1);
                tmem_ld16w(tmem + lanes + 256u + 16u * b, h);
                tmem_ld16w(tmem + lanes + 320u + 16u * b, l);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (b == kTN / 16 - 1) {  // every read of this set is complete: release it
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&aempty[set])) : "memory");
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    float hi = __uint_as_float(h[k]), lo = __uint_as_float(l[k]);
                    two_sum_acc(__uint_as_float(a[k]) + __uint_as_float(a1[k]), hi, lo);
                    h[k] = __float_as_uint(hi);
                    l[k] = __float_as_uint(lo);
                }
                tmem_st16w(tmem + lanes + 256u + 16u * b, h);
                tmem_st16w(tmem + lanes + 320u + 16u * b, l);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        const long long i = row0 + 32 * q4 + lane;
        if (!abort_flag) {
#pragma unroll
            for (int b = 0; b < kTN / 16; ++b) {
                uint32_t h[16], l[16];
                tmem_ld16w(tmem + lanes + 256u + 16u * b, h);
                tmem_ld16w(tmem + lanes + 320u + 16u * b, l);
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
    const bool toep = tc_toeplitz(p);
    const int Lr = std::min(p->n, kTM);
    if (toep && p->dim == 2)
        k1w_matvec_tc<2><<<g, kWThreads, kWSmem, s>>>(p->d_coord, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial,
                                                      d_err, p->d_table_tc, p->n, Lr);
    else if (toep)
        k1w_matvec_tc<3><<<g, kWThreads, kWSmem, s>>>(p->d_coord, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial,
                                                      d_err, p->d_table_tc, p->n, Lr);
    else if (p->dim == 2)
        k1t_matvec_tc<2><<<g, 256, dsm, s>>>(p->d_coord, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial, d_err);
    else
        k1t_matvec_tc<3><<<g, 256, dsm, s>>>(p->d_coord, xs.as<uint32_t>(), nrhs, p->N, cps, nchunks, partial, d_err);
    IE_LAUNCHED();
    return IE_OK;
}

// The Toeplitz-fed variant applies when n is a multiple of 32 and 128 rows are whole lines (n = 32,
// 64) or part of one (n a multiple of 128), and the table is built.
bool tc_toeplitz(const ie_problem *p) {
    return p->d_table_tc && p->n % 32 == 0 && (p->n >= kTM ? p->n % kTM == 0 : kTM % p->n == 0);
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
int tc_cols() { return kTN; }

int prepare_tc() {
    const int dsm = (int)(sizeof(uint32_t) * kStages * kStage);
    IE_TRY_CUDA(cudaFuncSetAttribute(k1t_matvec_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1t_matvec_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1w_matvec_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1w_matvec_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem));
    return IE_OK;
}
