// K1t: the batched-RHS matvec on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For a batch of right-hand sides the matvec is a dense contraction: a CTA owns 128 target rows
// and 64 right-hand sides; for each chunk of 32 source points it evaluates the 128 x 32 entry
// tile E (SFU rsqrt / log2, as K1) and stages the 64 x 32 slice of x, both split into TF32
// high and low parts (3xTF32: E_hi x_hi + E_hi x_lo + E_lo x_hi, FP32-class accuracy), and one
// thread issues 12 tcgen05.mma.kind::tf32 (M = 128, N = 64, K = 8) into an FP32 accumulator in
// tensor memory (64 TMEM columns).  Completion is tracked with tcgen05.commit on an mbarrier,
// with a bounded wait: a CTA that waits too long records an error code, still drains its own
// MMAs (bounded again), frees its TMEM and returns.  The epilogue reads the accumulator with
// tcgen05.ld (32x32b) and writes the same [split][rhs][N] FP64 partials as the CUDA-core kernel.
//
// Shared-memory operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, element (r, k) at (r / 8) * SBO + (k / 4) * LBO + (r % 8) * 16 + (k % 4) * 4 bytes,
// LBO = 128 (next 4 K elements), SBO = 1024 (next 8 rows, K = 32 per chunk).
#include <cuda_runtime.h>

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

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

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

// bounded wait for the given phase of the barrier; false if the limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_test(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ uint32_t op_off(int r, int k) {
    return (uint32_t)((r >> 3) * kSBO + (k >> 2) * kLBO + (r & 7) * 16 + (k & 3) * 4);
}

template <int DIM>
__global__ void __launch_bounds__(256)
k1t_matvec_tc(const float4 *__restrict__ coord, const double *__restrict__ x, long long ldx, int nrhs, long long N,
              int chunks_per_split, int nchunks, double *__restrict__ partial, int *__restrict__ err) {
    extern __shared__ __align__(128) uint32_t opnd[];  // A hi | A lo | B hi | B lo (48 KB)
    uint32_t *Ahi = opnd, *Alo = opnd + kTM * kTK, *Bhi = opnd + 2 * kTM * kTK, *Blo = Bhi + kTN * kTK;
    __shared__ float4 rc[kTM];
    __shared__ float4 cc[kTK];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long row0 = (long long)blockIdx.x * kTM;
    const int rhs0 = blockIdx.z * kTN;
    const uint32_t bar = smem_u32(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1u));
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

    const int k0 = blockIdx.y * chunks_per_split;
    const int k1 = min(k0 + chunks_per_split, nchunks);
    uint32_t phase = 0;
    bool issued_any = false;
    for (int ch = k0; ch < k1; ++ch) {
        const long long j0 = (long long)ch * kTK;
        if (tid < kTK) {
            const long long j = j0 + tid;
            cc[tid] = j < N ? coord[j] : make_float4(1e6f, 1e6f, 1e6f, 0.f);
        }
        __syncthreads();
        // entry tile: A[r][k] = K(row r, source k), split into TF32 high and low parts
        for (int e = tid; e < kTM * kTK; e += 256) {
            const int r = e / kTK, k = e % kTK;
            const float4 a = rc[r], b = cc[k];
            const float dx = a.x - b.x, dy = a.y - b.y;
            float v;
            if (DIM == 2) {
                v = __log2f(fmaf(dx, dx, fmaf(dy, dy, 0x1p-30f)));
            } else {
                const float dz = a.z - b.z;
                v = rsqrtf(fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), 1.0f));
            }
            const uint32_t hi = to_tf32(v);
            const uint32_t lo = to_tf32(v - __uint_as_float(hi));
            const uint32_t o = op_off(r, k) >> 2;
            Ahi[o] = hi;
            Alo[o] = lo;
        }
        // x slice: B[c][k] = x[rhs0 + c][j0 + k]
        for (int e = tid; e < kTN * kTK; e += 256) {
            const int c = e / kTK, k = e % kTK;
            const long long j = j0 + k;
            const float v = (j < N && rhs0 + c < nrhs) ? (float)x[(long long)(rhs0 + c) * ldx + j] : 0.f;
            const uint32_t hi = to_tf32(v);
            const uint32_t lo = to_tf32(v - __uint_as_float(hi));
            const uint32_t o = op_off(c, k) >> 2;
            Bhi[o] = hi;
            Blo[o] = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
            for (int s = 0; s < kTK / 8; ++s) {
                const uint32_t koff = (uint32_t)s * 2 * kLBO;  // 8 TF32 elements = two K core matrices
                mma_tf32(tmem, make_desc(ahi + koff), make_desc(bhi + koff), (issued_any || s > 0) ? 1u : 0u);
                mma_tf32(tmem, make_desc(ahi + koff), make_desc(blo + koff), 1u);
                mma_tf32(tmem, make_desc(alo + koff), make_desc(bhi + koff), 1u);
            }
            mma_commit(bar);
        }
        issued_any = true;
        // the operands may be overwritten only after the MMAs that read them complete
        const bool ok = mbar_wait(bar, phase);
        if (!ok) {
            abort_flag = 1;
            // drain our own MMAs before freeing tensor memory (bounded again)
            if (tid == 0) (void)mbar_wait(bar, phase);
        }
        phase ^= 1u;
        __syncthreads();
        if (abort_flag) break;
    }

    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag && issued_any) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31
        const int q = warp & 3, h = warp >> 2;
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
        const long long i = row0 + 32 * q + lane;
        if (i < N) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int r = rhs0 + 32 * h + c;
                if (r < nrhs) partial[((long long)blockIdx.y * nrhs + r) * N + i] = (double)__uint_as_float(v[c]);
            }
        }
    } else if (abort_flag) {
        if (tid == 0) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTN));
    }
}

}  // namespace

// y partials for nrhs >= 1 right-hand sides through the tensor cores; returns IE_ERR_TIMEOUT
// (after the launch completes) if a CTA gave up waiting for its MMAs.
int launch_matvec_tc(const ie_problem *p, const double *x, long long ldx, int nrhs, double *partial, int S, int cps,
                     int nchunks, int *d_err, cudaStream_t s) {
    const int rt = (int)((p->N + kTM - 1) / kTM);
    const int groups = (nrhs + kTN - 1) / kTN;
    const dim3 g(rt, S, groups);
    const size_t dsm = sizeof(uint32_t) * (2 * kTM * kTK + 2 * kTN * kTK);
    if (p->dim == 2)
        k1t_matvec_tc<2><<<g, 256, dsm, s>>>(p->d_coord, x, ldx, nrhs, p->N, cps, nchunks, partial, d_err);
    else
        k1t_matvec_tc<3><<<g, 256, dsm, s>>>(p->d_coord, x, ldx, nrhs, p->N, cps, nchunks, partial, d_err);
    IE_LAUNCHED();
    return IE_OK;
}

int tc_chunk() { return kTK; }
int tc_rows() { return kTM; }
int tc_cols() { return kTN; }

int prepare_tc() {
    const int dsm = (int)(sizeof(uint32_t) * (2 * kTM * kTK + 2 * kTN * kTK));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1t_matvec_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1t_matvec_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    return IE_OK;
}
