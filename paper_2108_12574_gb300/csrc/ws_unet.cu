// Learned warm start: a 4-level U-Net that maps a right-hand side f to an initial iterate u0
// for pcg_solve.  Not part of the paper; a production layer on top of the method.
//
// Network (NHWC, BF16 weights and activations, FP32 accumulation, FP32 master weights + Adam):
//   encoder  conv3x3+ReLU pairs with 12, 24, 48, 96 channels, 2x2 average pooling between levels
//   decoder  nearest 2x upsampling, concatenation [upsampled, skip], conv3x3+ReLU pairs
//            with 48, 24, 12 channels, then a 1x1 convolution to one output channel.
// Parameter vector (FP32, layer by layer): W[Cout][3][3][Cin] (W[Cout][Cin] for the 1x1), then
// b[Cout].  Layer table: kLayers below.  274,213 parameters.
//
// Inputs are two channels built from f (per right-hand side): f / rms(f) and the normalised
// 5-point Laplacian L(f/rms f) / rms(L(f/rms f)) (replicated boundary).  The network predicts
// u h^2 / (rms(f) rms(L(f/rms f))): in the interior of the domain u is close to -Laplace(f)
// (A is a discretised inverse Laplacian), so this target has unit scale; the network learns the
// boundary layer and the corrections.
//
// Kernels: every 3x3 convolution runs on the tcgen05 tensor cores with BF16 operands and FP32
// accumulators in tensor memory: the forward pass and the data gradient as implicit GEMMs over
// 128-pixel tiles (KW conv3x3_tc; the data gradient is the convolution of the masked output
// gradient with the flipped weights), the weight and bias gradients as a GEMM over the pixels
// (KWg conv3x3_wgrad_tc).  CUDA cores do the rest: weight packing, the ReLU mask, pooling,
// upsample+concat, the 1x1 convolution, MSE loss and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "iedd_internal.cuh"

namespace {

typedef __nv_bfloat16 bf16;

struct LayerDef {
    int cin, cout, k;  // k = 3 or 1
};
// c0a c0b c1a c1b c2a c2b c3a c3b u2a u2b u1a u1b u0a u0b out
constexpr int kNumLayers = 15;
const LayerDef kLayers[kNumLayers] = {
    {2, 12, 3},   {12, 12, 3}, {12, 24, 3},  {24, 24, 3}, {24, 48, 3}, {48, 48, 3}, {48, 96, 3}, {96, 96, 3},
    {144, 48, 3}, {48, 48, 3}, {72, 24, 3},  {24, 24, 3}, {36, 12, 3}, {12, 12, 3}, {12, 1, 1}};
constexpr int kMaxBatch = 16;


// four BF16 <-> four FP32 (the elementwise kernels take four channels per thread: every channel
// count of the network is a multiple of 4)
__device__ __forceinline__ float4 bf4_to_f4(uint2 v) {
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xFFFF0000u), __uint_as_float(v.y << 16),
                       __uint_as_float(v.y & 0xFFFF0000u));
}
__device__ __forceinline__ uint2 f4_to_bf4(float4 f) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(f.x, f.y), b = __floats2bfloat162_rn(f.z, f.w);
    return make_uint2(*reinterpret_cast<const uint32_t *>(&a), *reinterpret_cast<const uint32_t *>(&b));
}

// ---------------------------------------------------------------------------------------------
// Tensor-core 3x3 convolutions (tcgen05.mma kind::f16: BF16 operands, FP32 accumulators in tensor
// memory).  Shared-memory operands use the canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes (8 BF16 along K), LBO = bytes between the two core matrices of one
// K = 16 step, SBO = bytes between core matrices adjacent along M (or N).  One thread issues the
// MMAs and commits them to an mbarrier per operand stage; every wait is bounded and a CTA that
// gives up sets the error flag, still drains its MMAs and frees its tensor memory.
// ---------------------------------------------------------------------------------------------
constexpr long long kWSpin = 1LL << 22;

__device__ __forceinline__ uint32_t wsmem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t wdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // tcgen05 descriptor version; base offset 0, no swizzle
    return d;
}
// kind::f16: D FP32 (bit 4), A and B BF16 (bits 7, 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t widesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ bool wbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kWSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(1000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void wmma_issue(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc ? 1u : 0u));
}
__device__ __forceinline__ void wcommit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// tensor-memory columns for an N-wide FP32 accumulator: a power of two >= 32
__host__ __device__ inline uint32_t wtmem_cols(int npad) {
    return npad <= 32 ? 32u : npad <= 64 ? 64u : npad <= 128 ? 128u : 256u;
}
// 8 BF16 channels c0..c0+7 of row `row` of a [rows][C] array (C even), zero past C; vector loads
// as wide as C's alignment allows
__device__ __forceinline__ uint4 load_ch8(const bf16 *__restrict__ a, long long row, int C, int c0) {
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    const bf16 *p = a + row * C + c0;
    if ((C & 7) == 0) {
        r = *reinterpret_cast<const uint4 *>(p);
    } else if ((C & 3) == 0) {
        const uint2 lo = *reinterpret_cast<const uint2 *>(p);
        r.x = lo.x; r.y = lo.y;
        if (c0 + 4 < C) {
            const uint2 hi = *reinterpret_cast<const uint2 *>(p + 4);
            r.z = hi.x; r.w = hi.y;
        }
    } else {
        const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
        r.x = q[0];
        if (c0 + 2 < C) r.y = q[1];
        if (c0 + 4 < C) r.z = q[2];
        if (c0 + 6 < C) r.w = q[3];
    }
    return r;
}
__device__ __forceinline__ uint32_t u4get(const uint4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
// the 8 x 8 BF16 transpose of one core matrix: in[j] = 8 channels of pixel j; row i of the result
// (channel i of pixels 0..7) is written to dst + 16 i
__device__ __forceinline__ void store_transposed(unsigned char *dst, const uint4 (&in)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t sel = (i & 1) ? 0x7632u : 0x5410u;
        uint4 o;
        o.x = __byte_perm(u4get(in[0], i >> 1), u4get(in[1], i >> 1), sel);
        o.y = __byte_perm(u4get(in[2], i >> 1), u4get(in[3], i >> 1), sel);
        o.z = __byte_perm(u4get(in[4], i >> 1), u4get(in[5], i >> 1), sel);
        o.w = __byte_perm(u4get(in[6], i >> 1), u4get(in[7], i >> 1), sel);
        *reinterpret_cast<uint4 *>(dst + 16 * i) = o;
    }
}

// Packing of the 3x3 weights into the B-operand layout of conv3x3_tc, one launch for all layers
// and both directions.  Tensor t packs W for a convolution with Cin' input and Cout' output
// channels: wtc[dst + (tap * nchunk + chunk) * npad * 16 + canonical(r, k)] = W'[r][tap][chunk*16+k]
// with canonical(r, k) = (r / 8) * 128 + (k / 8) * 64 + (r % 8) * 8 + k % 8 elements, zero past
// Cout' or Cin'.  Forward: W' = W (Cin' = Cin).  Data gradient: W'[ci][tap][co] = W[co][8 - tap][ci]
// (the kernel flipped, input and output channels swapped: Cin' = Cout, Cout' = Cin).
constexpr int kPackMax = 2 * kNumLayers;
struct TcPackPlan {
    int n;
    int cin[kPackMax], cout[kPackMax], flip[kPackMax];  // the layer's own Cin, Cout
    long long src[kPackMax], dst[kPackMax], end[kPackMax];  // W in w16; packed tensor; element prefix
};
inline int tc_npad(int cout) { return (cout + 15) / 16 * 16; }
inline int tc_nchunk(int cin) { return (cin + 15) / 16; }

__global__ void pack_tc_all(const bf16 *__restrict__ w16, const TcPackPlan plan, bf16 *__restrict__ wtc) {
    const long long total = plan.end[plan.n - 1];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int t = 0;
        while (e >= plan.end[t]) ++t;
        const long long loc = e - (t ? plan.end[t - 1] : 0);
        const int lcin = plan.cin[t], lcout = plan.cout[t], flip = plan.flip[t];
        const int ci_n = flip ? lcout : lcin, co_n = flip ? lcin : lcout;  // the packed convolution's
        const int npad = (co_n + 15) / 16 * 16, nchunk = (ci_n + 15) / 16;
        const int k = (int)(loc % 16), r = (int)((loc / 16) % npad);
        const int tc = (int)(loc / (16LL * npad)), chunk = tc % nchunk, tap = tc / nchunk;
        const int ci = chunk * 16 + k;
        bf16 v = __float2bfloat16(0.f);
        if (r < co_n && ci < ci_n)
            v = flip ? w16[plan.src[t] + ((long long)ci * 9 + (8 - tap)) * lcin + r]
                     : w16[plan.src[t] + ((long long)r * 9 + tap) * lcin + ci];
        wtc[plan.dst[t] + (long long)tc * npad * 16 + (r / 8) * 128 + (k / 8) * 64 + (r % 8) * 8 + (k % 8)] = v;
    }
}

// ---------------------------------------------------------------------------------------------
// KW conv3x3_tc: out[p][co] = sum_{tap, ci} in[p + off_tap][ci] W'[co][tap][ci] (zero padding at
// the image edges) as an implicit GEMM: M = 128 consecutive pixels (row-major over all images),
// N = Cout rounded up to 16, K = 9 taps x Cin rounded up to 16, one K = 16 MMA per tap and
// 16-channel chunk.  128 threads, thread = pixel = accumulator lane.  Per K-step each thread writes
// its source pixel's 16 channels into the A stage (two 16-byte rows: 128 bytes between the K
// halves, 256 between 8-pixel groups) and the CTA copies the step's pre-packed B tile; the global
// loads of step k + 1 are issued before the MMA of step k, so they overlap it and the barrier.
// FWD: in = the BF16 activation, out = BF16 ReLU(acc + bias).  GRAD (data gradient): in = the
// BF16 masked output gradient, W' the flipped weights, out = FP32 acc.
// ---------------------------------------------------------------------------------------------
constexpr int kWTile = 128;                // pixels per CTA (MMA M)
constexpr uint32_t kWLBO = 128, kWSBO = 256;
constexpr int kWAOp = kWTile * 16 * 2;     // A stage bytes (4 KB)
constexpr int kWNMax = 144;                // largest N (Cout, or Cin for the data gradient)
constexpr int kWBMax = kWNMax * 16 * 2;    // largest B stage bytes
constexpr int kWStage = kWAOp + kWBMax;
constexpr int kWBq = (kWNMax * 2 + kWTile - 1) / kWTile;  // 16-byte B pieces per thread and step

template <bool GRAD>
__global__ void __launch_bounds__(kWTile)
conv3x3_tc(const bf16 *__restrict__ in, long long npix, int H, int W, int Cin, const bf16 *__restrict__ wtc,
           const float *__restrict__ bias, void *__restrict__ outp, int Cout, int npad, int nchunk, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char wsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long HW = (long long)H * W;
    const long long pix = (long long)blockIdx.x * kWTile + tid;  // this thread's pixel (all images)
    const bool valid = pix < npix;
    const long long q = pix % HW;                                // its place in its image
    const int y = (int)(q / W), x = (int)(q % W);
    const uint32_t ncols = wtmem_cols(npad);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(wsmem(&tmem_base)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(wsmem(&mbar[st])), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = widesc(kWTile, npad);
    const int nk = 9 * nchunk;
    const int bq = npad * 2;  // 16-byte pieces of one B tile
    uint4 a0, a1, bv[kWBq];
    // the global loads of step k into a0, a1, bv
    auto load_step = [&](int k) {
        const int tap = k / nchunk, c0 = (k % nchunk) * 16;
        const int sy = y + tap / 3 - 1, sx = x + tap % 3 - 1;
        a0 = make_uint4(0u, 0u, 0u, 0u);
        a1 = a0;
        if (valid && sy >= 0 && sy < H && sx >= 0 && sx < W) {
            const long long src = pix + (long long)(tap / 3 - 1) * W + (tap % 3 - 1);
            a0 = load_ch8(in, src, Cin, c0);
            if (c0 + 8 < Cin) a1 = load_ch8(in, src, Cin, c0 + 8);
        }
        const uint4 *wsrc = reinterpret_cast<const uint4 *>(wtc + (long long)k * npad * 16);
#pragma unroll
        for (int i = 0; i < kWBq; ++i)
            if (tid + i * kWTile < bq) bv[i] = wsrc[tid + i * kWTile];
    };
    load_step(0);
    uint32_t ph[2] = {0u, 0u};
    int pending[2] = {0, 0};  // thread 0: a commit on the stage not yet waited for
    for (int k = 0; k < nk; ++k) {
        const int st = k & 1;
        unsigned char *A = wsm + st * kWStage, *Bt = A + kWAOp;
        if (tid == 0 && pending[st]) {  // the MMA that read this stage two steps ago must be done
            if (wbar_wait(wsmem(&mbar[st]), ph[st])) {
                ph[st] ^= 1u;
                pending[st] = 0;
            } else {
                abort_flag = 1;  // still pending: the drain below waits for it once more
            }
        }
        __syncthreads();
        if (abort_flag) break;
        const uint32_t arow = (uint32_t)((tid >> 3) * kWSBO + (tid & 7) * 16);
        *reinterpret_cast<uint4 *>(A + arow) = a0;
        *reinterpret_cast<uint4 *>(A + arow + kWLBO) = a1;
#pragma unroll
        for (int i = 0; i < kWBq; ++i)
            if (tid + i * kWTile < bq) reinterpret_cast<uint4 *>(Bt)[tid + i * kWTile] = bv[i];
        if (k + 1 < nk) load_step(k + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            wmma_issue(tmem, wdesc(wsmem(A), kWLBO, kWSBO), wdesc(wsmem(Bt), kWLBO, kWSBO), idesc, k > 0);
            wcommit(wsmem(&mbar[st]));
            pending[st] = 1;
        }
    }
    // drain: the last commit of each stage (bounded; also after an abort, so no MMA is in flight)
    if (tid == 0)
        for (int st = 0; st < 2; ++st)
            if (pending[st] && !wbar_wait(wsmem(&mbar[st]), ph[st])) abort_flag = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag) {
        // thread = pixel = TMEM lane 32 warp + lane, 16 columns per load; Cout is even, so channel
        // pairs go out as one store
        for (int c0 = 0; c0 < npad; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const int co = c0 + j;
                if (!valid || co >= Cout) continue;
                float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
                if (GRAD) {
                    *reinterpret_cast<float2 *>(static_cast<float *>(outp) + pix * Cout + co) = make_float2(v0, v1);
                } else {
                    v0 = fmaxf(v0 + bias[co], 0.f);
                    v1 = fmaxf(v1 + bias[co + 1], 0.f);
                    *reinterpret_cast<__nv_bfloat162 *>(static_cast<bf16 *>(outp) + pix * Cout + co) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

// dpre = BF16(dout * (post > 0)): the output gradient through the layer's ReLU (post = its output);
// four channels per thread (cnt is a multiple of 4)
__global__ void relu_grad_bf16(const float *__restrict__ dout, const bf16 *__restrict__ post, bf16 *__restrict__ dpre,
                               long long cnt) {
    for (long long e = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); e < cnt; e += 4LL * gridDim.x * blockDim.x) {
        const float4 d = *reinterpret_cast<const float4 *>(dout + e);
        const float4 m = bf4_to_f4(*reinterpret_cast<const uint2 *>(post + e));
        *reinterpret_cast<uint2 *>(dpre + e) = f4_to_bf4(make_float4(m.x > 0.f ? d.x : 0.f, m.y > 0.f ? d.y : 0.f,
                                                                     m.z > 0.f ? d.z : 0.f, m.w > 0.f ? d.w : 0.f));
    }
}

// ---------------------------------------------------------------------------------------------
// KWg conv3x3_wgrad_tc: dW[co][tap][ci] += sum_p dpre[p][co] in[p + off_tap][ci] and
// db[co] += sum_p dpre[p][co], as a GEMM over pixels: D[row][co] = sum_p A[row][p] dpre[p][co] with
// rows (tap, ci) (tap-major, Cin rounded up to 8 per tap) plus one row of ones (the bias
// gradient), M = 128 rows per CTA (blockIdx.y), N = Cout rounded up to 16, K = the pixels, 128 per
// stage (8 MMAs).  Both operands are pixel-major in memory and K-major in shared memory, so each
// thread gathers one 8-row x 8-pixel core matrix (eight 16-byte channel loads) and transposes it
// in registers.  Core matrices adjacent in K are 144 bytes apart (16 of padding), which spreads a
// quarter-warp's rows over all banks.  256 threads; CTAs stride over the pixel stages
// (blockIdx.x), accumulate in tensor memory, and add their partial sums to dW, db with atomics.
// ---------------------------------------------------------------------------------------------
constexpr int kGP = 128;                         // pixels per stage (K)
constexpr int kGThreads = 256;
constexpr uint32_t kGLBO = 144;                  // K-adjacent core matrices
constexpr uint32_t kGSBO = (kGP / 8) * kGLBO;    // M- (N-) adjacent core matrices: 2304
constexpr int kGAOp = 16 * kGSBO;                // 128 rows: 36,864 bytes
constexpr int kGNMax = 96;                       // largest Cout
constexpr int kGBOp = (kGNMax / 8) * kGSBO;      // 27,648 bytes
constexpr int kGSmem = 2 * (kGAOp + kGBOp);      // 129,024 bytes at most: two stages
// two stages of A and of an npad-row B
inline int wgrad_smem(int npad) { return 2 * (kGAOp + (npad / 8) * (int)kGSBO); }

__global__ void __launch_bounds__(kGThreads, 2)
conv3x3_wgrad_tc(const bf16 *__restrict__ dpre, const bf16 *__restrict__ in, long long npix, int H, int W, int Cin,
                 int Cout, int npad, float *__restrict__ dW, float *__restrict__ db, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char wsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin8 = (Cin + 7) / 8 * 8, rows = 9 * cin8;  // row `rows` is the ones row
    const int stage_bytes = kGAOp + (npad / 8) * (int)kGSBO;
    const int row0 = blockIdx.y * 128;
    const long long nstage = (npix + kGP - 1) / kGP;
    const uint32_t ncols = wtmem_cols(npad);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(wsmem(&tmem_base)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(wsmem(&mbar[st])), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = widesc(128, npad);
    // this thread's core matrices: pixel group pg (8 pixels) of every stage; A row group ag; B row
    // group (output channels 8 bg ..) when bg < npad / 8
    const int pg = tid & 15, ag = tid >> 4, bg = tid >> 4;
    const bool has_b = bg < npad / 8;
    const int arow = row0 + 8 * ag;  // first row of the A core matrix
    const int tap = arow < rows ? arow / cin8 : 0, ac0 = arow < rows ? arow % cin8 : 0;
    const int ady = tap / 3 - 1, adx = tap % 3 - 1;
    uint4 av[8], bv[8];
    auto load_stage = [&](long long s) {
        long long p = s * kGP + 8 * pg;
        long long qq = p % ((long long)H * W);
        int yy = (int)(qq / W), xx = (int)(qq % W);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = p < npix;
            av[j] = make_uint4(0u, 0u, 0u, 0u);
            if (arow < rows) {
                const int sy = yy + ady, sx = xx + adx;
                if (ok && sy >= 0 && sy < H && sx >= 0 && sx < W) av[j] = load_ch8(in, p + (long long)ady * W + adx, Cin, ac0);
            } else if (arow == rows) {
                av[j].x = 0x3F80u;  // 1.0 in row 0 of the core matrix (channel slot 0)
            }
            bv[j] = make_uint4(0u, 0u, 0u, 0u);
            if (has_b && ok) bv[j] = load_ch8(dpre, p, Cout, 8 * bg);
            ++p;
            if (++xx == W) { xx = 0; if (++yy == H) yy = 0; }
        }
    };
    long long s = blockIdx.x;
    if (s < nstage) load_stage(s);
    uint32_t ph[2] = {0u, 0u};
    int pending[2] = {0, 0};
    bool any = false;
    for (int it = 0; s < nstage; ++it, s += gridDim.x) {
        const int st = it & 1;
        unsigned char *A = wsm + st * stage_bytes, *Bt = A + kGAOp;
        if (tid == 0 && pending[st]) {
            if (wbar_wait(wsmem(&mbar[st]), ph[st])) {
                ph[st] ^= 1u;
                pending[st] = 0;
            } else {
                abort_flag = 1;
            }
        }
        __syncthreads();
        if (abort_flag) break;
        store_transposed(A + ag * kGSBO + pg * kGLBO, av);
        if (has_b) store_transposed(Bt + bg * kGSBO + pg * kGLBO, bv);
        if (s + gridDim.x < nstage) load_stage(s + gridDim.x);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < kGP / 16; ++kk)
                wmma_issue(tmem, wdesc(wsmem(A) + kk * 2 * kGLBO, kGLBO, kGSBO), wdesc(wsmem(Bt) + kk * 2 * kGLBO, kGLBO, kGSBO),
                           idesc, any || kk > 0);
            wcommit(wsmem(&mbar[st]));
            pending[st] = 1;
        }
        any = true;
    }
    if (tid == 0)
        for (int st = 0; st < 2; ++st)
            if (pending[st] && !wbar_wait(wsmem(&mbar[st]), ph[st])) abort_flag = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag && any) {
        // warps w and w + 4 read TMEM lanes 32 (w % 4) ..: even and odd 8-column groups
        const int r = row0 + 32 * (warp & 3) + lane;
        const int rtap = r / cin8, rci = r % cin8;
        for (int c0 = 8 * (warp >> 2); c0 < npad; c0 += 16) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int co = c0 + j;
                if (co >= Cout) break;
                if (r < rows && rci < Cin) atomicAdd(&dW[((long long)co * 9 + rtap) * Cin + rci], __uint_as_float(v[j]));
                else if (r == rows) atomicAdd(&db[co], __uint_as_float(v[j]));
            }
        }
    } else if (abort_flag && tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

// out[b,y,x,c] = mean of in over the 2x2 children (H, W even)
__global__ void avgpool2(const bf16 *__restrict__ in, bf16 *__restrict__ out, int B, int H, int W, int C) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (output pixel, channel group)
    const int G = C / 4, Ho = H / 2, Wo = W / 2;
    if (e >= (long long)B * Ho * Wo * G) return;
    const int c = 4 * (int)(e % G);
    const long long po = e / G;
    const int x = (int)(po % Wo), y = (int)((po / Wo) % Ho);
    const long long b = po / ((long long)Wo * Ho);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const float4 v = bf4_to_f4(*reinterpret_cast<const uint2 *>(in + ((b * H + 2 * y + dy) * W + 2 * x + dx) * C + c));
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
    *reinterpret_cast<uint2 *>(out + po * C + c) = f4_to_bf4(make_float4(0.25f * s.x, 0.25f * s.y, 0.25f * s.z, 0.25f * s.w));
}

// din[b,Y,X,c] += 0.25 dout[b,Y/2,X/2,c]
__global__ void avgpool2_bwd(const float *__restrict__ dout, float *__restrict__ din, int B, int H, int W, int C) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (input pixel, channel group)
    const int G = C / 4;
    if (e >= (long long)B * H * W * G) return;
    const int c = 4 * (int)(e % G);
    const long long p = e / G;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long long b = p / ((long long)W * H);
    const float4 d = *reinterpret_cast<const float4 *>(dout + ((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c);
    float4 *o = reinterpret_cast<float4 *>(din + p * C + c);
    float4 v = *o;
    v.x += 0.25f * d.x; v.y += 0.25f * d.y; v.z += 0.25f * d.z; v.w += 0.25f * d.w;
    *o = v;
}

// cat[b,y,x,:] = [up[b,y/2,x/2,0:Cu], skip[b,y,x,0:Cs]]
__global__ void upcat(const bf16 *__restrict__ up, const bf16 *__restrict__ skip, bf16 *__restrict__ cat, int B, int H,
                      int W, int Cu, int Cs) {
    const int C = Cu + Cs, G = C / 4;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (pixel, channel group)
    if (e >= (long long)B * H * W * G) return;
    const int c = 4 * (int)(e % G);
    const long long p = e / G;
    const bf16 *src;
    if (c < Cu) {
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const long long b = p / ((long long)W * H);
        src = up + ((b * (H / 2) + y / 2) * (W / 2) + x / 2) * Cu + c;
    } else {
        src = skip + p * Cs + (c - Cu);
    }
    *reinterpret_cast<uint2 *>(cat + p * C + c) = *reinterpret_cast<const uint2 *>(src);
}

// dup[b,y',x',c] = sum over the 2x2 children of dcat[..., c]
__global__ void upcat_bwd_up(const float *__restrict__ dcat, float *__restrict__ dup, int B, int H, int W, int Cu, int Cs) {
    const int C = Cu + Cs, G = Cu / 4, Ho = H / 2, Wo = W / 2;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (half-resolution pixel, group)
    if (e >= (long long)B * Ho * Wo * G) return;
    const int c = 4 * (int)(e % G);
    const long long po = e / G;
    const int x = (int)(po % Wo), y = (int)((po / Wo) % Ho);
    const long long b = po / ((long long)Wo * Ho);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const float4 v = *reinterpret_cast<const float4 *>(dcat + ((b * H + 2 * y + dy) * W + 2 * x + dx) * C + c);
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
    *reinterpret_cast<float4 *>(dup + po * Cu + c) = s;
}

// dskip[b,y,x,c] = dcat[b,y,x,Cu + c]
__global__ void upcat_bwd_skip(const float *__restrict__ dcat, float *__restrict__ dskip, long long npix, int Cu, int Cs) {
    const int G = Cs / 4;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npix * G) return;
    const int c = 4 * (int)(e % G);
    const long long p = e / G;
    *reinterpret_cast<float4 *>(dskip + p * Cs + c) = *reinterpret_cast<const float4 *>(dcat + p * (Cu + Cs) + Cu + c);
}

// out[p] = b + sum_c in[p][c] w[c]   (1x1, one output channel, FP32 output)
__global__ void conv1x1_out(const bf16 *__restrict__ in, const bf16 *__restrict__ w, const float *__restrict__ b,
                            float *__restrict__ out, long long npix, int C) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    float s = b[0];
    for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(in[p * C + c]), __bfloat162float(w[c]), s);
    out[p] = s;
}

// din[p][c] = dout[p] w[c];  dW[c] += sum_p dout[p] in[p][c];  db += sum_p dout[p]
__global__ void conv1x1_bwd(const float *__restrict__ dout, const bf16 *__restrict__ in, const bf16 *__restrict__ w,
                            float *__restrict__ din, float *__restrict__ dW, float *__restrict__ db, long long npix, int C) {
    __shared__ float red[13][8];
    float part[13];
    for (int c = 0; c < 13; ++c) part[c] = 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
        const float d = dout[p];
        for (int c = 0; c < C && c < 12; ++c) {
            din[p * C + c] = d * __bfloat162float(w[c]);
            part[c] = fmaf(d, __bfloat162float(in[p * C + c]), part[c]);
        }
        part[12] += d;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < 13; ++c) {
        float v = part[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
        float v = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[threadIdx.x][q];
        if (threadIdx.x < 12) { if (threadIdx.x < C) atomicAdd(&dW[threadIdx.x], v); }
        else atomicAdd(db, v);
    }
}

// dout = 2 (out - t) / count;  loss partials = sum (out - t)^2 (FP64 atomics)
__global__ void mse_grad(const float *__restrict__ out, const float *__restrict__ tgt, float *__restrict__ dout,
                         long long count, double *__restrict__ loss) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - tgt[i];
        dout[i] = 2.f * d / (float)count;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / (double)count);
}

__global__ void adam_step(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                          bf16 *__restrict__ w16, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    w16[i] = __float2bfloat16(wi);
}

__global__ void to_bf16(const float *__restrict__ a, bf16 *__restrict__ b, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Per right-hand side k (column of f, N = n*n): Lraw(f) = 4 f - (4 neighbours, replicated at
// the boundary), written to lap (FP64).
__global__ void laplace5(const double *__restrict__ f, long long ldf, double *__restrict__ lap, int n) {
    const long long N = (long long)n * n;
    const int k = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int r = (int)(i / n), c = (int)(i % n);
    const double *fk = f + (long long)k * ldf;
    const double v = fk[i];
    const double up = fk[(long long)(r > 0 ? r - 1 : r) * n + c], dn = fk[(long long)(r < n - 1 ? r + 1 : r) * n + c];
    const double lf = fk[(long long)r * n + (c > 0 ? c - 1 : c)], rt = fk[(long long)r * n + (c < n - 1 ? c + 1 : c)];
    lap[(long long)k * N + i] = 4.0 * v - up - dn - lf - rt;
}

// features (NHWC, 2 channels, BF16): [f / rms_f, lap / (rms_f * s_l)];  target = u h^2 / (rms_f s_l)
// with rms_f^2 = ff[k] / N and s_l^2 = ll[k] / (N rms_f^2).
__global__ void make_features(const double *__restrict__ f, long long ldf, const double *__restrict__ lap,
                              const double *__restrict__ ff, const double *__restrict__ ll, const double *__restrict__ u,
                              long long ldu, double h2, bf16 *__restrict__ feat, float *__restrict__ tgt, long long N) {
    const int k = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double rf = sqrt(ff[k] / (double)N);
    const double rl = sqrt(ll[k] / (double)N);  // rms of lap(f), = rms_f * s_l
    const double inv_rf = rf > 0 ? 1.0 / rf : 0.0, inv_rl = rl > 0 ? 1.0 / rl : 0.0;
    feat[((long long)k * N + i) * 2 + 0] = __float2bfloat16((float)(f[(long long)k * ldf + i] * inv_rf));
    feat[((long long)k * N + i) * 2 + 1] = __float2bfloat16((float)(lap[(long long)k * N + i] * inv_rl));
    if (u && tgt) tgt[(long long)k * N + i] = (float)(u[(long long)k * ldu + i] * h2 * inv_rl);
}

// u0 = out * rms(lap f) / h^2
__global__ void unscale_output(const float *__restrict__ out, const double *__restrict__ ll, double inv_h2,
                               double *__restrict__ u0, long long ldu, long long N) {
    const int k = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double rl = sqrt(ll[k] / (double)N);
    u0[(long long)k * ldu + i] = (double)out[(long long)k * N + i] * rl * inv_h2;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Model handle
// ---------------------------------------------------------------------------------------------
struct ws_model {
    int device = 0;
    long long nparams = 0;
    long long woff[kNumLayers], boff[kNumLayers];
    float *w32 = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    bf16 *w16 = nullptr;
    bf16 *wtc = nullptr;                    // the 3x3 layers' weights in the tensor-core B layout
    long long tcoff[kNumLayers] = {0};      // forward convolution of layer l in wtc
    long long tcdoff[kNumLayers] = {0};     // its data-gradient convolution (flipped weights)
    int *d_err = nullptr;                   // a tensor-core convolution gave up waiting for its MMA
    int nsm = 1;                            // streaming multiprocessors of the device
    long long step = 0;
    // activation / gradient buffers for (batch, n)
    int cap_b = 0, cap_n = 0;
    std::vector<void *> bufs;
    bf16 *act[32] = {nullptr};
    float *grd[32] = {nullptr};
    float *out = nullptr, *dout = nullptr, *tgt = nullptr;
    bf16 *dpre = nullptr;                   // a layer's output gradient through its ReLU (BF16)
    double *lap = nullptr, *ffll = nullptr, *loss = nullptr;
    ~ws_model() {
        cudaFree(w32); cudaFree(m); cudaFree(v); cudaFree(g); cudaFree(w16);
        cudaFree(wtc); cudaFree(d_err);
        for (void *p : bufs) cudaFree(p);
    }
};

namespace {

// activation ids
enum {
    A_IN, A_A0, A_S0, A_P0, A_A1, A_S1, A_P1, A_A2, A_S2, A_P2, A_A3, A_B3,
    A_K2, A_E2, A_D2, A_K1, A_E1, A_D1, A_K0, A_E0, A_D0, A_COUNT
};
struct ActDef {
    int level, ch;
};
const ActDef kActs[A_COUNT] = {{0, 2},  {0, 12},  {0, 12}, {1, 12}, {1, 24}, {1, 24}, {2, 24},
                               {2, 48}, {2, 48},  {3, 48}, {3, 96}, {3, 96}, {2, 144}, {2, 48},
                               {2, 48}, {1, 72},  {1, 24}, {1, 24}, {0, 36}, {0, 12}, {0, 12}};

unsigned long long splitmix(unsigned long long &s) {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int ensure_buffers(ws_model *w, int B, int n) {
    if (B <= w->cap_b && n == w->cap_n) return IE_OK;
    for (void *p : w->bufs) cudaFree(p);
    w->bufs.clear();
    auto alloc = [&](size_t bytes, void **p) -> int {
        IE_TRY_CUDA(cudaMalloc(p, bytes));
        w->bufs.push_back(*p);
        return IE_OK;
    };
    const int Bc = std::max(B, 1);
    for (int a = 0; a < A_COUNT; ++a) {
        const long long side = n >> kActs[a].level;
        const long long cnt = (long long)Bc * side * side * kActs[a].ch;
        IE_TRY(alloc(sizeof(bf16) * cnt, (void **)&w->act[a]));
        IE_TRY(alloc(sizeof(float) * cnt, (void **)&w->grd[a]));
    }
    long long maxact = 0;  // the largest activation (bounds every layer's output)
    for (int a = 0; a < A_COUNT; ++a) {
        const long long side = n >> kActs[a].level;
        maxact = std::max(maxact, (long long)Bc * side * side * kActs[a].ch);
    }
    IE_TRY(alloc(sizeof(bf16) * maxact, (void **)&w->dpre));
    const long long npix = (long long)Bc * n * n;
    IE_TRY(alloc(sizeof(float) * npix, (void **)&w->out));
    IE_TRY(alloc(sizeof(float) * npix, (void **)&w->dout));
    IE_TRY(alloc(sizeof(float) * npix, (void **)&w->tgt));
    IE_TRY(alloc(sizeof(double) * npix, (void **)&w->lap));
    IE_TRY(alloc(sizeof(double) * 2 * kMaxBatch, (void **)&w->ffll));
    IE_TRY(alloc(sizeof(double), (void **)&w->loss));
    w->cap_b = Bc;
    w->cap_n = n;
    return IE_OK;
}

inline unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// the forward 3x3 convolutions run on the tensor cores (conv3x3_tc)
int conv_fwd(ws_model *w, int layer, int a_in, int a_out, int B, int n, cudaStream_t s) {
    const LayerDef &L = kLayers[layer];
    const int side = n >> kActs[a_in].level;
    const long long npix = (long long)B * side * side;
    const unsigned tiles = (unsigned)((npix + kWTile - 1) / kWTile);
    conv3x3_tc<false><<<tiles, kWTile, 2 * kWStage, s>>>(w->act[a_in], npix, side, side, L.cin, w->wtc + w->tcoff[layer],
                                                         w->w32 + w->boff[layer], w->act[a_out], L.cout, tc_npad(L.cout),
                                                         tc_nchunk(L.cin), w->d_err);
    IE_LAUNCHED();
    return IE_OK;
}

// the BF16 weights of every 3x3 layer into the tensor-core B layout, forward and flipped, in one
// launch (after each change of the weights: once per forward pass)
TcPackPlan pack_plan(const ws_model *w) {
    TcPackPlan P{};
    long long acc = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        if (kLayers[l].k != 3) continue;
        const LayerDef &L = kLayers[l];
        for (int flip = 0; flip < 2; ++flip) {
            const int t = P.n++;
            P.cin[t] = L.cin;
            P.cout[t] = L.cout;
            P.flip[t] = flip;
            P.src[t] = w->woff[l];
            P.dst[t] = flip ? w->tcdoff[l] : w->tcoff[l];
            acc += flip ? 9LL * tc_nchunk(L.cout) * tc_npad(L.cin) * 16 : 9LL * tc_nchunk(L.cin) * tc_npad(L.cout) * 16;
            P.end[t] = acc;
        }
    }
    return P;
}

int pack_tc_weights(ws_model *w, cudaStream_t s) {
    const TcPackPlan P = pack_plan(w);
    pack_tc_all<<<std::min<unsigned>(blocks_for(P.end[P.n - 1]), 1024), 256, 0, s>>>(w->w16, P, w->wtc);
    IE_LAUNCHED();
    return IE_OK;
}

// gradient through a conv3x3+ReLU layer whose output is a_out (post-ReLU) and input a_in:
// accumulates dW, db (tensor cores, over the pixels); writes d(a_in) (tensor cores, the flipped
// convolution of the masked gradient) unless skip_din.
int conv_bwd(ws_model *w, int layer, int a_in, int a_out, int B, int n, bool skip_din, cudaStream_t s) {
    const LayerDef &L = kLayers[layer];
    const int side = n >> kActs[a_in].level;
    const long long npix = (long long)B * side * side;
    const long long cnt = npix * L.cout;
    relu_grad_bf16<<<std::min<unsigned>(blocks_for(cnt / 4), 4096), 256, 0, s>>>(w->grd[a_out], w->act[a_out], w->dpre, cnt);
    IE_LAUNCHED();
    // one wave: as many CTAs as fit on the SMs at once (two per SM unless the B stage is large)
    const int mtiles = (9 * ((L.cin + 7) / 8 * 8) + 1 + 127) / 128;
    const long long nstage = (npix + kGP - 1) / kGP;
    const int smem = wgrad_smem(tc_npad(L.cout));
    const int per_sm = smem <= 113 * 1024 ? 2 : 1;
    const int nsplit = (int)std::max<long long>(1, std::min<long long>(nstage, per_sm * w->nsm / mtiles));
    conv3x3_wgrad_tc<<<dim3(nsplit, mtiles), kGThreads, smem, s>>>(w->dpre, w->act[a_in], npix, side, side, L.cin, L.cout,
                                                                     tc_npad(L.cout), w->g + w->woff[layer],
                                                                     w->g + w->boff[layer], w->d_err);
    IE_LAUNCHED();
    if (skip_din) return IE_OK;
    const unsigned tiles = (unsigned)((npix + kWTile - 1) / kWTile);
    conv3x3_tc<true><<<tiles, kWTile, 2 * kWStage, s>>>(w->dpre, npix, side, side, L.cout, w->wtc + w->tcdoff[layer], nullptr,
                                                        w->grd[a_in], L.cin, tc_npad(L.cin), tc_nchunk(L.cout), w->d_err);
    IE_LAUNCHED();
    return IE_OK;
}

int pool(ws_model *w, int a_in, int a_out, int B, int n, cudaStream_t s) {
    const int side = n >> kActs[a_in].level, C = kActs[a_in].ch;
    avgpool2<<<blocks_for((long long)B * (side / 2) * (side / 2) * C / 4), 256, 0, s>>>(w->act[a_in], w->act[a_out], B, side, side, C);
    IE_LAUNCHED();
    return IE_OK;
}

int up_cat(ws_model *w, int a_up, int a_skip, int a_cat, int B, int n, cudaStream_t s) {
    const int side = n >> kActs[a_cat].level;
    const int Cu = kActs[a_up].ch, Cs = kActs[a_skip].ch;
    upcat<<<blocks_for((long long)B * side * side * (Cu + Cs) / 4), 256, 0, s>>>(w->act[a_up], w->act[a_skip], w->act[a_cat], B,
                                                                            side, side, Cu, Cs);
    IE_LAUNCHED();
    return IE_OK;
}

int forward(ws_model *w, int B, int n, cudaStream_t s) {
    IE_TRY(pack_tc_weights(w, s));
    IE_TRY(conv_fwd(w, 0, A_IN, A_A0, B, n, s));
    IE_TRY(conv_fwd(w, 1, A_A0, A_S0, B, n, s));
    IE_TRY(pool(w, A_S0, A_P0, B, n, s));
    IE_TRY(conv_fwd(w, 2, A_P0, A_A1, B, n, s));
    IE_TRY(conv_fwd(w, 3, A_A1, A_S1, B, n, s));
    IE_TRY(pool(w, A_S1, A_P1, B, n, s));
    IE_TRY(conv_fwd(w, 4, A_P1, A_A2, B, n, s));
    IE_TRY(conv_fwd(w, 5, A_A2, A_S2, B, n, s));
    IE_TRY(pool(w, A_S2, A_P2, B, n, s));
    IE_TRY(conv_fwd(w, 6, A_P2, A_A3, B, n, s));
    IE_TRY(conv_fwd(w, 7, A_A3, A_B3, B, n, s));
    IE_TRY(up_cat(w, A_B3, A_S2, A_K2, B, n, s));
    IE_TRY(conv_fwd(w, 8, A_K2, A_E2, B, n, s));
    IE_TRY(conv_fwd(w, 9, A_E2, A_D2, B, n, s));
    IE_TRY(up_cat(w, A_D2, A_S1, A_K1, B, n, s));
    IE_TRY(conv_fwd(w, 10, A_K1, A_E1, B, n, s));
    IE_TRY(conv_fwd(w, 11, A_E1, A_D1, B, n, s));
    IE_TRY(up_cat(w, A_D1, A_S0, A_K0, B, n, s));
    IE_TRY(conv_fwd(w, 12, A_K0, A_E0, B, n, s));
    IE_TRY(conv_fwd(w, 13, A_E0, A_D0, B, n, s));
    const long long npix = (long long)B * n * n;
    conv1x1_out<<<blocks_for(npix), 256, 0, s>>>(w->act[A_D0], w->w16 + w->woff[14], w->w32 + w->boff[14], w->out, npix, 12);
    IE_LAUNCHED();
    return IE_OK;
}

int backward(ws_model *w, int B, int n, cudaStream_t s) {
    const long long npix = (long long)B * n * n;
    IE_TRY_CUDA(cudaMemsetAsync(w->g, 0, sizeof(float) * w->nparams, s));
    conv1x1_bwd<<<std::min<unsigned>(blocks_for(npix), 512), 256, 0, s>>>(w->dout, w->act[A_D0], w->w16 + w->woff[14],
                                                                         w->grd[A_D0], w->g + w->woff[14], w->g + w->boff[14],
                                                                         npix, 12);
    IE_LAUNCHED();
    auto upcat_bwd = [&](int a_cat, int a_up, int a_skip) -> int {
        const int side = n >> kActs[a_cat].level;
        const int Cu = kActs[a_up].ch, Cs = kActs[a_skip].ch;
        const long long np = (long long)B * side * side;
        upcat_bwd_up<<<blocks_for((long long)B * (side / 2) * (side / 2) * Cu / 4), 256, 0, s>>>(w->grd[a_cat], w->grd[a_up], B,
                                                                                            side, side, Cu, Cs);
        IE_LAUNCHED();
        upcat_bwd_skip<<<blocks_for(np * Cs / 4), 256, 0, s>>>(w->grd[a_cat], w->grd[a_skip], np, Cu, Cs);
        IE_LAUNCHED();
        return IE_OK;
    };
    auto pool_bwd = [&](int a_in, int a_out) -> int {
        const int side = n >> kActs[a_in].level, C = kActs[a_in].ch;
        avgpool2_bwd<<<blocks_for((long long)B * side * side * C / 4), 256, 0, s>>>(w->grd[a_out], w->grd[a_in], B, side, side, C);
        IE_LAUNCHED();
        return IE_OK;
    };
    IE_TRY(conv_bwd(w, 13, A_E0, A_D0, B, n, false, s));
    IE_TRY(conv_bwd(w, 12, A_K0, A_E0, B, n, false, s));
    IE_TRY(upcat_bwd(A_K0, A_D1, A_S0));
    IE_TRY(conv_bwd(w, 11, A_E1, A_D1, B, n, false, s));
    IE_TRY(conv_bwd(w, 10, A_K1, A_E1, B, n, false, s));
    IE_TRY(upcat_bwd(A_K1, A_D2, A_S1));
    IE_TRY(conv_bwd(w, 9, A_E2, A_D2, B, n, false, s));
    IE_TRY(conv_bwd(w, 8, A_K2, A_E2, B, n, false, s));
    IE_TRY(upcat_bwd(A_K2, A_B3, A_S2));
    IE_TRY(conv_bwd(w, 7, A_A3, A_B3, B, n, false, s));
    IE_TRY(conv_bwd(w, 6, A_P2, A_A3, B, n, false, s));
    IE_TRY(pool_bwd(A_S2, A_P2));
    IE_TRY(conv_bwd(w, 5, A_A2, A_S2, B, n, false, s));
    IE_TRY(conv_bwd(w, 4, A_P1, A_A2, B, n, false, s));
    IE_TRY(pool_bwd(A_S1, A_P1));
    IE_TRY(conv_bwd(w, 3, A_A1, A_S1, B, n, false, s));
    IE_TRY(conv_bwd(w, 2, A_P0, A_A1, B, n, false, s));
    IE_TRY(pool_bwd(A_S0, A_P0));
    IE_TRY(conv_bwd(w, 1, A_A0, A_S0, B, n, false, s));
    IE_TRY(conv_bwd(w, 0, A_IN, A_A0, B, n, true, s));
    return IE_OK;
}

int check_grid(const ws_model *w, int n) {
    if (!w) { ie_set_error("ws: NULL model"); return IE_ERR_ARG; }
    if (n < 16 || n % 16 != 0) { ie_set_error("ws: the grid side must be a multiple of 16"); return IE_ERR_ARG; }
    return IE_OK;
}

// features (and target when u != nullptr) for B right-hand sides of a 2D problem
int prepare(ws_model *w, const ie_problem *p, const double *f, long long ldf, const double *u, long long ldu, int B,
            cudaStream_t s) {
    const int n = p->n;
    const long long N = p->N;
    dim3 g(blocks_for(N), B);
    laplace5<<<g, 256, 0, s>>>(f, ldf, w->lap, n);
    IE_LAUNCHED();
    IE_TRY(launch_dots(f, ldf, f, ldf, N, B, w->ffll, s));
    IE_TRY(launch_dots(w->lap, N, w->lap, N, N, B, w->ffll + kMaxBatch, s));
    make_features<<<g, 256, 0, s>>>(f, ldf, w->lap, w->ffll, w->ffll + kMaxBatch, u, ldu, p->h * p->h, w->act[A_IN],
                                    u ? w->tgt : nullptr, N);
    IE_LAUNCHED();
    return IE_OK;
}

}  // namespace

extern "C" int ws_create(int device, unsigned long long seed, ws_model **out) {
    if (!out) { ie_set_error("ws_create: out is NULL"); return IE_ERR_ARG; }
    *out = nullptr;
    int ndev = 0;
    IE_TRY_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) { ie_set_error("ws_create: bad device"); return IE_ERR_ARG; }
    DeviceGuard g(device);
    ws_model *w = new (std::nothrow) ws_model();
    if (!w) { ie_set_error("ws_create: out of host memory"); return IE_ERR_OOM; }
    w->device = device;
    long long off = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        const long long nw = (long long)kLayers[l].cout * kLayers[l].k * kLayers[l].k * kLayers[l].cin;
        w->woff[l] = off;
        off += nw;
        w->boff[l] = off;
        off += kLayers[l].cout;
    }
    w->nparams = off;
    // He-normal initial weights (Box-Muller over SplitMix64), zero biases
    std::vector<float> h((size_t)off, 0.f);
    unsigned long long st = seed;
    for (int l = 0; l < kNumLayers; ++l) {
        const long long nw = w->boff[l] - w->woff[l];
        const double fan_in = (double)kLayers[l].k * kLayers[l].k * kLayers[l].cin;
        const double sd = std::sqrt(2.0 / fan_in) * (l == kNumLayers - 1 ? 0.5 : 1.0);
        for (long long i = 0; i < nw; ++i) {
            const double u1 = ((splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
            const double u2 = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
            h[(size_t)(w->woff[l] + i)] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    auto fail = [&](cudaError_t e) {
        ie_set_error(std::string("ws_create: ") + cudaGetErrorString(e));
        delete w;
        return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&w->w32, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&w->m, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&w->v, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&w->g, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&w->w16, sizeof(bf16) * off)) != cudaSuccess) return fail(e);
    long long tco = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        if (kLayers[l].k != 3) continue;
        w->tcoff[l] = tco;
        tco += 9LL * tc_nchunk(kLayers[l].cin) * tc_npad(kLayers[l].cout) * 16;
        w->tcdoff[l] = tco;
        tco += 9LL * tc_nchunk(kLayers[l].cout) * tc_npad(kLayers[l].cin) * 16;
    }
    if ((e = cudaFuncSetAttribute(conv3x3_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem)) != cudaSuccess)
        return fail(e);
    if ((e = cudaDeviceGetAttribute(&w->nsm, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&w->wtc, sizeof(bf16) * std::max<long long>(tco, 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&w->d_err, sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(w->d_err, 0, sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(w->w32, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(w->m, 0, sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(w->v, 0, sizeof(float) * off)) != cudaSuccess) return fail(e);
    to_bf16<<<blocks_for(off), 256>>>(w->w32, w->w16, off);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
    *out = w;
    return IE_OK;
}

extern "C" void ws_destroy(ws_model *w) {
    if (!w) return;
    DeviceGuard g(w->device);
    delete w;
}

extern "C" long long ws_num_params(const ws_model *w) { return w ? w->nparams : -1; }

extern "C" int ws_get_params(const ws_model *w, float *host) {
    if (!w || !host) { ie_set_error("ws_get_params: NULL argument"); return IE_ERR_ARG; }
    DeviceGuard g(w->device);
    IE_TRY_CUDA(cudaMemcpy(host, w->w32, sizeof(float) * w->nparams, cudaMemcpyDeviceToHost));
    return IE_OK;
}

extern "C" int ws_set_params(ws_model *w, const float *host) {
    if (!w || !host) { ie_set_error("ws_set_params: NULL argument"); return IE_ERR_ARG; }
    DeviceGuard g(w->device);
    IE_TRY_CUDA(cudaMemcpy(w->w32, host, sizeof(float) * w->nparams, cudaMemcpyHostToDevice));
    IE_TRY_CUDA(cudaMemset(w->m, 0, sizeof(float) * w->nparams));
    IE_TRY_CUDA(cudaMemset(w->v, 0, sizeof(float) * w->nparams));
    w->step = 0;
    to_bf16<<<blocks_for(w->nparams), 256>>>(w->w32, w->w16, w->nparams);
    IE_LAUNCHED();
    IE_TRY_CUDA(cudaDeviceSynchronize());
    return IE_OK;
}

// after a stream synchronize: a tensor-core convolution that gave up waiting for its MMAs (its
// output is then unspecified) turns the call's status into IE_ERR_TIMEOUT; the flag is cleared
int take_tc_error(ws_model *w, const char *who) {
    int err = 0;
    IE_TRY_CUDA(cudaMemcpy(&err, w->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!err) return IE_OK;
    IE_TRY_CUDA(cudaMemset(w->d_err, 0, sizeof(int)));
    ie_set_error(std::string(who) + ": a tensor-core convolution timed out waiting for its MMAs");
    return IE_ERR_TIMEOUT;
}

extern "C" int ws_forward_raw(ws_model *w, const float *in, float *out, int B, int n, void *stream) {
    IE_TRY(check_grid(w, n));
    if (B < 1 || B > kMaxBatch || !in || !out) { ie_set_error("ws_forward_raw: bad arguments"); return IE_ERR_ARG; }
    DeviceGuard g(w->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    IE_TRY(ensure_buffers(w, B, n));
    const long long cnt = (long long)B * n * n * 2;
    DevBuf tmp;
    IE_TRY(tmp.alloc(sizeof(float) * cnt, s));
    IE_TRY_CUDA(cudaMemcpyAsync(tmp.ptr, in, sizeof(float) * cnt, cudaMemcpyDefault, s));
    to_bf16<<<blocks_for(cnt), 256, 0, s>>>(tmp.as<float>(), w->act[A_IN], cnt);
    IE_LAUNCHED();
    IE_TRY(forward(w, B, n, s));
    IE_TRY_CUDA(cudaMemcpyAsync(out, w->out, sizeof(float) * B * n * n, cudaMemcpyDefault, s));
    IE_TRY_CUDA(cudaStreamSynchronize(s));
    return take_tc_error(w, "ws_forward_raw");
}

extern "C" int ws_backward_raw(ws_model *w, const float *in, const float *dout, float *grad, int B, int n, void *stream) {
    IE_TRY(check_grid(w, n));
    if (B < 1 || B > kMaxBatch || !in || !dout || !grad) { ie_set_error("ws_backward_raw: bad arguments"); return IE_ERR_ARG; }
    DeviceGuard g(w->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    IE_TRY(ensure_buffers(w, B, n));
    const long long cnt = (long long)B * n * n * 2;
    DevBuf tmp;
    IE_TRY(tmp.alloc(sizeof(float) * cnt, s));
    IE_TRY_CUDA(cudaMemcpyAsync(tmp.ptr, in, sizeof(float) * cnt, cudaMemcpyDefault, s));
    to_bf16<<<blocks_for(cnt), 256, 0, s>>>(tmp.as<float>(), w->act[A_IN], cnt);
    IE_LAUNCHED();
    IE_TRY(forward(w, B, n, s));
    IE_TRY_CUDA(cudaMemcpyAsync(w->dout, dout, sizeof(float) * B * n * n, cudaMemcpyDefault, s));
    IE_TRY(backward(w, B, n, s));
    IE_TRY_CUDA(cudaMemcpyAsync(grad, w->g, sizeof(float) * w->nparams, cudaMemcpyDefault, s));
    IE_TRY_CUDA(cudaStreamSynchronize(s));
    return take_tc_error(w, "ws_backward_raw");
}

extern "C" int ws_train_step(ws_model *w, const ie_problem *p, const double *f, const double *u, int batch, long long ld,
                             float lr, double *loss, void *stream) {
    if (!p || p->dim != 2) { ie_set_error("ws_train_step: needs a 2D problem"); return IE_ERR_ARG; }
    IE_TRY(check_grid(w, p->n));
    if (batch < 1 || batch > kMaxBatch || !f || !u || ld < p->N) { ie_set_error("ws_train_step: bad arguments"); return IE_ERR_ARG; }
    if (!ie_is_device_ptr(f) || !ie_is_device_ptr(u)) { ie_set_error("ws_train_step: f and u must be device memory"); return IE_ERR_ARG; }
    DeviceGuard g(w->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    IE_TRY(ensure_buffers(w, batch, p->n));
    IE_TRY(prepare(w, p, f, ld, u, ld, batch, s));
    IE_TRY(forward(w, batch, p->n, s));
    const long long cnt = (long long)batch * p->N;
    IE_TRY_CUDA(cudaMemsetAsync(w->loss, 0, sizeof(double), s));
    mse_grad<<<std::min<unsigned>(blocks_for(cnt), 1024), 256, 0, s>>>(w->out, w->tgt, w->dout, cnt, w->loss);
    IE_LAUNCHED();
    IE_TRY(backward(w, batch, p->n, s));
    w->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)w->step), c2 = 1.f - std::pow(b2, (float)w->step);
    adam_step<<<blocks_for(w->nparams), 256, 0, s>>>(w->w32, w->m, w->v, w->g, w->w16, w->nparams, lr, b1, b2, 1e-8f, c1, c2);
    IE_LAUNCHED();
    if (loss) {
        IE_TRY_CUDA(cudaMemcpyAsync(loss, w->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        IE_TRY_CUDA(cudaStreamSynchronize(s));
        return take_tc_error(w, "ws_train_step");
    }
    return IE_OK;
}

extern "C" int ws_predict(ws_model *w, const ie_problem *p, const double *f, double *u0, int nrhs, long long ld,
                          void *stream) {
    if (!p || p->dim != 2) { ie_set_error("ws_predict: needs a 2D problem"); return IE_ERR_ARG; }
    IE_TRY(check_grid(w, p->n));
    if (nrhs < 1 || !f || !u0 || ld < p->N) { ie_set_error("ws_predict: bad arguments"); return IE_ERR_ARG; }
    if (!ie_is_device_ptr(f) || !ie_is_device_ptr(u0)) { ie_set_error("ws_predict: f and u0 must be device memory"); return IE_ERR_ARG; }
    DeviceGuard g(w->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int k0 = 0; k0 < nrhs; k0 += kMaxBatch) {
        const int B = std::min(kMaxBatch, nrhs - k0);
        IE_TRY(ensure_buffers(w, B, p->n));
        IE_TRY(prepare(w, p, f + (long long)k0 * ld, ld, nullptr, 0, B, s));
        IE_TRY(forward(w, B, p->n, s));
        dim3 gg(blocks_for(p->N), B);
        unscale_output<<<gg, 256, 0, s>>>(w->out, w->ffll + kMaxBatch, 1.0 / (p->h * p->h), u0 + (long long)k0 * ld, ld, p->N);
        IE_LAUNCHED();
    }
    return IE_OK;
}
