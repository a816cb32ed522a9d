// Stored-matrix fallback matvec: A is materialised once in HBM (FP32, dense row-major, zero
// diagonal) and each product streams it: y = diag x + A_off x.  The diagonal stays FP64.
//
// K3 k3_gemv_f32   a CTA of 256 threads owns 8 rows; per 2048-column chunk it stages x (FP32)
//                  in shared memory once and each warp streams one row's chunk with 16-byte
//                  loads, 4-way unrolled, FP32 partial sums per lane reduced with shuffles and
//                  accumulated in FP64 per chunk.  Bound: HBM, 4 N^2 bytes per product.
//
// Entries come from the per-offset FP64 table (the matrix of the uniform grid is Toeplitz in
// each coordinate), rounded to FP32.
#include <cuda_runtime.h>

#include <string>

#include "iedd_internal.cuh"

namespace {

constexpr int kRowsPerCta = 8;
constexpr int kChunk = 2048;

// rows row0 + blockIdx.y of A (A points at row row0)
__global__ void build_stored(float *__restrict__ A, const double *__restrict__ table64, int dim, int n, long long N,
                             long long row0) {
    const long long i = row0 + blockIdx.y;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (j != i) {
            long long a = i, b = j, mul = 1;
            // |offset| per coordinate, as the index of the n^dim table (last coordinate fastest)
            long long idx = 0;
            for (int d = 0; d < dim; ++d) {
                const long long ca = a % n, cb = b % n;
                a /= n;
                b /= n;
                idx += (ca > cb ? ca - cb : cb - ca) * mul;
                mul *= n;
            }
            v = (float)table64[idx];
        }
        A[(long long)blockIdx.y * N + j] = v;
    }
}

__global__ void __launch_bounds__(256)
k3_gemv_f32(const float *__restrict__ A, const double *__restrict__ x, double diag, double *__restrict__ y, long long N) {
    __shared__ __align__(16) float xs[kChunk];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * kRowsPerCta + warp;
    const bool active = row < N;
    double acc = 0.0;
    for (long long c0 = 0; c0 < N; c0 += kChunk) {
        const int len = (int)(N - c0 < kChunk ? N - c0 : kChunk);
        __syncthreads();
        for (int e = threadIdx.x; e < kChunk; e += 256) xs[e] = e < len ? (float)x[c0 + e] : 0.f;
        __syncthreads();
        if (active) {
            const float *ar = A + row * N + c0;
            float s = 0.f;
            if ((N & 3) == 0) {
                const float4 *a4 = reinterpret_cast<const float4 *>(ar);
                const float4 *x4 = reinterpret_cast<const float4 *>(xs);
                const int n4 = len / 4;
#pragma unroll 4
                for (int k = lane; k < n4; k += 32) {
                    const float4 av = __ldcs(a4 + k), xv = x4[k];
                    s = fmaf(av.x, xv.x, s);
                    s = fmaf(av.y, xv.y, s);
                    s = fmaf(av.z, xv.z, s);
                    s = fmaf(av.w, xv.w, s);
                }
            } else {
                for (int k = lane; k < len; k += 32) s = fmaf(__ldcs(ar + k), xs[k], s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            acc += (double)s;
        }
    }
    if (active && lane == 0) y[row] = fma(diag, x[row], acc);
}

}  // namespace

extern "C" int ie_store_matrix(ie_problem *p, void *stream) {
    if (!p) { ie_set_error("ie_store_matrix: NULL problem"); return IE_ERR_ARG; }
    DeviceGuard g(p->device);
    if (p->d_stored) return IE_OK;
    const double bytes = 4.0 * (double)p->N * (double)p->N;
    size_t freeb = 0, totalb = 0;
    IE_TRY_CUDA(cudaMemGetInfo(&freeb, &totalb));
    if (bytes > 0.9 * (double)freeb) {
        ie_set_error("ie_store_matrix: the dense FP32 matrix needs " + std::to_string(bytes / 1e9) + " GB, " +
                     std::to_string(freeb / 1e9) + " GB free");
        return IE_ERR_OOM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    IE_TRY_CUDA(cudaMalloc((void **)&p->d_stored, (size_t)bytes));
    const long long N = p->N;
    for (long long r0 = 0; r0 < N; r0 += 65535) {
        const unsigned rows = (unsigned)(N - r0 < 65535 ? N - r0 : 65535);
        dim3 gr((unsigned)((N + 255) / 256 < 64 ? (N + 255) / 256 : 64), rows);
        build_stored<<<gr, 256, 0, s>>>(p->d_stored + r0 * N, p->d_table64, p->dim, p->n, N, r0);
        IE_LAUNCHED();
    }
    IE_TRY_CUDA(cudaStreamSynchronize(s));
    return IE_OK;
}

extern "C" int ie_release_matrix(ie_problem *p) {
    if (!p) { ie_set_error("ie_release_matrix: NULL problem"); return IE_ERR_ARG; }
    DeviceGuard g(p->device);
    if (p->d_stored) IE_TRY_CUDA(cudaFree(p->d_stored));
    p->d_stored = nullptr;
    return IE_OK;
}

int launch_matvec_stored(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy, int nrhs,
                         cudaStream_t s) {
    if (!p->d_stored) { ie_set_error("ie_matvec: IE_STORED needs ie_store_matrix first"); return IE_ERR_ARG; }
    const long long N = p->N;
    const unsigned blocks = (unsigned)((N + kRowsPerCta - 1) / kRowsPerCta);
    for (int k = 0; k < nrhs; ++k) {
        k3_gemv_f32<<<blocks, 256, 0, s>>>(p->d_stored, x + (long long)k * ldx, p->diag, y + (long long)k * ldy, N);
        IE_LAUNCHED();
    }
    return IE_OK;
}
