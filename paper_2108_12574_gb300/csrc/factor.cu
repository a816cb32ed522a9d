// dd_factor: regenerate every subdomain block A_i = R_i A R_i^T (Eq. e:ai) and factor it by
// dense Cholesky, A_i = L_i L_i^T (the exact subdomain solver of Sec. 4.3), all blocks at once.
//
// Storage: block i is padded to npad_i = 32 * ceil(n_i / 32) with an identity in the padding
// (so its factor is diag(L_i, I) and every tile is full), row-major, at d_loff[i] in one pool.
//
// K4 gather_blocks   one thread per entry (a, c), c <= a: the entry of the problem's per-offset FP64
//                    table at the integer lattice offset of points idx[a], idx[c] (the same FP64
//                    values as every matvec's), rounded once to the factor's type; the upper part
//                    is zeroed.
// K5 chol_blocked    one CTA of 256 threads per block (largest blocks first), right-looking
//                    blocked Cholesky with 32 x 32 tiles: factor the diagonal tile in shared
//                    memory, solve the panel below it (one warp per row, lanes = columns), then
//                    the symmetric rank-32 update of the trailing lower tiles (tile pairs staged
//                    in shared memory).  The first non-positive pivot is recorded in info and
//                    the block stops.
// K5t (tc_factor.cu) for FP32 factors applied through explicit inverses: the same Cholesky and
//                    the inverse M_i = L_i^{-T} L_i^{-1} with the bulk on the tensor cores.
#include <cuda_runtime.h>

#include <algorithm>

#include "iedd_internal.cuh"

namespace {

template <typename T>
__global__ void gather_blocks(T *__restrict__ pool, const long long *__restrict__ loff,
                              const int *__restrict__ npad, const int *__restrict__ nb,
                              const long long *__restrict__ offs, const int *__restrict__ idx,
                              const float4 *__restrict__ coord, const double *__restrict__ t64, int n) {
    const int b = blockIdx.x;
    const int np = npad[b], nbk = nb[b];
    T *A = pool + loff[b];
    const int *id = idx + offs[b];
    const long long total = (long long)np * np;
    for (long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.y * blockDim.x) {
        const int a = (int)(e / np), c = (int)(e % np);
        T v = 0;
        if (c > a) {
            v = 0;
        } else if (a >= nbk || c >= nbk) {
            v = (a == c) ? T(1) : T(0);
        } else {
            // the entry of the per-offset FP64 table at the integer lattice offset (exact small
            // integers in the coordinates; entry 0 is the diagonal), rounded once to T
            const float4 pa = coord[id[a]], pc = coord[id[c]];
            const long long dx = (long long)fabsf(pa.x - pc.x), dy = (long long)fabsf(pa.y - pc.y),
                            dz = (long long)fabsf(pa.z - pc.z);
            v = (T)t64[dx + n * (dy + (long long)n * dz)];
        }
        A[e] = v;
    }
}

template <typename T> __device__ __forceinline__ T tsqrt(T v);
template <> __device__ __forceinline__ float tsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double tsqrt<double>(double v) { return sqrt(v); }

template <typename T>
__global__ void __launch_bounds__(256)
chol_blocked(T *__restrict__ pool, const long long *__restrict__ loff, const int *__restrict__ npad,
             const int *__restrict__ order, int *__restrict__ info) {
    __shared__ T D[32][33];
    __shared__ T P1[32][33];
    __shared__ T P2[32][33];
    __shared__ int bad;
    const int b = order[blockIdx.x];
    const int np = npad[b], nt = np / 32;
    T *A = pool + loff[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) bad = -1;
    __syncthreads();
    for (int k = 0; k < nt; ++k) {
        const int k0 = k * 32;
        // 1. diagonal tile -> shared
        for (int e = tid; e < 1024; e += 256) D[e >> 5][e & 31] = A[(long long)(k0 + (e >> 5)) * np + k0 + (e & 31)];
        __syncthreads();
        // 2. unblocked Cholesky of the tile (column by column)
        for (int j = 0; j < 32; ++j) {
            if (tid == 0) {
                T piv = D[j][j];
                if (!(piv > T(0))) bad = k0 + j;
                D[j][j] = tsqrt(piv > T(0) ? piv : T(1));
            }
            __syncthreads();
            if (bad >= 0) break;
            if (tid > j && tid < 32) D[tid][j] /= D[j][j];
            __syncthreads();
            for (int e = tid; e < 1024; e += 256) {
                const int i = e >> 5, c = e & 31;
                if (c > j && i >= c) D[i][c] -= D[i][j] * D[c][j];
            }
            __syncthreads();
        }
        if (bad >= 0) break;
        for (int e = tid; e < 1024; e += 256) {
            const int i = e >> 5, c = e & 31;
            if (c <= i) A[(long long)(k0 + i) * np + k0 + c] = D[i][c];
        }
        // 3. panel solve: rows below, X L_kk^T = A_panel (one warp per row, lane = column)
        for (int row = k0 + 32 + warp; row < np; row += 8) {
            T *ar = A + (long long)row * np + k0;
            T v = ar[lane];
            for (int c = 0; c < 32; ++c) {
                const T xc = __shfl_sync(0xffffffffu, v, c) / D[c][c];
                if (lane == c) v = xc;
                if (lane > c) v -= xc * D[lane][c];
            }
            ar[lane] = v;
        }
        __syncthreads();
        // 4. trailing update of the lower tiles: A_ij -= P_i P_j^T, k < j <= i < nt
        for (int i = k + 1; i < nt; ++i) {
            for (int e = tid; e < 1024; e += 256)
                P1[e >> 5][e & 31] = A[(long long)(i * 32 + (e >> 5)) * np + k0 + (e & 31)];
            for (int j = k + 1; j <= i; ++j) {
                __syncthreads();
                for (int e = tid; e < 1024; e += 256)
                    P2[e >> 5][e & 31] = A[(long long)(j * 32 + (e >> 5)) * np + k0 + (e & 31)];
                __syncthreads();
                // thread: row r = tid / 8, columns c = (tid % 8) + 8 q, q = 0..3
                const int r = tid >> 3, cb = tid & 7;
                T acc[4] = {0, 0, 0, 0};
#pragma unroll 8
                for (int t = 0; t < 32; ++t) {
                    const T pr = P1[r][t];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += pr * P2[cb + 8 * q][t];
                }
                T *dst = A + (long long)(i * 32 + r) * np + j * 32;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = cb + 8 * q;
                    if (i != j || c <= r) dst[c] -= acc[q];
                }
            }
            __syncthreads();
        }
        __syncthreads();
    }
    if (tid == 0) info[b] = bad;
}

}  // namespace

int launch_factor(dd_factor_t *f, cudaStream_t s) {
    const ie_problem *p = f->prob;
    const dd_partition_t *part = f->part;
    if (f->nblocks == 0) return IE_OK;
    // enough CTAs per block for the largest one (CBD colour blocks hold up to 6.5e8 entries)
    const long long ent = (long long)f->max_pad * f->max_pad;
    dim3 g(f->nblocks, (unsigned)std::min<long long>(65535, std::max<long long>(64, ent / (256LL * 1024))));
    if (f->precision == IE_FP64) {
        gather_blocks<double><<<g, 256, 0, s>>>((double *)f->d_pool, f->d_loff, f->d_npad, f->d_n, part->d_offs,
                                                part->d_idx, p->d_coord, p->d_table64, p->n);
        IE_LAUNCHED();
        chol_blocked<double><<<f->nblocks, 256, 0, s>>>((double *)f->d_pool, f->d_loff, f->d_npad, f->d_order,
                                                       f->d_info);
        IE_LAUNCHED();
    } else {
        gather_blocks<float><<<g, 256, 0, s>>>((float *)f->d_pool, f->d_loff, f->d_npad, f->d_n, part->d_offs,
                                               part->d_idx, p->d_coord, p->d_table64, p->n);
        IE_LAUNCHED();
        if (f->inverse) return IE_OK;  // Cholesky and inverse on the tensor cores (launch_factor_tc)
        chol_blocked<float><<<f->nblocks, 256, 0, s>>>((float *)f->d_pool, f->d_loff, f->d_npad, f->d_order,
                                                      f->d_info);
        IE_LAUNCHED();
    }
    return IE_OK;
}
