// dd_apply: z = T^{-1} r = sum_i R_i^T L_i^{-T} L_i^{-1} R_i r  (Eq. e:ad).
//
// K6 apply_blocks   one CTA of 256 threads per (subdomain, right-hand side): gather R_i r into
//                   shared memory, forward solve with L_i and backward solve with L_i^T, 32-row
//                   tiles at a time.  The off-diagonal part of each tile step is a GEMV spread
//                   over the 8 warps (coalesced reads of L rows); the 32 x 32 diagonal triangle is
//                   solved by one warp with shuffles.  L_i is read twice (both passes), which is
//                   the HBM traffic that bounds the step.  The block result goes to a scratch
//                   vector [rhs][sum n_i].
// K6b overlap_sum   z_p = sum of the block results of every subdomain containing p, in increasing
//                   subdomain order (inverse index map), so the sum is deterministic.
#include <cuda_runtime.h>

#include "iedd_internal.cuh"

namespace {

// TL: storage type of the factor; T: arithmetic type of the solves.  FP32 factors are solved in
// FP64 arithmetic: FP32 substitution is not symmetric to working accuracy (its error grows with
// cond(A_i) ~ 1e3), and an operator T^{-1} that is not symmetric slows PCG down measurably.
template <typename TL, typename T>
__global__ void __launch_bounds__(256)
apply_blocks(const TL *__restrict__ pool, const long long *__restrict__ loff, const int *__restrict__ npad,
             const int *__restrict__ nb, const long long *__restrict__ offs, const int *__restrict__ idx,
             const int *__restrict__ order, const double *__restrict__ r, long long ldr,
             double *__restrict__ zbuf, long long total) {
    extern __shared__ unsigned char smem_raw[];
    T *Y = reinterpret_cast<T *>(smem_raw);
    __shared__ T D[32][33];
    __shared__ T red[8][32];
    const int b = order[blockIdx.x];
    const int k = blockIdx.y;
    const int np = npad[b], n = nb[b], nt = np / 32;
    const TL *L = pool + loff[b];
    const int *id = idx + offs[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *rk = r + (long long)k * ldr;
    for (int a = tid; a < np; a += 256) Y[a] = a < n ? (T)rk[id[a]] : T(0);
    __syncthreads();

    // forward: L y = R_i r
    for (int t = 0; t < nt; ++t) {
        const int t0 = t * 32;
        for (int e = tid; e < 1024; e += 256) D[e >> 5][e & 31] = (T)L[(long long)(t0 + (e >> 5)) * np + t0 + (e & 31)];
        for (int q = 0; q < 4; ++q) {
            const int row = t0 + warp + 8 * q;
            const TL *lr = L + (long long)row * np;
            T s = 0;
            for (int c = lane; c < t0; c += 32) s += (T)lr[c] * Y[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) red[0][warp + 8 * q] = s;
        }
        __syncthreads();
        if (warp == 0) {
            T v = Y[t0 + lane] - red[0][lane];
            for (int j = 0; j < 32; ++j) {
                const T yj = __shfl_sync(0xffffffffu, v, j) / D[j][j];
                if (lane == j) v = yj;
                if (lane > j) v -= D[lane][j] * yj;
            }
            Y[t0 + lane] = v;
        }
        __syncthreads();
    }
    // backward: L^T z = y
    for (int t = nt - 1; t >= 0; --t) {
        const int t0 = t * 32;
        for (int e = tid; e < 1024; e += 256) D[e >> 5][e & 31] = (T)L[(long long)(t0 + (e >> 5)) * np + t0 + (e & 31)];
        T part = 0;
        for (int row = t0 + 32 + warp; row < np; row += 8) part += (T)L[(long long)row * np + t0 + lane] * Y[row];
        red[warp][lane] = part;
        __syncthreads();
        if (warp == 0) {
            T sacc = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) sacc += red[w][lane];
            T v = Y[t0 + lane] - sacc;
            for (int j = 31; j >= 0; --j) {
                const T zj = __shfl_sync(0xffffffffu, v, j) / D[j][j];
                if (lane == j) v = zj;
                if (lane < j) v -= D[j][lane] * zj;
            }
            Y[t0 + lane] = v;
        }
        __syncthreads();
    }
    double *zk = zbuf + (long long)k * total + offs[b];
    for (int a = tid; a < n; a += 256) zk[a] = (double)Y[a];
}

// K6m apply_blocks_multi: one CTA per (subdomain, group of R right-hand sides).  The factor is
// read once per group instead of once per right-hand side: each 32-row step stages 32 x 32
// tiles of L in shared memory and applies them to all R columns held in shared memory (GEMM
// updates, thread (row, column group) accumulating 4 columns), then solves the 32 x 32
// triangle for the R columns (R / 8 columns per warp).  Arithmetic type T: FP64 (R = 16) for
// FP64 factors and for 2D, FP32 (R = 32) for FP32 factors of 3D problems, whose blocks and
// operator are well conditioned (cond(A) = O(N^{2/3})) so that FP32 substitution does not slow PCG.
constexpr int kRM = 16;  // right-hand sides per CTA (FP64 arithmetic); 32 in FP32

template <typename TL, typename T, int R>
__global__ void __launch_bounds__(256)
apply_blocks_multi(const TL *__restrict__ pool, const long long *__restrict__ loff, const int *__restrict__ npad,
                   const int *__restrict__ nb, const long long *__restrict__ offs, const int *__restrict__ idx,
                   const int *__restrict__ order, const double *__restrict__ r, long long ldr, int nrhs,
                   double *__restrict__ zbuf, long long total) {
    extern __shared__ __align__(16) unsigned char ysm_raw[];
    T *Ysm = reinterpret_cast<T *>(ysm_raw);  // [npad][R]
    __shared__ T Lt[32][33];
    constexpr int JQ = R / 8;  // columns per thread in the updates
    const int b = order[blockIdx.x];
    const int g0 = blockIdx.y * R;
    const int np = npad[b], n = nb[b], nt = np / 32;
    const TL *L = pool + loff[b];
    const int *id = idx + offs[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < np * R; e += 256) {
        const int a = e / R, j = e % R;
        Ysm[e] = (a < n && g0 + j < nrhs) ? (T)r[(long long)(g0 + j) * ldr + id[a]] : T(0);
    }
    __syncthreads();
    // thread layout for the updates: rr = tid / 8 (tile row 0..31), jq = tid % 8 -> columns JQ jq + q
    const int rr = tid >> 3, jq = tid & 7;
    // forward: L y = R_i r
    for (int t = 0; t < nt; ++t) {
        const int t0 = t * 32;
        T acc[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) acc[q] = T(0);
        for (int c0 = 0; c0 < t0; c0 += 32) {
            __syncthreads();
            for (int e = tid; e < 1024; e += 256) Lt[e >> 5][e & 31] = (T)L[(long long)(t0 + (e >> 5)) * np + c0 + (e & 31)];
            __syncthreads();
#pragma unroll 8
            for (int c = 0; c < 32; ++c) {
                const T l = Lt[rr][c];
#pragma unroll
                for (int q = 0; q < JQ; ++q) acc[q] = fma(l, Ysm[(c0 + c) * R + JQ * jq + q], acc[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < JQ; ++q) Ysm[(t0 + rr) * R + JQ * jq + q] -= acc[q];
        for (int e = tid; e < 1024; e += 256) Lt[e >> 5][e & 31] = (T)L[(long long)(t0 + (e >> 5)) * np + t0 + (e & 31)];
        __syncthreads();
        // triangle: warp w solves columns w R/8 .. (w+1) R/8 - 1 (lanes = rows)
        for (int q = 0; q < JQ; ++q) {
            const int j = JQ * warp + q;
            T v = Ysm[(t0 + lane) * R + j];
            for (int i = 0; i < 32; ++i) {
                const T yi = __shfl_sync(0xffffffffu, v, i) / Lt[i][i];
                if (lane == i) v = yi;
                if (lane > i) v -= Lt[lane][i] * yi;
            }
            Ysm[(t0 + lane) * R + j] = v;
        }
        __syncthreads();
    }
    // backward: L^T z = y
    for (int t = nt - 1; t >= 0; --t) {
        const int t0 = t * 32;
        T acc[JQ];
#pragma unroll
        for (int q = 0; q < JQ; ++q) acc[q] = T(0);
        for (int r0 = t0 + 32; r0 < np; r0 += 32) {
            __syncthreads();
            for (int e = tid; e < 1024; e += 256) Lt[e >> 5][e & 31] = (T)L[(long long)(r0 + (e >> 5)) * np + t0 + (e & 31)];
            __syncthreads();
#pragma unroll 8
            for (int qq = 0; qq < 32; ++qq) {
                const T l = Lt[qq][rr];  // L[r0 + qq][t0 + rr]
#pragma unroll
                for (int q = 0; q < JQ; ++q) acc[q] = fma(l, Ysm[(r0 + qq) * R + JQ * jq + q], acc[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < JQ; ++q) Ysm[(t0 + rr) * R + JQ * jq + q] -= acc[q];
        for (int e = tid; e < 1024; e += 256) Lt[e >> 5][e & 31] = (T)L[(long long)(t0 + (e >> 5)) * np + t0 + (e & 31)];
        __syncthreads();
        for (int q = 0; q < JQ; ++q) {
            const int j = JQ * warp + q;
            T v = Ysm[(t0 + lane) * R + j];
            for (int i = 31; i >= 0; --i) {
                const T zi = __shfl_sync(0xffffffffu, v, i) / Lt[i][i];
                if (lane == i) v = zi;
                if (lane < i) v -= Lt[i][lane] * zi;
            }
            Ysm[(t0 + lane) * R + j] = v;
        }
        __syncthreads();
    }
    for (int e = tid; e < n * R; e += 256) {
        const int a = e / R, j = e % R;
        if (g0 + j < nrhs) zbuf[(long long)(g0 + j) * total + offs[b] + a] = (double)Ysm[e];
    }
}

__global__ void overlap_sum(const double *__restrict__ zbuf, long long total, const long long *__restrict__ inv_ptr,
                            const long long *__restrict__ inv_pos, double *__restrict__ z, long long ldz, long long N) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= N) return;
    const double *zb = zbuf + (long long)k * total;
    double s = 0.0;
    for (long long q = inv_ptr[i]; q < inv_ptr[i + 1]; ++q) s += zb[inv_pos[q]];
    z[(long long)k * ldz + i] = s;
}

}  // namespace

// Raise the dynamic shared-memory limit of the apply kernels (outside any stream capture).  The
// opt-in is needed whenever static + dynamic shared memory exceeds 48 KB, and the attribute is
// per kernel for the whole process, so it is set to one fixed ceiling that covers every factor.
constexpr int kApplySmemCeiling = 200 * 1024;

int prepare_apply(const dd_factor_t *f) {
    (void)f;
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks_multi<double, double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks_multi<float, double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks_multi<float, float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    return IE_OK;
}

int launch_apply(const dd_factor_t *f, const double *r, long long ldr, double *z, long long ldz, int nrhs,
                 cudaStream_t s) {
    const ie_problem *p = f->prob;
    const dd_partition_t *part = f->part;
    DevBuf zbuf;
    IE_TRY(zbuf.alloc(sizeof(double) * (size_t)std::max<long long>(part->total, 1) * nrhs, s));
    const size_t smm = sizeof(double) * f->max_pad * kRM;
    if (f->nblocks > 0 && nrhs >= 4 && smm <= (size_t)kApplySmemCeiling) {
        if (f->precision == IE_FP64) {
            dim3 g(f->nblocks, (nrhs + 15) / 16);
            apply_blocks_multi<double, double, 16><<<g, 256, smm, s>>>((const double *)f->d_pool, f->d_loff, f->d_npad,
                                                                       f->d_n, part->d_offs, part->d_idx, f->d_order, r,
                                                                       ldr, nrhs, zbuf.as<double>(), part->total);
        } else if (p->dim == 2) {
            dim3 g(f->nblocks, (nrhs + 15) / 16);
            apply_blocks_multi<float, double, 16><<<g, 256, smm, s>>>((const float *)f->d_pool, f->d_loff, f->d_npad,
                                                                      f->d_n, part->d_offs, part->d_idx, f->d_order, r,
                                                                      ldr, nrhs, zbuf.as<double>(), part->total);
        } else {
            dim3 g(f->nblocks, (nrhs + 31) / 32);
            apply_blocks_multi<float, float, 32><<<g, 256, smm, s>>>((const float *)f->d_pool, f->d_loff, f->d_npad,
                                                                     f->d_n, part->d_offs, part->d_idx, f->d_order, r,
                                                                     ldr, nrhs, zbuf.as<double>(), part->total);
        }
        IE_LAUNCHED();
    } else if (f->nblocks > 0) {
        dim3 g(f->nblocks, nrhs);
        const size_t sm = sizeof(double) * f->max_pad;
        if (f->precision == IE_FP64) {
            apply_blocks<double, double><<<g, 256, sm, s>>>((const double *)f->d_pool, f->d_loff, f->d_npad, f->d_n, part->d_offs,
                                                   part->d_idx, f->d_order, r, ldr, zbuf.as<double>(), part->total);
            IE_LAUNCHED();
        } else {
            apply_blocks<float, double><<<g, 256, sm, s>>>((const float *)f->d_pool, f->d_loff, f->d_npad, f->d_n, part->d_offs,
                                                  part->d_idx, f->d_order, r, ldr, zbuf.as<double>(), part->total);
            IE_LAUNCHED();
        }
    }
    dim3 g2((unsigned)((p->N + 255) / 256), nrhs);
    overlap_sum<<<g2, 256, 0, s>>>(zbuf.as<double>(), part->total, part->d_inv_ptr, part->d_inv_pos, z, ldz, p->N);
    IE_LAUNCHED();
    return IE_OK;
}
