// dd_apply: z = T^{-1} r = sum_i R_i^T L_i^{-T} L_i^{-1} R_i r  (Eq. e:ad).
//
// K6 apply_blocks   one CTA of 256 threads per (subdomain, right-hand side): gather R_i r into
//                   shared memory, forward solve with L_i and backward solve with L_i^T, 32-row
//                   tiles at a time.  The off-diagonal part of each tile step is a GEMV spread
//                   over the 8 warps (coalesced reads of L rows); the 32 x 32 diagonal triangle is
//                   solved by one warp with shuffles.  L_i is read twice (both passes), which is
//                   the HBM traffic that bounds the step.  The block result goes to a scratch
//                   vector [rhs][sum n_i].
// K6s apply_split   (FP32 explicit inverses) per (subdomain, right-hand side): R_i r scaled by a
//                   power of two and split into FP32 hi/lo words, once per apply.
// K6i apply_inverse one CTA of 256 threads per (64 rows of a subdomain, group of R right-hand
//                   sides): z_i = M_i (R_i r) with the symmetric M_i = A_i^{-1} stored in FP32, a
//                   batched GEMV (R = 1) or GEMM (R = 4, 8) streaming M_i once per group, every row
//                   independent.  Products and sums are double-float (~2^-48 of the
//                   partial sums), so the operator applied is the fixed symmetric matrix M_i to
//                   working accuracy.  FP32 sums would not be: their error acts like a
//                   preconditioner that changes from one iteration to the next, and PCG slows
//                   down (by 2 iterations at 128^2 already with sums good to 2^-48 of the
//                   largest row sum instead of the partial sums).
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

// Double-float accumulation of one term m (h + l) into (s, c): p = m h rounded (kept out of any
// FMA contraction), its exact error and m l go to c together with the exact TwoSum error of
// s + p.  11 FP32 operations; the sum is good to ~2^-48 of the partial sums' magnitudes.
__device__ __forceinline__ void df_fma(float &s, float &c, float m, float h, float l) {
    const float p = __fmul_rn(m, h);
    const float pe = fmaf(m, l, fmaf(m, h, -p));
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + pe;
}

// Butterfly sum of the (hi, lo) pairs of a group of kLPR lanes with exact TwoSum errors; every
// lane of the group ends with the same pair (the exact error of hi_a + hi_b does not depend on
// the order of the operands).
__device__ __forceinline__ void df_group_sum(float &hi, float &lo) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const float hs = __shfl_xor_sync(0xffffffffu, hi, o), ls = __shfl_xor_sync(0xffffffffu, lo, o);
        const float t = hi + hs;
        const float bp = t - hi;
        const float err = (hi - (t - bp)) + (hs - bp);
        hi = t;
        lo = (lo + ls) + err;
    }
}

// x 2^e, exact whenever the result is a normal double: two multiplies by powers of two built
// from their bits (each half of e stays in the normal exponent range), instead of ldexp.
__device__ __forceinline__ double pow2_bits(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
__device__ __forceinline__ double scale2(double x, int e) {
    const int e1 = e / 2;
    return (x * pow2_bits(e1)) * pow2_bits(e - e1);
}

// K6s: x = r 2^-e per (subdomain, right-hand side), e the exponent with max_a |r_a| < 2^e (an exact
// scaling: the FP32 words of x neither overflow nor lose bits to underflow whatever the scale of
// r), split into FP32 hi and (LO) lo words, padded with zeros to the block's padded size.
template <bool LO>
__global__ void __launch_bounds__(256)
apply_split(const int *__restrict__ npad, const int *__restrict__ nb, const long long *__restrict__ offs,
            const int *__restrict__ idx, const long long *__restrict__ xoff, const double *__restrict__ r,
            long long ldr, long long xtotal, int nblocks, float *__restrict__ xh, float *__restrict__ xl,
            int *__restrict__ xexp) {
    __shared__ double wmax[8];
    __shared__ int se;
    const int b = blockIdx.x, k = blockIdx.y;
    const int np = npad[b], n = nb[b];
    const int *id = idx + offs[b];
    const double *rk = r + (long long)k * ldr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double m = 0.0;
    for (int a = tid; a < n; a += 256) m = fmax(m, fabs(rk[id[a]]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    if (tid == 0) {
        double mm = 0.0;
        for (int w = 0; w < 8; ++w) mm = fmax(mm, wmax[w]);
        int e = 0;
        frexp(mm, &e);  // mm = f 2^e, f in [0.5, 1)
        se = e;
        xexp[(long long)k * nblocks + b] = e;
    }
    __syncthreads();
    const long long base = (long long)k * xtotal + xoff[b];
    for (int a = tid; a < np; a += 256) {
        const double x = a < n ? scale2(rk[id[a]], -se) : 0.0;
        const float h = (float)x;
        xh[base + a] = h;
        if (LO) xl[base + a] = (float)(x - (double)h);
    }
}

// K6i: one CTA per (chunk of `rows` rows of one subdomain, group of R right-hand sides).  The
// CTA stages the block's split x for its R columns in shared memory.  A row is taken by LPR = 8
// lanes (the padded size is a multiple of 32, so every lane has the same np/32 float4 columns:
// lane c of the group reads float4 columns c, c + 8, ...); a warp covers 4 x RW rows per pass,
// the 4 row groups reading the same x words (shared-memory broadcast), U float4 loads per lane
// and row issued before any arithmetic.  The column order of every sum is the same for every R,
// so a column's result does not depend on how many right-hand sides share the pass.  EXACT:
// double-float products and sums (df_fma); otherwise FP32 FMAs on the hi words.  The FP64
// conversion of each result runs in one lane only (FP64 is 1/64 of the FP32 rate).
constexpr int kLPR = 8;

template <int R, int RW, int U, bool EXACT>
__device__ __forceinline__ void inverse_chunk(float (&s)[RW][R], float (&c)[RW][R], const float4 *const (&mrow)[RW],
                                              int u, int cl, int np4, const float4 *xh4, const float4 *xl4) {
    float4 m4[RW][U];
#pragma unroll
    for (int uu = 0; uu < U; ++uu)
#pragma unroll
        for (int q = 0; q < RW; ++q) m4[q][uu] = __ldg(mrow[q] + (u + uu) * kLPR);
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
        const int c4 = cl + (u + uu) * kLPR;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const float4 h = xh4[j * np4 + c4];
            if (EXACT) {
                const float4 l = xl4[j * np4 + c4];
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                    df_fma(s[q][j], c[q][j], m4[q][uu].x, h.x, l.x);
                    df_fma(s[q][j], c[q][j], m4[q][uu].y, h.y, l.y);
                    df_fma(s[q][j], c[q][j], m4[q][uu].z, h.z, l.z);
                    df_fma(s[q][j], c[q][j], m4[q][uu].w, h.w, l.w);
                }
            } else {
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                    s[q][j] = fmaf(m4[q][uu].x, h.x, s[q][j]);
                    s[q][j] = fmaf(m4[q][uu].y, h.y, s[q][j]);
                    s[q][j] = fmaf(m4[q][uu].z, h.z, s[q][j]);
                    s[q][j] = fmaf(m4[q][uu].w, h.w, s[q][j]);
                }
            }
        }
    }
}

template <int R, int RW, int U, bool EXACT>
__global__ void __launch_bounds__(256)
apply_inverse(const float *__restrict__ pool, const long long *__restrict__ loff, const int *__restrict__ npad,
              const int *__restrict__ nb, const long long *__restrict__ offs, const int2 *__restrict__ chunks,
              const long long *__restrict__ xoff, const float *__restrict__ xh_g, const float *__restrict__ xl_g,
              const int *__restrict__ xexp, long long xtotal, int nblocks, int nrhs, double *__restrict__ zbuf,
              long long total, int rows) {
    constexpr int SUB = 32 / kLPR;                  // row groups per warp
    constexpr int K = (RW * R + kLPR - 1) / kLPR;   // results per lane and pass
    extern __shared__ __align__(16) float xs[];     // x hi words [R][np], then (EXACT) lo words [R][np]
    const int2 ch = chunks[blockIdx.x];
    const int b = ch.x, row0 = ch.y;
    const int g0 = blockIdx.y * R;
    const int np = npad[b], n = nb[b];
    const int rend = min(row0 + rows, n);
    const float *M = pool + loff[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / kLPR, cl = lane % kLPR;
    const int np4 = np >> 2, cnt = np4 / kLPR;
    float4 *xh4 = reinterpret_cast<float4 *>(xs), *xl4 = xh4 + R * np4;
    for (int e = tid; e < R * np4; e += 256) {
        const int j = e / np4, c4 = e - j * np4;
        const long long src = ((long long)(g0 + j) * xtotal + xoff[b]) / 4 + c4;
        const bool ok = g0 + j < nrhs;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        xh4[e] = ok ? reinterpret_cast<const float4 *>(xh_g)[src] : zero;
        if (EXACT) xl4[e] = ok ? reinterpret_cast<const float4 *>(xl_g)[src] : zero;
    }
    __syncthreads();
    for (int a0 = row0 + warp * SUB * RW; a0 < rend; a0 += 8 * SUB * RW) {
        const int ab = a0 + sub * RW;  // first row of this lane's group
        const float4 *mrow[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q)
            mrow[q] = reinterpret_cast<const float4 *>(M + (long long)min(ab + q, n - 1) * np) + cl;
        float s[RW][R], c[RW][R];
#pragma unroll
        for (int q = 0; q < RW; ++q)
#pragma unroll
            for (int j = 0; j < R; ++j) { s[q][j] = 0.f; c[q][j] = 0.f; }
        int u = 0;
        for (; u + U <= cnt; u += U) inverse_chunk<R, RW, U, EXACT>(s, c, mrow, u, cl, np4, xh4, xl4);
        for (; u < cnt; ++u) inverse_chunk<R, RW, 1, EXACT>(s, c, mrow, u, cl, np4, xh4, xl4);
        float oh[K], ol[K];
#pragma unroll
        for (int t = 0; t < K; ++t) { oh[t] = 0.f; ol[t] = 0.f; }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                float hi = s[q][j], lo = c[q][j];
                if (EXACT) {
                    df_group_sum(hi, lo);
                } else {
#pragma unroll
                    for (int o = kLPR / 2; o > 0; o >>= 1) hi += __shfl_xor_sync(0xffffffffu, hi, o);
                }
                const int k = q * R + j;
                if (cl == k % kLPR) { oh[k / kLPR] = hi; ol[k / kLPR] = lo; }
            }
        }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int k = t * kLPR + cl, q = k / R, j = k % R;
            if (k < RW * R && ab + q < rend && g0 + j < nrhs)
                zbuf[(long long)(g0 + j) * total + offs[b] + ab + q] =
                    scale2((double)oh[t] + (double)ol[t], xexp[(long long)(g0 + j) * nblocks + b]);
        }
    }
}

// K6c: the exact single-column apply for blocks padded above kApplyColFrom points (the paper's CBD
// colour blocks).  Staging a whole block's split x would leave one CTA per SM to stream the
// inverse; here a work item is (block, kApplyColRows rows, kApplyColChunk columns) and stages only
// that slice (32 KB), so several CTAs share an SM.  Each item leaves its rows' partial double-float
// sums for its column chunk; apply_col_combine adds a row's chunk partials in FP64, in chunk
// order, and applies the block's scale.  The same rows and lanes as K6i otherwise (8 lanes per row,
// RW rows per lane group, U float4 loads in flight).
template <int RW, int U>
__global__ void __launch_bounds__(256)
apply_inverse_cols(const float *__restrict__ pool, const long long *__restrict__ loff, const int *__restrict__ npad,
                   const int *__restrict__ nb, const long long *__restrict__ offs, const int4 *__restrict__ items,
                   const long long *__restrict__ xoff, const float *__restrict__ xh_g, const float *__restrict__ xl_g,
                   long long xtotal, long long total, int maxcol, float2 *__restrict__ zpart) {
    constexpr int SUB = 32 / kLPR;
    constexpr int K = (RW + kLPR - 1) / kLPR;
    __shared__ __align__(16) float4 xs4[2 * kApplyColChunk / 4];  // hi words, then lo words
    const int4 it = items[blockIdx.x];
    const int b = it.x, row0 = it.y, col0 = it.z, chunk = it.w;
    const int k = blockIdx.y;  // right-hand side
    const int np = npad[b], n = nb[b];
    const int cw4 = min(kApplyColChunk, np - col0) >> 2;  // np and col0 are multiples of 32
    const int rend = min(row0 + kApplyColRows, n);
    const float *M = pool + loff[b] + col0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / kLPR, cl = lane % kLPR;
    const int cnt = cw4 / kLPR;
    float4 *xh4 = xs4, *xl4 = xs4 + kApplyColChunk / 4;
    const long long src0 = ((long long)k * xtotal + xoff[b] + col0) / 4;
    for (int e = tid; e < cw4; e += 256) {
        xh4[e] = reinterpret_cast<const float4 *>(xh_g)[src0 + e];
        xl4[e] = reinterpret_cast<const float4 *>(xl_g)[src0 + e];
    }
    __syncthreads();
    for (int a0 = row0 + warp * SUB * RW; a0 < rend; a0 += 8 * SUB * RW) {
        const int ab = a0 + sub * RW;
        const float4 *mrow[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q)
            mrow[q] = reinterpret_cast<const float4 *>(M + (long long)min(ab + q, n - 1) * np) + cl;
        float s[RW][1], c[RW][1];
#pragma unroll
        for (int q = 0; q < RW; ++q) { s[q][0] = 0.f; c[q][0] = 0.f; }
        int u = 0;
        for (; u + U <= cnt; u += U) inverse_chunk<1, RW, U, true>(s, c, mrow, u, cl, cw4, xh4, xl4);
        for (; u < cnt; ++u) inverse_chunk<1, RW, 1, true>(s, c, mrow, u, cl, cw4, xh4, xl4);
        float oh[K], ol[K];
#pragma unroll
        for (int t = 0; t < K; ++t) { oh[t] = 0.f; ol[t] = 0.f; }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            float hi = s[q][0], lo = c[q][0];
            df_group_sum(hi, lo);
            if (cl == q % kLPR) { oh[q / kLPR] = hi; ol[q / kLPR] = lo; }
        }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int q = t * kLPR + cl;
            if (q < RW && ab + q < rend)
                zpart[((long long)k * total + offs[b] + ab + q) * maxcol + chunk] = make_float2(oh[t], ol[t]);
        }
    }
}

// a row's chunk partials summed in FP64 in chunk order, scaled back by the block's 2^e
__global__ void apply_col_combine(const float2 *__restrict__ zpart, const int *__restrict__ npad,
                                  const int *__restrict__ nb, const long long *__restrict__ offs,
                                  const int *__restrict__ xexp, int nblocks, long long total, int maxcol,
                                  double *__restrict__ zbuf) {
    const int b = blockIdx.x, k = blockIdx.z;
    const int a = blockIdx.y * blockDim.x + threadIdx.x;
    if (a >= nb[b]) return;
    const int nch = (npad[b] + kApplyColChunk - 1) / kApplyColChunk;
    const long long row = (long long)k * total + offs[b] + a;
    const float2 *p = zpart + row * maxcol;
    double z = 0.0;
    for (int c = 0; c < nch; ++c) z += (double)p[c].x + (double)p[c].y;
    zbuf[row] = scale2(z, xexp[(long long)k * nblocks + b]);
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

// The explicit-inverse apply's candidate configurations: class (kApplyE1 / E4 / F8) x variant
// (rows per warp pass RW, float4 loads in flight U) x rows per work item (kApplyRowOpts).  Every
// candidate sums each row in the same order, so they differ in speed only.
#define IE_AINV_VARIANTS(X)                                                                         \
    X(0, 1, 2, 4, true) X(1, 1, 4, 2, true) X(2, 1, 1, 8, true)                                     \
    X(3, 4, 2, 2, true) X(4, 4, 1, 4, true) X(5, 4, 4, 1, true)                                     \
    X(6, 8, 2, 4, false) X(7, 8, 1, 4, false) X(8, 8, 4, 2, false)

int launch_apply_inverse(const dd_factor_t *f, int klass, int cfg, const float *xh, const float *xl, const int *xe,
                         int nrhs, double *zbuf, cudaStream_t s) {
    const dd_partition_t *part = f->part;
    const int v = cfg / 3, ri = cfg % 3;
    const unsigned nch = (unsigned)f->nchunks[ri];
    const float *M = (const float *)f->d_pool;
    switch (klass * 3 + v) {
#define IE_AINV_CASE(ID, R_, RW_, U_, EX_)                                                                     \
    case ID:                                                                                                  \
        apply_inverse<R_, RW_, U_, EX_><<<dim3(nch, (nrhs + R_ - 1) / R_), 256,                               \
                                          sizeof(float) * (EX_ ? 2 : 1) * R_ * f->max_pad, s>>>(              \
            M, f->d_loff, f->d_npad, f->d_n, part->d_offs, f->d_chunks[ri], f->d_xoff, xh, xl, xe, f->xtotal,  \
            f->nblocks, nrhs, zbuf, part->total, kApplyRowOpts[ri]);                                          \
        break;
        IE_AINV_VARIANTS(IE_AINV_CASE)
#undef IE_AINV_CASE
        default:
            ie_set_error("dd_apply: bad apply configuration");
            return IE_ERR_ARG;
    }
    IE_LAUNCHED();
    return IE_OK;
}

int prepare_apply(const dd_factor_t *f) {
    (void)f;
#define IE_AINV_ATTR(ID, R_, RW_, U_, EX_) \
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_inverse<R_, RW_, U_, EX_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_AINV_VARIANTS(IE_AINV_ATTR)
#undef IE_AINV_ATTR
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks_multi<double, double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks_multi<float, double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks_multi<float, float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(apply_blocks<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmemCeiling));
    return IE_OK;
}

int launch_apply(const dd_factor_t *f, const double *r, long long ldr, double *z, long long ldz, int nrhs,
                 cudaStream_t s) {
    if (f->rs) return launch_apply_rs(f, r, ldr, z, ldz, nrhs, s);
    const ie_problem *p = f->prob;
    const dd_partition_t *part = f->part;
    DevBuf zbuf;
    IE_TRY(zbuf.alloc(sizeof(double) * (size_t)std::max<long long>(part->total, 1) * nrhs, s));
    const size_t smm = sizeof(double) * f->max_pad * kRM;
    if (f->nblocks > 0 && f->inverse) {
        // 2D blocks, and single columns, get the double-float sums; batches of 3D columns FP32
        // the batched variants stage 32 bytes per point; larger blocks take the columns one by one
        const bool batch_fits = sizeof(float) * 8 * (size_t)f->max_pad <= (size_t)kApplySmemCeiling;
        const bool exact = p->dim == 2 || nrhs < 4 || !batch_fits;
        DevBuf xb, xe;
        IE_TRY(xb.alloc(sizeof(float) * (size_t)f->xtotal * nrhs * (exact ? 2 : 1), s));
        IE_TRY(xe.alloc(sizeof(int) * (size_t)f->nblocks * nrhs, s));
        float *xh = xb.as<float>(), *xl = exact ? xh + f->xtotal * nrhs : nullptr;
        dim3 gs(f->nblocks, nrhs);
        if (exact) {
            apply_split<true><<<gs, 256, 0, s>>>(f->d_npad, f->d_n, part->d_offs, part->d_idx, f->d_xoff, r, ldr,
                                                 f->xtotal, f->nblocks, xh, xl, xe.as<int>());
        } else {
            apply_split<false><<<gs, 256, 0, s>>>(f->d_npad, f->d_n, part->d_offs, part->d_idx, f->d_xoff, r, ldr,
                                                  f->xtotal, f->nblocks, xh, xl, xe.as<int>());
        }
        IE_LAUNCHED();
        const int klass = !exact ? kApplyF8 : (nrhs >= 4 && batch_fits) ? kApplyE4 : kApplyE1;
        if (klass == kApplyF8 && nrhs >= kApplyTensorFrom) {
            // 3D batches of 32 or more columns: GEMM tasks on the tensor cores (measured on GB300,
            // 32^3 blocks: 0.27 ms for 64 columns against 0.40 ms with FP32 FMAs; at 16 columns the
            // FMA kernel is faster)
            IE_TRY(launch_apply_tc(f, xh, xe.as<int>(), nrhs, zbuf.as<double>(), s));
        } else if (klass == kApplyE1 && f->ncitems > 0) {
            // large blocks: column-chunked work items, then the FP64 chunk sums
            DevBuf zp;
            IE_TRY(zp.alloc(sizeof(float2) * (size_t)part->total * nrhs * f->maxcol, s));
            apply_inverse_cols<2, 4><<<dim3((unsigned)f->ncitems, nrhs), 256, 0, s>>>(
                (const float *)f->d_pool, f->d_loff, f->d_npad, f->d_n, part->d_offs, f->d_citems, f->d_xoff, xh, xl,
                f->xtotal, part->total, f->maxcol, zp.as<float2>());
            IE_LAUNCHED();
            apply_col_combine<<<dim3(f->nblocks, (part->max_block + 255) / 256, nrhs), 256, 0, s>>>(
                zp.as<float2>(), f->d_npad, f->d_n, part->d_offs, xe.as<int>(), f->nblocks, part->total, f->maxcol,
                zbuf.as<double>());
            IE_LAUNCHED();
        } else if (f->nchunks[0] > 0) {
            IE_TRY(launch_apply_inverse(f, klass, f->apply_cfg[klass], xh, xl, xe.as<int>(), nrhs, zbuf.as<double>(), s));
        }
    } else if (f->nblocks > 0 && nrhs >= 4 && smm <= (size_t)kApplySmemCeiling) {
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

// Times every configuration of each apply class this factor uses (a zero input: the kernels are
// data-independent) on its own stream position, keeps the fastest, and caches the choice for the
// partition's shape.  Runs at factor time, outside any capture.
int tune_apply(dd_factor_t *f, cudaStream_t s) {
    for (int k = 0; k < 3; ++k) f->apply_cfg[k] = 1;  // variant 0, 64-row work items
    if (!autotune_enabled() || !f->inverse || f->nblocks == 0) return IE_OK;
    const ie_problem *p = f->prob;
    const dd_partition_t *part = f->part;
    const bool batch_fits = sizeof(float) * 8 * (size_t)f->max_pad <= (size_t)kApplySmemCeiling;
    const std::string shape = "d" + std::to_string(p->dim) + "/n" + std::to_string(p->n) + "/blocks" +
                              std::to_string(f->nblocks) + "/total" + std::to_string(part->total) + "/max" +
                              std::to_string(f->max_pad);
    struct Cls { int klass, nrhs; bool use; };
    const Cls classes[3] = {{kApplyE1, 1, f->ncitems == 0}, {kApplyE4, 8, p->dim == 2 && batch_fits},
                            {kApplyF8, 8, p->dim == 3 && batch_fits}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    IE_TRY_CUDA(cudaEventCreate(&e0));
    IE_TRY_CUDA(cudaEventCreate(&e1));
    int st = IE_OK;
    for (const Cls &c : classes) {
        if (!c.use) continue;
        const std::string key = "apply/" + std::to_string(c.klass) + "/" + shape;
        int best = 1;
        if (tune_get(key, &best)) { f->apply_cfg[c.klass] = best; continue; }
        DevBuf r, z;
        if ((st = r.alloc(sizeof(double) * (size_t)p->N * c.nrhs, s)) != IE_OK) break;
        if ((st = z.alloc(sizeof(double) * (size_t)p->N * c.nrhs, s)) != IE_OK) break;
        if (cudaMemsetAsync(r.ptr, 0, sizeof(double) * (size_t)p->N * c.nrhs, s) != cudaSuccess) { st = IE_ERR_CUDA; break; }
        float best_ms = 0.f;
        std::string detail;
        for (int cand = 0; cand < 9 && st == IE_OK; ++cand) {
            f->apply_cfg[c.klass] = cand;
            if ((st = launch_apply(f, r.as<double>(), p->N, z.as<double>(), p->N, c.nrhs, s)) != IE_OK) break;
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 3 && st == IE_OK; ++rep)
                st = launch_apply(f, r.as<double>(), p->N, z.as<double>(), p->N, c.nrhs, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = IE_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            detail += (cand ? " " : "") + std::to_string(cand) + ":" + std::to_string((int)(ms * 1000.f)) + "us";
            if (cand == 0 || ms < best_ms) { best_ms = ms; best = cand; }
        }
        if (st != IE_OK) break;
        f->apply_cfg[c.klass] = best;
        tune_put(key, best, detail);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IE_OK) for (int k = 0; k < 3; ++k) f->apply_cfg[k] = 1;
    return st;
}
