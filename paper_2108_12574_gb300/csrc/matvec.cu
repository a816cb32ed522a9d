// Matrix-free matvec y = A x for the collocation matrix of Sec. 2.1 (Eqs. e:a_2d, e:a_3d).
//
// All kernels work on the integer lattice offset D = i - j of two grid points (the points are
// x_j = offset + s * j, so x_i - x_j = s * D):
//   2D  A_ij = w K(s D) = c_const + c_ln ln|D|^2,    3D  A_ij = c_r / |D|,     i != j,
// and A_ii = the self-cell integral.  |D|^2 is an exact small integer in FP32 (|D|^2 < 2^24
// for n <= 2048 in 2D and n <= 2364 in 3D), so the only rounding in an FP32 entry is that of
// the SFU log2 / rsqrt, and the large constant c_const is kept out of the FP32 sums.
//
// K1  k1_matvec_f32      FP32 entries, one right-hand side.  Source points are staged through
//                        shared memory 256 at a time as float4 {D-coords, x_j}; each thread keeps
//                        R target rows in registers; per pair (2D): 2 FADD + 2 FFMA for
//                        |D|^2 + 2^-30, one SFU op (MUFU.LG2; MUFU.RSQ in 3D), FMUL, and a
//                        Kahan-compensated FP32 add (4 FADD).  Work is split over (row tile,
//                        column split) so the grid fills the GPU; each split's compensated sum
//                        goes to a [split][N] FP64 scratch and the splits are combined in FP64
//                        with the FP64 diagonal and constant terms.
// Kd  kd_matvec_f64      the same in FP64 with the natural log / rsqrt of double (plain FP64).
// K2  k2_accurate_{2d,3d} FP64-class y = A x from the per-|offset| entry table (translation
//                        invariance of A on the uniform grid): entry hi/lo FP32 pairs, products
//                        split exactly with FMA, sums as double-float (TwoSum) per 256-column
//                        tile, flushed to FP64 per tile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "iedd_internal.cuh"
#include "reduce.cuh"

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------------
// Problem tables
// ---------------------------------------------------------------------------------------------
__global__ void coord_kernel(float4 *coord, int dim, int n, long long N) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    long long t = i;
    float c[3] = {0.f, 0.f, 0.f};
    for (int d = dim - 1; d >= 0; --d) { c[d] = (float)(t % n); t /= n; }
    coord[i] = make_float4(c[0], c[1], c[2], 0.f);
}

// Entry for every |offset| (d_1, ..., d_dim) in [0, n)^dim, FP64, and its hi/lo FP32 split
// (zero at offset 0: see below).
__global__ void table_kernel(float2 *t32, double *t64, int dim, int n, long long T, double diag,
                             double c_const, double c_ln, double c_r) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= T) return;
    long long t = q;
    double r2 = 0.0;
    for (int d = 0; d < dim; ++d) { double v = (double)(t % n); r2 += v * v; t /= n; }
    double e;
    if (r2 == 0.0) e = diag;
    else if (dim == 2) e = c_const + c_ln * log(r2);
    else e = c_r / sqrt(r2);
    float hi = (float)e;
    float lo = (float)(e - (double)hi);
    // the double-float table leaves the diagonal out (it is added in FP64 by the final sum), so a
    // large diagonal (second-kind shift) does not coarsen the accumulation windows
    t32[q] = r2 == 0.0 ? make_float2(0.f, 0.f) : make_float2(hi, lo);
    t64[q] = e;
}

// ---------------------------------------------------------------------------------------------
// K1: FP32 SFU matvec, one right-hand side
// ---------------------------------------------------------------------------------------------
// 2D: the i = j pair is made harmless without a branch or a clamp: |D|^2 + 2^-30 equals |D|^2
// exactly for every |D|^2 >= 1, and is 2^-30 for i = j, whose term log2(2^-30) x_i the combine
// removes again (with the same SFU value).  3D clamps |D|^2 to >= 1 and removes rsqrt(1) x_i.
// The sums are compensated (Kahan): a plain FP32 running sum over thousands of terms of nearly
// equal magnitude loses the small result that the oscillatory search directions of PCG produce
// (their A p is ~1/cond(A) of ||A|| ||p||), which costs many iterations; the compensation keeps
// the sum at FP32-entry accuracy.  Intrinsics keep the compiler from re-associating it.
constexpr float kTiny2D = 0x1p-30f;

// Kahan step with the product fused into the compensated term: y = k x - c in one FFMA.
__device__ __forceinline__ void kahan_fma(float k, float xv, float &acc, float &cmp) {
    const float y = __fmaf_rn(k, xv, -cmp);
    const float t = __fadd_rn(acc, y);
    cmp = __fsub_rn(__fsub_rn(t, acc), y);
    acc = t;
}

// CONSEC: the R rows of a thread are consecutive points of one grid line (n % R == 0), so the
// offsets along the slow axes are shared by the R pairs of a source point:
//   2D per pair: FADD (dy), FFMA (dy^2 + dx^2 + 2^-30), MUFU.LG2, FFMA + 3 FADD (Kahan).
template <int DIM, int R, bool CONSEC>
__global__ void __launch_bounds__(kThreads)
k1_matvec_f32(const float4 *__restrict__ coord, const double *__restrict__ x, long long N,
              int tiles_per_split, int ntiles, double *__restrict__ partial) {
    __shared__ float4 sc[kThreads];
    const long long row0 = (long long)blockIdx.x * (kThreads * R);
    auto row_of = [&](int r) -> long long {
        return CONSEC ? row0 + (long long)threadIdx.x * R + r : row0 + threadIdx.x + (long long)r * kThreads;
    };
    float px[R], py[R], pz[R], acc[R], cmp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row_of(r);
        float4 c = i < N ? coord[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        px[r] = c.x; py[r] = c.y; pz[r] = c.z; acc[r] = 0.f; cmp[r] = 0.f;
    }
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    for (int t = t0; t < t1; ++t) {
        long long j = (long long)t * kThreads + threadIdx.x;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);  // padding source: x = 0 contributes nothing
        if (j < N) { c = coord[j]; c.w = (float)x[j]; }
        __syncthreads();
        sc[threadIdx.x] = c;
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < kThreads; ++jj) {
            const float4 s = sc[jj];
            if (CONSEC) {
                if (DIM == 2) {
                    const float dx = px[0] - s.x;
                    const float dxx = __fmaf_rn(dx, dx, kTiny2D);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float dy = py[r] - s.y;
                        kahan_fma(__log2f(__fmaf_rn(dy, dy, dxx)), s.w, acc[r], cmp[r]);
                    }
                } else {
                    const float dx = px[0] - s.x, dy = py[0] - s.y;
                    const float dxy = __fmaf_rn(dx, dx, dy * dy);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float dz = pz[r] - s.z;
                        kahan_fma(rsqrtf(fmaxf(__fmaf_rn(dz, dz, dxy), 1.0f)), s.w, acc[r], cmp[r]);
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float dx = px[r] - s.x, dy = py[r] - s.y;
                    float k;
                    if (DIM == 2) {
                        k = __log2f(fmaf(dx, dx, fmaf(dy, dy, kTiny2D)));
                    } else {
                        const float dz = pz[r] - s.z;
                        k = rsqrtf(fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), 1.0f));
                    }
                    kahan_fma(k, s.w, acc[r], cmp[r]);
                }
            }
        }
    }
    double *out = partial + (long long)blockIdx.y * N;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row_of(r);
        if (i < N) out[i] = (double)acc[r] - (double)cmp[r];
    }
}

// ---------------------------------------------------------------------------------------------
// K1m: FP32 SFU matvec for a batch of right-hand sides (GEMM-shaped)
// ---------------------------------------------------------------------------------------------
// A CTA owns 128 target rows and NR right-hand sides.  For every chunk of 32 source points it
// evaluates the 128 x 32 entry tile once (one SFU op per entry, spread over the CTA) into shared
// memory, stages the 32 x NR slice of x, and each thread accumulates an 8 x (NR/16) block of the
// product with FFMA -- the entry cost is amortised over NR right-hand sides.  FP32 partial sums
// are flushed every 8 chunks (256 source points) into FP64 accumulators kept in (dynamic)
// shared memory, so registers hold only the FP32 block.  Same entry conventions as K1.
constexpr int kMBM = 128, kMBK = 32;

template <int DIM, int NR>
__global__ void __launch_bounds__(kThreads)
k1m_matvec_f32(const float4 *__restrict__ coord, const double *__restrict__ x, long long ldx, int nrhs,
               long long N, int chunks_per_split, int nchunks, double *__restrict__ partial) {
    constexpr int TN = NR / 16;
    __shared__ float4 rc[kMBM];
    __shared__ float4 cc[kMBK];
    __shared__ __align__(16) float E[kMBK][kMBM];
    __shared__ __align__(16) float Xs[kMBK][NR];
    const long long row0 = (long long)blockIdx.x * kMBM;
    const int rhs0 = blockIdx.z * NR;
    const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
    if (tid < kMBM) {
        const long long i = row0 + tid;
        rc[tid] = i < N ? coord[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    extern __shared__ double dacc_s[];  // [8 * TN][kThreads]
    float acc[8][TN];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) { acc[a][b] = 0.f; dacc_s[(a * TN + b) * kThreads + tid] = 0.0; }
    const int k0 = blockIdx.y * chunks_per_split;
    const int k1 = min(k0 + chunks_per_split, nchunks);
    for (int ch = k0; ch < k1; ++ch) {
        const long long j0 = (long long)ch * kMBK;
        __syncthreads();
        if (tid < kMBK) {
            const long long j = j0 + tid;
            cc[tid] = j < N ? coord[j] : make_float4(1e6f, 1e6f, 1e6f, 0.f);
        }
        // x slice: Xs[c][r] = x[(rhs0 + r) * ldx + j0 + c]  (zero outside)
        for (int e = tid; e < kMBK * NR; e += kThreads) {
            const int r = e / kMBK, c = e % kMBK;
            const long long j = j0 + c;
            Xs[c][r] = (j < N && rhs0 + r < nrhs) ? (float)x[(long long)(rhs0 + r) * ldx + j] : 0.f;
        }
        __syncthreads();
        // entry tile E[c][m]
        for (int e = tid; e < kMBK * kMBM; e += kThreads) {
            const int m = e % kMBM, c = e / kMBM;
            const float4 a = rc[m], b = cc[c];
            const float dx = a.x - b.x, dy = a.y - b.y;
            float k;
            if (DIM == 2) {
                k = __log2f(fmaf(dx, dx, fmaf(dy, dy, kTiny2D)));
            } else {
                const float dz = a.z - b.z;
                k = rsqrtf(fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), 1.0f));
            }
            E[c][m] = k;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < kMBK; ++c) {
            const float4 e0 = *reinterpret_cast<const float4 *>(&E[c][tm * 8]);
            const float4 e1 = *reinterpret_cast<const float4 *>(&E[c][tm * 8 + 4]);
            const float ev[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
            float xv[TN];
#pragma unroll
            for (int b = 0; b < TN; ++b) xv[b] = Xs[c][tn * TN + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) acc[a][b] = fmaf(ev[a], xv[b], acc[a][b]);
        }
        if (((ch - k0) & 7) == 7 || ch == k1 - 1) {
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) {
                    dacc_s[(a * TN + b) * kThreads + tid] += (double)acc[a][b];
                    acc[a][b] = 0.f;
                }
        }
    }
    // partial layout: [split][rhs][N]
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const long long i = row0 + tm * 8 + a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < TN; ++b) {
            const int r = rhs0 + tn * TN + b;
            if (r < nrhs) partial[((long long)blockIdx.y * nrhs + r) * N + i] = dacc_s[(a * TN + b) * kThreads + tid];
        }
    }
}

// Combine for K1m: column r of y from the [split][rhs][N] partials.
__global__ void combine_multi_kernel(const double *__restrict__ partial, int nsplit, int nrhs,
                                     const double *__restrict__ x, long long ldx, double *__restrict__ y,
                                     long long ldy, long long N, int dim, double diag, double c_const,
                                     double c_sum, const double *__restrict__ xsum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= N) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += partial[((long long)k * nrhs + r) * N + i];
    const double xi = x[(long long)r * ldx + i];
    double y0;
    if (dim == 2) {
        const double self = (double)__log2f(kTiny2D) * (double)(float)xi;
        y0 = diag * xi + c_const * (xsum[r] - xi) + c_sum * (s - self);
    } else {
        y0 = diag * xi + c_sum * (s - (double)(float)xi);
    }
    y[(long long)r * ldy + i] = y0;
}

// Multi-RHS partials of exact off-diagonal entries (the Toeplitz-fed tensor-core matvec).
__global__ void combine_exact_multi_kernel(const double *__restrict__ partial, int nsplit, int nrhs,
                                           const double *__restrict__ x, long long ldx, double *__restrict__ y,
                                           long long ldy, long long N, double diag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= N) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += partial[((long long)k * nrhs + r) * N + i];
    y[(long long)r * ldy + i] = fma(diag, x[(long long)r * ldx + i], s);
}

// y_i = diag x_i + off-diagonal part from the split partials (FP64 combine).
template <typename TP>
__global__ void combine_kernel(const TP *__restrict__ partial, int nsplit, const double *__restrict__ x,
                               double *__restrict__ y, long long N, int dim, int mode, double diag,
                               double c_const, double c_sum, const double *__restrict__ xsum) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += (double)partial[(long long)k * N + i];
    const double xi = x[i];
    double y0;
    if (dim == 2) {
        // mode 0 (FP32 sums of log2(|D|^2 + 2^-30)): c_sum = c_log2, the i = j pair added
        // log2(2^-30) x_i; mode 1 (FP64 ln of max(|D|^2, 1)): c_sum = c_ln, the pair added 0
        const double self = mode == 0 ? (double)__log2f(kTiny2D) * (double)(float)xi : 0.0;
        y0 = diag * xi + c_const * (xsum[0] - xi) + c_sum * (s - self);
    } else {
        // the clamped i = j pair added rsqrt(1) * x_i (rounded as the kernel saw it)
        const double xi_k = mode == 0 ? (double)(float)xi : xi;
        y0 = diag * xi + c_sum * (s - xi_k);
    }
    y[i] = y0;
}

// ---------------------------------------------------------------------------------------------
// Kd: FP64 matvec with entries regenerated in FP64 (plain FP64 mode)
// ---------------------------------------------------------------------------------------------
template <int DIM, int R>
__global__ void __launch_bounds__(kThreads)
kd_matvec_f64(const float4 *__restrict__ coord, const double *__restrict__ x, long long N,
              int tiles_per_split, int ntiles, double *__restrict__ partial) {
    __shared__ double4 sc[kThreads];
    const long long row0 = (long long)blockIdx.x * (kThreads * R) + threadIdx.x;
    double px[R], py[R], pz[R], acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        long long i = row0 + (long long)r * kThreads;
        float4 c = i < N ? coord[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        px[r] = c.x; py[r] = c.y; pz[r] = c.z; acc[r] = 0.0;
    }
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    for (int t = t0; t < t1; ++t) {
        long long j = (long long)t * kThreads + threadIdx.x;
        double4 c = make_double4(0.0, 0.0, 0.0, 0.0);
        if (j < N) { float4 f = coord[j]; c = make_double4(f.x, f.y, f.z, x[j]); }
        __syncthreads();
        sc[threadIdx.x] = c;
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < kThreads; ++jj) {
            const double4 s = sc[jj];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double dx = px[r] - s.x, dy = py[r] - s.y;
                double r2 = DIM == 2 ? fma(dx, dx, dy * dy) : fma(dx, dx, fma(dy, dy, (pz[r] - s.z) * (pz[r] - s.z)));
                r2 = fmax(r2, 1.0);
                const double k = DIM == 2 ? log(r2) : rsqrt(r2);
                acc[r] = fma(k, s.w, acc[r]);
            }
        }
    }
    double *out = partial + (long long)blockIdx.y * N;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        long long i = row0 + (long long)r * kThreads;
        if (i < N) out[i] = acc[r];
    }
}

// ---------------------------------------------------------------------------------------------
// K2: accurate (double-float) matvec from the per-|offset| entry table
// ---------------------------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

// (sh, sl) += t * x  with t = th + tl, x = xh + xl: exact product split by FMA, TwoSum for the
// high parts (intrinsics keep the compiler from contracting the rounded product into an FMA).
__device__ __forceinline__ void df_fma(float th, float tl, float xh, float xl, float &sh, float &sl) {
    const float p = __fmul_rn(th, xh);
    float e = fmaf(th, xh, -p);
    e = fmaf(th, xl, e);
    e = fmaf(tl, xh, e);
    const float s = __fadd_rn(sh, p);
    const float bp = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// 2D: a CTA owns a 16 x 64 patch of target points and walks over 16 x 64 patches of source
// points.  Per source patch it stages x and the 31 x 127 window of table entries that the
// offsets between the two patches can reach.  Thread (t1, t2) owns the rows (t1, t2 + 16 k),
// k = 0..3.  Because the entry depends only on the offset, the entries that row k needs for
// source column c0 + 16 m are the window values at (t2 - c0) + 16 (k - m): for each (c1, c0)
// the thread loads 7 window values and 4 x values and does 16 pairs (Toeplitz register reuse).
//
// Exact accumulation in 6 FP32 operations per pair.  Each 64-term window of a row starts its
// high word at a power of two M >= 2 * (64 max|t_hi| max|x_hi| over the window), so |high| >=
// |product| holds throughout and Fast2Sum is exact: with p = fl(t_hi x_hi), s = fl(high + p),
// z = s - high (exact), the rounding errors of both the product and the sum are
// t_hi x_hi - z, which one FMA returns.  The low word collects that, t_lo x_hi (and t_hi x_lo
// when x carries a low part) and is renormalised into the high word every RENORM steps; the
// window's value (high - M) + low (exact subtraction by Sterbenz) is added to a double-float
// patch sum with TwoSum, and the patch sum to FP64 once per source patch (1024 columns).
// The diagonal is not in the table (added in FP64 afterwards), so the offsets M stay small.
// XSPLIT = false is used inside PCG, whose search directions are rounded to FP32.
constexpr int kP1 = 16, kP2 = 64;

template <bool XSPLIT, int RENORM>
__global__ void __launch_bounds__(kThreads)
k2_accurate_2d(const float2 *__restrict__ table, const double *__restrict__ x, int n,
               int patches_per_split, double *__restrict__ partial) {
    __shared__ float2 W[2 * kP1 - 1][2 * kP2];
    __shared__ float2 X[kP1][kP2];
    __shared__ float wmax[2 * kP1 - 1];
    __shared__ float xmax[kP1];
    const int np1 = (n + kP1 - 1) / kP1, np2 = (n + kP2 - 1) / kP2;
    const int I1 = (blockIdx.x / np2) * kP1, I2 = (blockIdx.x % np2) * kP2;
    const int t1 = threadIdx.x >> 4, t2 = threadIdx.x & 15;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long N = (long long)n * n;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int q0 = blockIdx.y * patches_per_split;
    const int q1 = min(q0 + patches_per_split, np1 * np2);
    for (int q = q0; q < q1; ++q) {
        const int J1 = (q / np2) * kP1, J2 = (q % np2) * kP2;
        float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};  // patch sums (double-float)
        __syncthreads();
        for (int e = threadIdx.x; e < kP1 * kP2; e += kThreads) {
            const int c1 = e / kP2, c2 = e % kP2;
            const int j1 = J1 + c1, j2 = J2 + c2;
            const double v = (j1 < n && j2 < n) ? x[(long long)j1 * n + j2] : 0.0;
            const float h = (float)v;
            X[c1][c2] = make_float2(h, XSPLIT ? (float)(v - (double)h) : 0.f);
        }
        for (int e = threadIdx.x; e < (2 * kP1 - 1) * (2 * kP2 - 1); e += kThreads) {
            const int a = e / (2 * kP2 - 1), b = e % (2 * kP2 - 1);
            const int d1 = min(abs(I1 - J1 + a - (kP1 - 1)), n - 1);
            const int d2 = min(abs(I2 - J2 + b - (kP2 - 1)), n - 1);
            W[a][b] = table[(long long)d1 * n + d2];
        }
        __syncthreads();
        // per-row maxima of |x_hi| (16 rows of 64) and |t_hi| (31 rows of 127)
        for (int r = warp; r < kP1; r += kThreads / 32) {
            float v = fmaxf(fabsf(X[r][lane].x), fabsf(X[r][lane + 32].x));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) xmax[r] = v;
        }
        for (int r = warp; r < 2 * kP1 - 1; r += kThreads / 32) {
            float v = 0.f;
            for (int b = lane; b < 2 * kP2 - 1; b += 32) v = fmaxf(v, fabsf(W[r][b].x));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) wmax[r] = v;
        }
        __syncthreads();
        for (int c1 = 0; c1 < kP1; ++c1) {
            const int a = t1 - c1 + kP1 - 1;
            const float2 *Wa = W[a];
            const float2 *Xc = X[c1];
            int ex;
            frexpf(64.f * wmax[a] * xmax[c1], &ex);
            const float M = ldexpf(1.f, ex + 1);  // >= 2 * bound, a power of two
            float sh[4] = {M, M, M, M}, sl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
            for (int c0 = 0; c0 < 16; ++c0) {
                const int base = t2 - c0 + kP2 - 1;
                float2 w[7], xv[4];
#pragma unroll
                for (int d = 0; d < 7; ++d) w[d] = Wa[base + 16 * (d - 3)];
#pragma unroll
                for (int m = 0; m < 4; ++m) xv[m] = Xc[c0 + 16 * m];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float th = w[k - m + 3].x, tl = w[k - m + 3].y, xh = xv[m].x;
                        const float pr = __fmul_rn(th, xh);
                        const float sn = __fadd_rn(sh[k], pr);
                        const float z = __fsub_rn(sn, sh[k]);
                        const float d = __fmaf_rn(th, xh, -z);
                        float lo = __fmaf_rn(tl, xh, sl[k]);
                        if (XSPLIT) lo = __fmaf_rn(th, xv[m].y, lo);
                        sl[k] = __fadd_rn(lo, d);
                        sh[k] = sn;
                    }
                }
                if ((c0 + 1) % RENORM == 0) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float t = __fadd_rn(sh[k], sl[k]);
                        sl[k] = __fsub_rn(sl[k], __fsub_rn(t, sh[k]));
                        sh[k] = t;
                    }
                }
            }
            // add the window ((high - M) exactly, + low) to the patch sum with TwoSum
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float wv = __fsub_rn(sh[k], M);
                const float sn = __fadd_rn(ah[k], wv);
                const float bp = __fsub_rn(sn, ah[k]);
                const float er = __fadd_rn(__fsub_rn(ah[k], __fsub_rn(sn, bp)), __fsub_rn(wv, bp));
                al[k] = __fadd_rn(al[k], __fadd_rn(er, sl[k]));
                ah[k] = sn;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += (double)ah[k] + (double)al[k];
    }
    const int i1 = I1 + t1;
    if (i1 < n) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i2 = I2 + t2 + 16 * k;
            if (i2 < n) partial[(long long)blockIdx.y * N + (long long)i1 * n + i2] = acc[k];
        }
    }
}

// 3D: 4 x 8 x 8 patches; the offset window is 7 x 15 x 15.  Same exact accumulation as the 2D
// kernel (power-of-two offset per 64-term window, Fast2Sum + one FMA for both rounding errors,
// renormalisation every 8 terms), one target row per thread.
__global__ void __launch_bounds__(kThreads)
k2_accurate_3d(const float2 *__restrict__ table, const double *__restrict__ x, int n,
               int patches_per_split, double *__restrict__ partial) {
    __shared__ float2 W[7][15][16];
    __shared__ float2 X[4][8][8];
    __shared__ float wmax[7];
    __shared__ float xmax[4];
    const int n1 = (n + 3) / 4, n2 = (n + 7) / 8;  // patches along dim 0 and along dims 1, 2
    const int npatch = n1 * n2 * n2;
    const int b = blockIdx.x;
    const int I1 = (b / (n2 * n2)) * 4, I2 = ((b / n2) % n2) * 8, I3 = (b % n2) * 8;
    const int r1 = threadIdx.x >> 6, r2 = (threadIdx.x >> 3) & 7, r3 = threadIdx.x & 7;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i1 = I1 + r1, i2 = I2 + r2, i3 = I3 + r3;
    const long long N = (long long)n * n * n;
    double acc = 0.0;
    const int q0 = blockIdx.y * patches_per_split;
    const int q1 = min(q0 + patches_per_split, npatch);
    for (int q = q0; q < q1; ++q) {
        const int J1 = (q / (n2 * n2)) * 4, J2 = ((q / n2) % n2) * 8, J3 = (q % n2) * 8;
        __syncthreads();
        {
            const int j1 = J1 + r1, j2 = J2 + r2, j3 = J3 + r3;
            double v = (j1 < n && j2 < n && j3 < n) ? x[((long long)j1 * n + j2) * n + j3] : 0.0;
            float h = (float)v;
            X[r1][r2][r3] = make_float2(h, (float)(v - (double)h));
        }
        for (int e = threadIdx.x; e < 7 * 15 * 15; e += kThreads) {
            const int a = e / 225, bb = (e / 15) % 15, c = e % 15;
            int d1 = min(abs(I1 - J1 + a - 3), n - 1);
            int d2 = min(abs(I2 - J2 + bb - 7), n - 1);
            int d3 = min(abs(I3 - J3 + c - 7), n - 1);
            W[a][bb][c] = table[((long long)d1 * n + d2) * n + d3];
        }
        __syncthreads();
        // maxima of |x_hi| per c1 plane (64 values) and of |t_hi| per a plane (225 values)
        if (warp < 4) {
            const float* xp = &X[warp][0][0].x;
            float v = fmaxf(fabsf(xp[2 * lane]), fabsf(xp[2 * (lane + 32)]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) xmax[warp] = v;
        } else {
            for (int a = warp - 4; a < 7; a += 4) {
                float v = 0.f;
                for (int e = lane; e < 225; e += 32) v = fmaxf(v, fabsf(W[a][e / 15][e % 15].x));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) wmax[a] = v;
            }
        }
        __syncthreads();
        float ah = 0.f, al = 0.f;
        for (int c1 = 0; c1 < 4; ++c1) {
            const int a = r1 - c1 + 3;
            int ex;
            frexpf(64.f * wmax[a] * xmax[c1], &ex);
            const float M = ldexpf(1.f, ex + 1);
            float sh = M, sl = 0.f;
#pragma unroll 2
            for (int c2 = 0; c2 < 8; ++c2) {
#pragma unroll
                for (int c3 = 0; c3 < 8; ++c3) {
                    const float2 t = W[a][r2 - c2 + 7][r3 - c3 + 7];
                    const float2 v = X[c1][c2][c3];
                    const float pr = __fmul_rn(t.x, v.x);
                    const float sn = __fadd_rn(sh, pr);
                    const float z = __fsub_rn(sn, sh);
                    const float d = __fmaf_rn(t.x, v.x, -z);
                    float lo = __fmaf_rn(t.y, v.x, sl);
                    lo = __fmaf_rn(t.x, v.y, lo);
                    sl = __fadd_rn(lo, d);
                    sh = sn;
                }
                const float tt = __fadd_rn(sh, sl);
                sl = __fsub_rn(sl, __fsub_rn(tt, sh));
                sh = tt;
            }
            const float wv = __fsub_rn(sh, M);
            const float sn = __fadd_rn(ah, wv);
            const float bp = __fsub_rn(sn, ah);
            const float er = __fadd_rn(__fsub_rn(ah, __fsub_rn(sn, bp)), __fsub_rn(wv, bp));
            al = __fadd_rn(al, __fadd_rn(er, sl));
            ah = sn;
        }
        acc += (double)ah + (double)al;
    }
    if (i1 < n && i2 < n && i3 < n) partial[(long long)blockIdx.y * N + ((long long)i1 * n + i2) * n + i3] = acc;
}

// y_i = diag x_i + the split partial sums of the off-diagonal pairs (FP64).
__global__ void sum_splits_kernel(const double *__restrict__ partial, int nsplit, const double *__restrict__ x,
                                  double diag, double *__restrict__ y, long long N) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += partial[(long long)k * N + i];
    y[i] = fma(diag, x[i], s);
}

int splits_for(long long items, long long work_units, int sm_count, int per_sm) {
    long long target = (long long)sm_count * per_sm * 8;
    long long s = (target + items - 1) / items;
    s = std::max<long long>(1, std::min<long long>(s, work_units));
    return (int)s;
}

}  // namespace

int build_problem_tables(ie_problem *p) {
    IE_TRY(prepare_tc());
    IE_TRY_CUDA(cudaMalloc(&p->d_err, sizeof(int)));
    IE_TRY_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    // dynamic shared memory of the batched matvec (set outside any stream capture)
    const int dsm64 = (int)(sizeof(double) * 8 * 4 * kThreads);
    IE_TRY_CUDA(cudaFuncSetAttribute(k1m_matvec_f32<2, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm64));
    IE_TRY_CUDA(cudaFuncSetAttribute(k1m_matvec_f32<3, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm64));
    IE_TRY_CUDA(cudaMalloc(&p->d_coord, sizeof(float4) * p->N));
    long long T = p->N;  // n^dim offsets
    IE_TRY_CUDA(cudaMalloc(&p->d_table, sizeof(float2) * T));
    IE_TRY_CUDA(cudaMalloc(&p->d_table64, sizeof(double) * T));
    coord_kernel<<<(unsigned)((p->N + 255) / 256), 256>>>(p->d_coord, p->dim, p->n, p->N);
    IE_LAUNCHED();
    table_kernel<<<(unsigned)((T + 255) / 256), 256>>>(p->d_table, p->d_table64, p->dim, p->n, T, p->diag,
                                                      p->c_const, p->c_ln, p->c_r);
    IE_LAUNCHED();
    IE_TRY(build_tc_table(p));
    IE_TRY_CUDA(cudaDeviceSynchronize());
    return IE_OK;
}

int launch_matvec_dot(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy,
                      int nrhs, int precision, double *dot_out, cudaStream_t s) {
    const long long N = p->N;
    if (precision == IE_FFT) {
        IE_TRY(launch_matvec_fft(p, x, ldx, y, ldy, nrhs, s));
        if (dot_out) IE_TRY(launch_dots(x, ldx, y, ldy, N, nrhs, dot_out, s));
        return IE_OK;
    }
    if (precision == IE_TENSOR_EXACT) {
        IE_TRY(launch_matvec_tc_exact(p, x, ldx, y, ldy, nrhs, s));
        if (dot_out) IE_TRY(launch_dots(x, ldx, y, ldy, N, nrhs, dot_out, s));
        return IE_OK;
    }
    const int ntiles = (int)((N + kThreads - 1) / kThreads);
    DevBuf xsum;
    if (p->dim == 2 && (precision == IE_MIXED || precision == IE_FP64 || (precision == IE_TENSOR && !tc_toeplitz(p)))) {
        DevBuf part;
        IE_TRY(part.alloc(sizeof(double) * iedd::kRedBlocks * nrhs, s));
        IE_TRY(xsum.alloc(sizeof(double) * nrhs, s));
        iedd::dot_partial_kernel<<<dim3(iedd::kRedBlocks, nrhs), iedd::kRedThreads, 0, s>>>(
            x, ldx, nullptr, 0, N, part.as<double>());
        IE_LAUNCHED();
        iedd::dot_final_kernel<<<nrhs, iedd::kRedBlocks, 0, s>>>(part.as<double>(), xsum.as<double>());
        IE_LAUNCHED();
    }
    if (precision == IE_TENSOR) {
        const int rt = (int)((N + tc_rows() - 1) / tc_rows());
        const int nchunks = (int)((N + tc_chunk() - 1) / tc_chunk());
        const int groups = (nrhs + tc_cols() - 1) / tc_cols();
        int S = tc_toeplitz(p) ? tc_splits_toeplitz((N + tc_block_rows() - 1) / tc_block_rows() * groups, nchunks, p->sm_count)
                               : std::min(splits_for((long long)rt * groups, nchunks, p->sm_count, 3), 16);
        const int cps = (nchunks + S - 1) / S;
        const int Se = (nchunks + cps - 1) / cps;
        DevBuf part;
        IE_TRY(part.alloc(sizeof(double) * N * nrhs * Se, s));
        IE_TRY(launch_matvec_tc(p, x, ldx, nrhs, part.as<double>(), Se, cps, nchunks, p->d_err, s));
        if (tc_toeplitz(p)) {  // exact off-diagonal entries: y = diag x + the partial sums
            combine_exact_multi_kernel<<<dim3((unsigned)((N + 255) / 256), nrhs), 256, 0, s>>>(
                part.as<double>(), Se, nrhs, x, ldx, y, ldy, N, p->diag);
        } else {
            combine_multi_kernel<<<dim3((unsigned)((N + 255) / 256), nrhs), 256, 0, s>>>(
                part.as<double>(), Se, nrhs, x, ldx, y, ldy, N, p->dim, p->diag, p->c_const,
                p->dim == 2 ? p->c_log2 : p->c_r, xsum.ptr ? xsum.as<double>() : nullptr);
        }
        IE_LAUNCHED();
        if (dot_out) IE_TRY(launch_dots(x, ldx, y, ldy, N, nrhs, dot_out, s));
        return IE_OK;
    }
    if (precision == IE_MIXED && nrhs >= 4) {
        const int NR = nrhs > 16 ? 64 : 16;
        const int rt = (int)((N + kMBM - 1) / kMBM);
        const int nchunks = (int)((N + kMBK - 1) / kMBK);
        const int groups = (nrhs + NR - 1) / NR;
        int S = splits_for((long long)rt * groups, nchunks, p->sm_count, 3);
        S = std::min(S, 16);
        const int cps = (nchunks + S - 1) / S;
        const int Se = (nchunks + cps - 1) / cps;
        DevBuf part;
        IE_TRY(part.alloc(sizeof(double) * N * nrhs * Se, s));
        const dim3 g(rt, Se, groups);
        const size_t dsm = sizeof(double) * 8 * (NR / 16) * kThreads;
        if (p->dim == 2) {
            if (NR == 64) k1m_matvec_f32<2, 64><<<g, kThreads, dsm, s>>>(p->d_coord, x, ldx, nrhs, N, cps, nchunks, part.as<double>());
            else k1m_matvec_f32<2, 16><<<g, kThreads, dsm, s>>>(p->d_coord, x, ldx, nrhs, N, cps, nchunks, part.as<double>());
        } else {
            if (NR == 64) k1m_matvec_f32<3, 64><<<g, kThreads, dsm, s>>>(p->d_coord, x, ldx, nrhs, N, cps, nchunks, part.as<double>());
            else k1m_matvec_f32<3, 16><<<g, kThreads, dsm, s>>>(p->d_coord, x, ldx, nrhs, N, cps, nchunks, part.as<double>());
        }
        IE_LAUNCHED();
        combine_multi_kernel<<<dim3((unsigned)((N + 255) / 256), nrhs), 256, 0, s>>>(
            part.as<double>(), Se, nrhs, x, ldx, y, ldy, N, p->dim, p->diag, p->c_const,
            p->dim == 2 ? p->c_log2 : p->c_r, xsum.ptr ? xsum.as<double>() : nullptr);
        IE_LAUNCHED();
        if (dot_out) IE_TRY(launch_dots(x, ldx, y, ldy, N, nrhs, dot_out, s));
        return IE_OK;
    }
    for (int k = 0; k < nrhs; ++k) {
        const double *xk = x + (long long)k * ldx;
        double *yk = y + (long long)k * ldy;
        const double *xs = xsum.ptr ? xsum.as<double>() + k : nullptr;
        if (precision == IE_MIXED) {
            constexpr int R = 4;
            const int rt = (int)((N + kThreads * R - 1) / (kThreads * R));
            const int S = splits_for(rt, ntiles, p->sm_count, 6);
            const int tps = (ntiles + S - 1) / S;
            const int Se = (ntiles + tps - 1) / tps;
            DevBuf part;
            IE_TRY(part.alloc(sizeof(double) * N * Se, s));
            const bool consec = p->n % R == 0;
            if (p->dim == 2 && consec)
                k1_matvec_f32<2, R, true><<<dim3(rt, Se), kThreads, 0, s>>>(p->d_coord, xk, N, tps, ntiles, part.as<double>());
            else if (p->dim == 2)
                k1_matvec_f32<2, R, false><<<dim3(rt, Se), kThreads, 0, s>>>(p->d_coord, xk, N, tps, ntiles, part.as<double>());
            else if (consec)
                k1_matvec_f32<3, R, true><<<dim3(rt, Se), kThreads, 0, s>>>(p->d_coord, xk, N, tps, ntiles, part.as<double>());
            else
                k1_matvec_f32<3, R, false><<<dim3(rt, Se), kThreads, 0, s>>>(p->d_coord, xk, N, tps, ntiles, part.as<double>());
            IE_LAUNCHED();
            combine_kernel<double><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
                part.as<double>(), Se, xk, yk, N, p->dim, 0, p->diag, p->c_const,
                p->dim == 2 ? p->c_log2 : p->c_r, xs);
            IE_LAUNCHED();
        } else if (precision == IE_FP64) {
            constexpr int R = 2;
            const int rt = (int)((N + kThreads * R - 1) / (kThreads * R));
            const int S = splits_for(rt, ntiles, p->sm_count, 4);
            const int tps = (ntiles + S - 1) / S;
            const int Se = (ntiles + tps - 1) / tps;
            DevBuf part;
            IE_TRY(part.alloc(sizeof(double) * N * Se, s));
            if (p->dim == 2)
                kd_matvec_f64<2, R><<<dim3(rt, Se), kThreads, 0, s>>>(p->d_coord, xk, N, tps, ntiles, part.as<double>());
            else
                kd_matvec_f64<3, R><<<dim3(rt, Se), kThreads, 0, s>>>(p->d_coord, xk, N, tps, ntiles, part.as<double>());
            IE_LAUNCHED();
            combine_kernel<double><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
                part.as<double>(), Se, xk, yk, N, p->dim, 1, p->diag, p->c_const,
                p->dim == 2 ? p->c_ln : p->c_r, xs);
            IE_LAUNCHED();
        } else {
            const int n = p->n;
            int npatch, rowpatch;
            if (p->dim == 2) {
                npatch = ((n + kP1 - 1) / kP1) * ((n + kP2 - 1) / kP2);
                rowpatch = npatch;
            } else {
                const int n1 = (n + 3) / 4, n2 = (n + 7) / 8;
                npatch = n1 * n2 * n2;
                rowpatch = npatch;
            }
            const int S = splits_for(rowpatch, npatch, p->sm_count, 4);
            const int pps = (npatch + S - 1) / S;
            const int Se = (npatch + pps - 1) / pps;
            DevBuf part;
            IE_TRY(part.alloc(sizeof(double) * N * Se, s));
            if (p->dim == 2 && precision == IE_ACCURATE)
                k2_accurate_2d<true, 1><<<dim3(rowpatch, Se), kThreads, 0, s>>>(p->d_table, xk, n, pps, part.as<double>());
            else if (p->dim == 2 && precision == IE_ACCURATE_R4)
                k2_accurate_2d<true, 4><<<dim3(rowpatch, Se), kThreads, 0, s>>>(p->d_table, xk, n, pps, part.as<double>());
            else if (p->dim == 2 && precision == IE_ACCURATE_R16)
                k2_accurate_2d<true, 16><<<dim3(rowpatch, Se), kThreads, 0, s>>>(p->d_table, xk, n, pps, part.as<double>());
            else if (p->dim == 2)
                k2_accurate_2d<false, 2><<<dim3(rowpatch, Se), kThreads, 0, s>>>(p->d_table, xk, n, pps, part.as<double>());
            else
                k2_accurate_3d<<<dim3(rowpatch, Se), kThreads, 0, s>>>(p->d_table, xk, n, pps, part.as<double>());
            IE_LAUNCHED();
            sum_splits_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(part.as<double>(), Se, xk, p->diag, yk, N);
            IE_LAUNCHED();
        }
    }
    if (dot_out) IE_TRY(launch_dots(x, ldx, y, ldy, N, nrhs, dot_out, s));
    return IE_OK;
}

int launch_matvec(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy,
                  int nrhs, int precision, cudaStream_t s) {
    return launch_matvec_dot(p, x, ldx, y, ldy, nrhs, precision, nullptr, s);
}

int launch_dots(const double *a, long long lda, const double *b, long long ldb, long long N, int nrhs,
                double *out, cudaStream_t s) {
    DevBuf part;
    IE_TRY(part.alloc(sizeof(double) * iedd::kRedBlocks * nrhs, s));
    iedd::dot_partial_kernel<<<dim3(iedd::kRedBlocks, nrhs), iedd::kRedThreads, 0, s>>>(a, lda, b, ldb, N,
                                                                                       part.as<double>());
    IE_LAUNCHED();
    iedd::dot_final_kernel<<<nrhs, iedd::kRedBlocks, 0, s>>>(part.as<double>(), out);
    IE_LAUNCHED();
    return IE_OK;
}
