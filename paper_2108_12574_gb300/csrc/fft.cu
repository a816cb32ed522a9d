// FFT matvec (the paper's matvec, Sec. 6): on the uniform grid A_ij depends only on the integer
// offset i - j, so A is Toeplitz in every coordinate (block-Toeplitz with Toeplitz blocks in 2D,
// three levels in 3D).  Embedded in a circulant on the periodic grid of L^d points
// (L = 2^lg >= 2n - 1), A x is the first n^d entries of IFFT(FFT(c) . FFT(x padded)), with
// c(k) = A(offset d(k)), d_a(k_a) = k_a for k_a < n and k_a - L for k_a > L - n, 0 elsewhere.
// Everything is FP64.
//
// Layout: a complex L^d grid per pair of right-hand sides (the first as real part, the second as
// imaginary part: c is real and even, so its spectrum is real and the two never mix).  Every
// transform runs in place in shared memory, a line (one axis, all other coordinates fixed) at a
// time, with no bit reversal anywhere: the forward passes are decimation in frequency (natural
// order in, bit-reversed order out along the axis), the spectrum of c is produced by the same
// forward passes (so it sits in the same permuted layout, scaled by L^-d), and the inverse passes
// are decimation in time (bit-reversed in, natural out).
//
// KF fft_axis<MODE>  CTA = `cb` lines along one axis: load (positions >= nin are zero and not
//                    read), MODE 0 forward / MODE 1 forward x spectrum x inverse / MODE 2 inverse,
//                    store (MODE 1, 2: natural positions < nout only).  Lines whose input is zero
//                    are not launched: the forward passes only visit lines whose other coordinates
//                    are < n (or whose other axes were transformed already), the inverse passes only
//                    lines whose other coordinates are outputs.
// KP fft_pack / fft_unpack  the n^d block of two FP64 columns into / out of the complex grid.
// Per matvec: pack, d - 1 forward passes, one MODE 1 pass, d - 1 inverse passes, unpack.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "iedd_internal.cuh"

namespace {

constexpr int kFftThreads = 256;
constexpr size_t kFftSmemCeiling = 200 * 1024;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
    return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 w) {  // a * conj(w)
    return make_double2(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}

// Decimation in frequency over `lines` lines of length L = 2^lg at z + c * ls; W[k] =
// exp(-2 pi i k / L), k < L / 2.  Stage s has span h = L / 2^(s+1); the butterfly at offset o
// within its block of 2h takes the twiddle W[o 2^s] (1 in the last stage).
__device__ void fft_dif(double2 *z, int ls, int lines, int lg, const double2 *W) {
    const int half = 1 << (lg - 1);
    const int nb = lines << (lg - 1);
    for (int s = 0; s < lg; ++s) {
        const int h = half >> s;
        for (int b = threadIdx.x; b < nb; b += kFftThreads) {
            const int c = b >> (lg - 1), j = b & (half - 1);
            const int off = j & (h - 1);
            const int a = ((j - off) << 1) + off;
            double2 *zl = z + c * ls;
            const double2 u = zl[a], v = zl[a + h];
            zl[a] = cadd(u, v);
            zl[a + h] = h == 1 ? csub(u, v) : cmul(csub(u, v), W[off << s]);
        }
        __syncthreads();
    }
}

// Decimation in time, the inverse of fft_dif up to the factor L: spans h = 1, 2, ..., L / 2 with
// the conjugate twiddles.
__device__ void fft_dit(double2 *z, int ls, int lines, int lg, const double2 *W) {
    const int half = 1 << (lg - 1);
    const int nb = lines << (lg - 1);
    for (int s = lg - 1; s >= 0; --s) {
        const int h = half >> s;
        for (int b = threadIdx.x; b < nb; b += kFftThreads) {
            const int c = b >> (lg - 1), j = b & (half - 1);
            const int off = j & (h - 1);
            const int a = ((j - off) << 1) + off;
            double2 *zl = z + c * ls;
            const double2 u = zl[a];
            const double2 t = h == 1 ? zl[a + h] : cmulc(zl[a + h], W[off << s]);
            zl[a] = cadd(u, t);
            zl[a + h] = csub(u, t);
        }
        __syncthreads();
    }
}

// One pass along `axis` of the complex L^d grids (one per pair: blockIdx.y).  Lines are numbered
// over the other axes o1 < o2 (o1 absent in 2D: ext1 = 1) with extents ext1 x ext2; the CTA takes
// lines blockIdx.x * cb .. + cb - 1.  Shared memory: cb lines of stride L + 1, then W.
template <int MODE>
__global__ void __launch_bounds__(kFftThreads)
fft_axis(double2 *__restrict__ Z, long long zstride, const double *__restrict__ chat, const double2 *__restrict__ Wg,
         int d, int axis, int lg, int cb, int ext1, int ext2, int nin, int nout) {
    extern __shared__ double2 fsm[];
    const int L = 1 << lg, ls = L + 1;
    double2 *z = fsm;
    double2 *W = fsm + (size_t)cb * ls;
    for (int k = threadIdx.x; k < L / 2; k += kFftThreads) W[k] = Wg[k];
    // the other axes and the element stride along `axis` (last axis contiguous)
    int o1 = -1, o2 = -1;
    for (int a = 0; a < d; ++a)
        if (a != axis) { if (o2 < 0 && o1 < 0 && d == 3) o1 = a; else o2 = a; }
    // element stride of axis a: L^(d - 1 - a)
    auto stride_of = [&](int a) { return a < 0 ? 0LL : (long long)1 << (lg * (d - 1 - a)); };
    const long long es = stride_of(axis), s1 = stride_of(o1), s2 = stride_of(o2);
    const long long lines = (long long)ext1 * ext2;
    const long long l0 = (long long)blockIdx.x * cb;
    double2 *Zp = Z + (long long)blockIdx.y * zstride;
    auto line_base = [&](long long l) { return (l / ext2) * s1 + (l % ext2) * s2; };
    const bool contiguous = axis == d - 1;
    const int total = cb * L;
    // load: positions >= nin are zero; lines beyond the last are zero (computed, not stored)
    for (int e = threadIdx.x; e < total; e += kFftThreads) {
        const int c = contiguous ? e / L : e % cb, k = contiguous ? e % L : e / cb;
        const long long l = l0 + c;
        double2 v = make_double2(0.0, 0.0);
        if (k < nin && l < lines) v = Zp[line_base(l) + k * es];
        z[c * ls + k] = v;
    }
    __syncthreads();
    if (MODE == 0 || MODE == 1) fft_dif(z, ls, cb, lg, W);
    if (MODE == 1) {
        for (int e = threadIdx.x; e < total; e += kFftThreads) {
            const int c = contiguous ? e / L : e % cb, k = contiguous ? e % L : e / cb;
            const long long l = l0 + c;
            if (l < lines) {
                const double s = chat[line_base(l) + k * es];
                double2 &v = z[c * ls + k];
                v.x *= s;
                v.y *= s;
            }
        }
        __syncthreads();
    }
    if (MODE == 1 || MODE == 2) fft_dit(z, ls, cb, lg, W);
    const int kmax = MODE == 0 ? L : nout;
    for (int e = threadIdx.x; e < total; e += kFftThreads) {
        const int c = contiguous ? e / L : e % cb, k = contiguous ? e % L : e / cb;
        const long long l = l0 + c;
        if (k < kmax && l < lines) Zp[line_base(l) + k * es] = z[c * ls + k];
    }
}

// the n^d block of columns 2p (real part) and 2p + 1 (imaginary part, zero if absent)
__global__ void fft_pack(const double *__restrict__ x, long long ldx, int nrhs, int d, int n, int lg,
                         long long zstride, double2 *__restrict__ Z) {
    const long long N = d == 2 ? (long long)n * n : (long long)n * n * n;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (i >= N) return;
    const int ka = 2 * p, kb = 2 * p + 1;
    const double a = x[(long long)ka * ldx + i];
    const double b = kb < nrhs ? x[(long long)kb * ldx + i] : 0.0;
    long long t = i, zi = 0, mul = 1;
    for (int q = 0; q < d; ++q) { zi += (t % n) * mul; t /= n; mul <<= lg; }
    Z[(long long)p * zstride + zi] = make_double2(a, b);
}

__global__ void fft_unpack(const double2 *__restrict__ Z, long long zstride, int nrhs, int d, int n, int lg,
                           double *__restrict__ y, long long ldy) {
    const long long N = d == 2 ? (long long)n * n : (long long)n * n * n;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (i >= N) return;
    long long t = i, zi = 0, mul = 1;
    for (int q = 0; q < d; ++q) { zi += (t % n) * mul; t /= n; mul <<= lg; }
    const double2 v = Z[(long long)p * zstride + zi];
    y[(long long)(2 * p) * ldy + i] = v.x;
    if (2 * p + 1 < nrhs) y[(long long)(2 * p + 1) * ldy + i] = v.y;
}

// c on the periodic grid (real part), from the per-|offset| FP64 table (diagonal at offset 0)
__global__ void fft_cext(const double *__restrict__ t64, int d, int n, int lg, double2 *__restrict__ Z) {
    const int L = 1 << lg;
    const long long T = (long long)1 << (lg * d);
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T) return;
    long long t = k, idx = 0, mul = 1;
    bool inside = true;
    for (int q = 0; q < d; ++q) {  // last axis first
        const int ka = (int)(t & (L - 1));
        t >>= lg;
        int off;
        if (ka < n) off = ka;
        else if (ka > L - n) off = L - ka;
        else { inside = false; off = 0; }
        idx += (long long)off * mul;
        mul *= n;
    }
    Z[k] = make_double2(inside ? t64[idx] : 0.0, 0.0);
}

__global__ void fft_chat(const double2 *__restrict__ Z, double inv, long long T, double *__restrict__ chat) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < T) chat[k] = Z[k].x * inv;
}

// Launch shape cfg = 3 a + b: enough CTAs to fill the GPU (1 << a) times where the line count
// allows, and strided passes keep at least (2 << b) adjacent lines per CTA (global accesses in
// runs of 32 (2 << b) bytes).  The default is cfg 4; prepare_fft times all nine.
int lines_per_cta(int lg, long long lines, int sms, bool strided, int cfg) {
    const size_t per_line = sizeof(double2) * (size_t)((1 << lg) + 1);
    const size_t tw = sizeof(double2) * (size_t)(1 << lg) / 2;
    const long long cap = std::min<long long>((long long)((kFftSmemCeiling - tw) / per_line), 64);
    const int a = cfg / 3, b = cfg % 3;
    long long cb = std::min<long long>(cap, std::max<long long>(1, lines / ((long long)(1 << a) * sms)));
    if (strided) cb = std::max<long long>(cb, std::min<long long>(cap, 2 << b));
    return (int)std::max<long long>(cb, 1);
}

// One pass; ext1, ext2: extents of the other axes (o1 < o2; ext1 = 1 in 2D).
template <int MODE>
int fft_pass(const ie_problem *p, double2 *Z, long long zstride, int npairs, int axis, int ext1, int ext2, int nin,
             int nout, cudaStream_t s) {
    const int lg = p->fft_lg, L = 1 << lg;
    const long long lines = (long long)ext1 * ext2;
    const int cb = lines_per_cta(lg, lines, p->sm_count, axis != p->dim - 1, p->fft_cfg);
    const size_t smem = sizeof(double2) * ((size_t)cb * (L + 1) + (size_t)L / 2);
    const long long ctas = (lines + cb - 1) / cb;
    if (ctas > 0x7fffffffLL || npairs > 65535) {
        ie_set_error("ie_matvec: FFT grid too large");
        return IE_ERR_ARG;
    }
    fft_axis<MODE><<<dim3((unsigned)ctas, npairs), kFftThreads, smem, s>>>(Z, zstride, p->d_fft_chat, p->d_fft_tw, p->dim,
                                                                          axis, lg, cb, ext1, ext2, nin, nout);
    IE_LAUNCHED();
    return IE_OK;
}

}  // namespace

int fft_supported(const ie_problem *p, std::string *why) {
    // a line must fit one CTA's shared memory: L <= 8192
    if (2 * p->n - 1 > 8192) {
        if (why) *why = "the FFT matvec supports n <= 4096";
        return 0;
    }
    return 1;
}

// Times the nine launch shapes on one matvec of a zero vector (the transforms are
// data-independent) and keeps the fastest; cached per (dim, n).
int tune_fft(ie_problem *p) {
    p->fft_cfg = 4;
    if (!autotune_enabled()) return IE_OK;
    const std::string key = "fft/d" + std::to_string(p->dim) + "/n" + std::to_string(p->n);
    int best = 4;
    if (tune_get(key, &best)) { p->fft_cfg = best; return IE_OK; }
    double *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = IE_OK;
    if (cudaMalloc(&x, sizeof(double) * p->N) != cudaSuccess || cudaMalloc(&y, sizeof(double) * p->N) != cudaSuccess ||
        cudaMemset(x, 0, sizeof(double) * p->N) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        st = IE_ERR_CUDA;
    }
    float best_ms = 0.f;
    std::string detail;
    for (int cand = 0; cand < 9 && st == IE_OK; ++cand) {
        p->fft_cfg = cand;
        st = launch_matvec_fft(p, x, p->N, y, p->N, 1, nullptr);
        cudaEventRecord(e0, nullptr);
        for (int rep = 0; rep < 3 && st == IE_OK; ++rep) st = launch_matvec_fft(p, x, p->N, y, p->N, 1, nullptr);
        cudaEventRecord(e1, nullptr);
        if (st == IE_OK && cudaEventSynchronize(e1) != cudaSuccess) st = IE_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        detail += (cand ? " " : "") + std::to_string(cand) + ":" + std::to_string((int)(ms * 1000.f)) + "us";
        if (cand == 0 || ms < best_ms) { best_ms = ms; best = cand; }
    }
    cudaFree(x);
    cudaFree(y);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != IE_OK) { p->fft_cfg = 4; return st; }
    p->fft_cfg = best;
    tune_put(key, best, detail);
    return IE_OK;
}

int prepare_fft(const ie_problem *cp) {
    ie_problem *p = const_cast<ie_problem *>(cp);
    if (p->d_fft_chat) return IE_OK;
    std::string why;
    if (!fft_supported(p, &why)) { ie_set_error("ie_matvec: " + why); return IE_ERR_ARG; }
    int lg = 1;
    while ((1 << lg) < 2 * p->n - 1) ++lg;
    const int L = 1 << lg;
    const long long T = (long long)1 << (lg * p->dim);
    IE_TRY_CUDA(cudaFuncSetAttribute(fft_axis<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(fft_axis<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemCeiling));
    IE_TRY_CUDA(cudaFuncSetAttribute(fft_axis<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemCeiling));
    // twiddles exp(-2 pi i k / L) from the host's FP64 cos / sin of the reduced angle
    std::vector<double2> tw((size_t)L / 2);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < L / 2; ++k) {
        const double ang = 2.0 * pi * (double)k / (double)L;
        tw[(size_t)k] = make_double2(std::cos(ang), -std::sin(ang));
    }
    double2 *d_tw = nullptr, *Z = nullptr;
    double *chat = nullptr;
    auto fail = [&](int st) {
        cudaFree(d_tw);
        cudaFree(Z);
        cudaFree(chat);
        return st;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&d_tw, sizeof(double2) * tw.size())) != cudaSuccess ||
        (e = cudaMalloc(&chat, sizeof(double) * T)) != cudaSuccess ||
        (e = cudaMalloc(&Z, sizeof(double2) * T)) != cudaSuccess) {
        ie_set_error(std::string("ie_matvec: ") + cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA);
    }
    if ((e = cudaMemcpy(d_tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
        ie_set_error(std::string("ie_matvec: ") + cudaGetErrorString(e));
        return fail(IE_ERR_CUDA);
    }
    p->fft_lg = lg;
    p->d_fft_tw = d_tw;
    p->d_fft_chat = chat;  // read by no pass below (MODE 0 only)
    cudaStream_t s = nullptr;
    fft_cext<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(p->d_table64, p->dim, p->n, lg, Z);
    int st = cudaGetLastError() == cudaSuccess ? IE_OK : IE_ERR_CUDA;
    // forward transform along every axis, all lines
    for (int axis = p->dim - 1; axis >= 0 && st == IE_OK; --axis) {
        const int e1 = p->dim == 3 ? L : 1;
        st = fft_pass<0>(p, Z, T, 1, axis, e1, L, L, L, s);
    }
    if (st == IE_OK) {
        fft_chat<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(Z, 1.0 / (double)T, T, chat);
        if (cudaGetLastError() != cudaSuccess) st = IE_ERR_CUDA;
    }
    if (st == IE_OK && cudaDeviceSynchronize() != cudaSuccess) st = IE_ERR_CUDA;
    cudaFree(Z);
    if (st == IE_OK) st = tune_fft(p);
    if (st != IE_OK) {
        ie_set_error("ie_matvec: building the FFT of the kernel failed");
        p->d_fft_tw = nullptr;
        p->d_fft_chat = nullptr;
        p->fft_lg = 0;
        cudaFree(d_tw);
        cudaFree(chat);
    }
    return st;
}

// y = A x for nrhs FP64 columns through the FFT (prepare_fft must have run).
int launch_matvec_fft(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy, int nrhs,
                      cudaStream_t s) {
    if (!p->d_fft_chat) { ie_set_error("ie_matvec: FFT plan missing"); return IE_ERR_ARG; }
    const int d = p->dim, n = p->n, lg = p->fft_lg, L = 1 << lg;
    const long long T = (long long)1 << (lg * d);
    const int npairs = (nrhs + 1) / 2;
    DevBuf zb;
    IE_TRY(zb.alloc(sizeof(double2) * (size_t)T * npairs, s));
    double2 *Z = zb.as<double2>();
    dim3 gp((unsigned)((p->N + 255) / 256), npairs);
    fft_pack<<<gp, 256, 0, s>>>(x, ldx, nrhs, d, n, lg, T, Z);
    IE_LAUNCHED();
    if (d == 2) {
        IE_TRY(fft_pass<0>(p, Z, T, npairs, 1, 1, n, n, L, s));  // rows j0 < n
        IE_TRY(fft_pass<1>(p, Z, T, npairs, 0, 1, L, n, n, s));  // all columns, keep rows < n
        IE_TRY(fft_pass<2>(p, Z, T, npairs, 1, 1, n, L, n, s));  // rows < n, keep columns < n
    } else {
        IE_TRY(fft_pass<0>(p, Z, T, npairs, 2, n, n, n, L, s));  // lines (j0, j1) < n
        IE_TRY(fft_pass<0>(p, Z, T, npairs, 1, n, L, n, L, s));  // lines (j0 < n, k2)
        IE_TRY(fft_pass<1>(p, Z, T, npairs, 0, L, L, n, n, s));  // lines (k1, k2)
        IE_TRY(fft_pass<2>(p, Z, T, npairs, 1, n, L, L, n, s));  // lines (i0 < n, k2), keep i1 < n
        IE_TRY(fft_pass<2>(p, Z, T, npairs, 2, n, n, L, n, s));  // lines (i0, i1) < n, keep i2 < n
    }
    fft_unpack<<<gp, 256, 0, s>>>(Z, T, nrhs, d, n, lg, y, ldy);
    IE_LAUNCHED();
    return IE_OK;
}
