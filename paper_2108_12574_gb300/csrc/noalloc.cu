// ie_matvec_noalloc: the FP32 SFU matvec (the kernel ie_matvec runs for IE_MIXED) for callers
// that cannot allocate device memory -- code running where cudaMalloc is forbidden or unsafe,
// such as inside a custom allocator, a memory-capped plug-in, or a process whose allocations
// are all made up front.  The paper has no counterpart; this is a deployment variant.
//
// Everything the call needs besides the caller's x and y lives in one file-scope device array,
// g_noalloc_scratch (IE_NOALLOC_SCRATCH_BYTES = 32 MiB, 256-byte aligned).  The array is part of
// this file's device code: it is reserved on a device when that code is loaded there, which
// CUDA does lazily by default (at the first launch or symbol lookup), and it stays until the
// process exits.  Host code never uses the array's name as an address: the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device current) and caches
// it for the life of the process.  Point coordinates are derived from the grid index inside the
// kernel, so no problem handle (and no allocation) is needed either.
//
// Calls share the array: a call overwrites every word it later reads (each split's partial sum
// for every row, every reduction slot), so nothing has to start at zero, and calls whose GPU
// work overlaps (different streams, or different host threads without ordering) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "iedd_internal.cuh"
#include "noalloc_args.h"

namespace {

constexpr long long kScratchDoubles = IE_NOALLOC_SCRATCH_BYTES / 8;  // 4 Mi doubles
constexpr int kReserve = 1024;     // reduction partials and the column sum
constexpr int kRedBlocksNA = 128;
constexpr int kThreadsNA = 256;
constexpr int kRowsNA = 4;
constexpr float kTinyNA = 0x1p-30f;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

double *g_scratch_ptr[256] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_current_device(double **out) {
    int dev = 0;
    IE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) { ie_set_error("ie_matvec_noalloc: device ordinal out of range"); return IE_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        IE_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return IE_OK;
}

// The device that owns p's memory: its ordinal for device memory, the current device for
// managed memory (reachable from it), -1 for host or unregistered memory.
int owning_device(const void *p, int current) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear: an unknown pointer is host memory
        return -1;
    }
    if (a.type == cudaMemoryTypeManaged) return current;
    return a.type == cudaMemoryTypeDevice ? a.device : -1;
}

__device__ __forceinline__ float4 lattice_point(long long i, int dim, int n) {
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (dim == 2) {
        c.x = (float)(i / n);
        c.y = (float)(i % n);
    } else {
        c.z = (float)(i % n);
        c.y = (float)((i / n) % n);
        c.x = (float)(i / ((long long)n * n));
    }
    return c;
}

__global__ void __launch_bounds__(kThreadsNA)
colsum_partial(const double *__restrict__ x, long long N, double *__restrict__ part) {
    __shared__ double sh[32];
    const long long chunk = (N + kRedBlocksNA - 1) / kRedBlocksNA;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < N ? lo + chunk : N;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += x[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

__global__ void colsum_final(const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < kRedBlocksNA; ++b) s += part[b];
        out[0] = s;
    }
}

// The K1 pair loop (FP32 SFU entry, Kahan-compensated sum with the product fused) with the
// coordinates computed from the grid index.
template <int DIM>
__global__ void __launch_bounds__(kThreadsNA)
k1na_matvec_f32(const double *__restrict__ x, int n, long long N, int tiles_per_split, int ntiles,
                double *__restrict__ partial) {
    __shared__ float4 sc[kThreadsNA];
    const long long row0 = (long long)blockIdx.x * (kThreadsNA * kRowsNA) + threadIdx.x;
    float px[kRowsNA], py[kRowsNA], pz[kRowsNA], acc[kRowsNA], cmp[kRowsNA];
#pragma unroll
    for (int r = 0; r < kRowsNA; ++r) {
        const long long i = row0 + (long long)r * kThreadsNA;
        const float4 c = lattice_point(i < N ? i : 0, DIM, n);
        px[r] = c.x; py[r] = c.y; pz[r] = c.z; acc[r] = 0.f; cmp[r] = 0.f;
    }
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    for (int t = t0; t < t1; ++t) {
        const long long j = (long long)t * kThreadsNA + threadIdx.x;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < N) { c = lattice_point(j, DIM, n); c.w = (float)x[j]; }
        __syncthreads();
        sc[threadIdx.x] = c;
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < kThreadsNA; ++jj) {
            const float4 s = sc[jj];
#pragma unroll
            for (int r = 0; r < kRowsNA; ++r) {
                const float dx = px[r] - s.x, dy = py[r] - s.y;
                float k;
                if (DIM == 2) {
                    k = __log2f(fmaf(dx, dx, fmaf(dy, dy, kTinyNA)));
                } else {
                    const float dz = pz[r] - s.z;
                    k = rsqrtf(fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), 1.0f));
                }
                const float y = __fmaf_rn(k, s.w, -cmp[r]);
                const float tt = __fadd_rn(acc[r], y);
                cmp[r] = __fsub_rn(__fsub_rn(tt, acc[r]), y);
                acc[r] = tt;
            }
        }
    }
    double *out = partial + (long long)blockIdx.y * N;
#pragma unroll
    for (int r = 0; r < kRowsNA; ++r) {
        const long long i = row0 + (long long)r * kThreadsNA;
        if (i < N) out[i] = (double)acc[r] - (double)cmp[r];
    }
}

__global__ void combine_na(const double *__restrict__ partial, int nsplit, const double *__restrict__ x,
                           double *__restrict__ y, long long N, int dim, double diag, double c_const,
                           double c_sum, const double *__restrict__ xsum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += partial[(long long)k * N + i];
    const double xi = x[i];
    if (dim == 2) {
        const double self = (double)__log2f(kTinyNA) * (double)(float)xi;
        y[i] = diag * xi + c_const * (xsum[0] - xi) + c_sum * (s - self);
    } else {
        y[i] = diag * xi + c_sum * (s - (double)(float)xi);
    }
}

}  // namespace

extern "C" int ie_matvec_noalloc(int dim, int n, double a_shift, int grid, const double *x, double *y,
                                 void *stream) {
    int dev = 0;
    IE_TRY_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NoallocArgs args;
    args.dim = dim; args.n = n; args.grid = grid; args.a_shift = a_shift; args.x = x; args.y = y;
    args.dev_current = dev;
    args.x_device = x ? owning_device(x, dev) : -1;
    args.y_device = y ? owning_device(y, dev) : -1;
    args.stream_device = dev;
    if (s != nullptr) IE_TRY_CUDA(cudaStreamGetDevice(s, &args.stream_device));
    long long N = 0;
    const char *why = "";
    if (noalloc_check_args(args, IE_NOALLOC_MAX_N, &N, &why) != 0) {
        std::string msg = std::string("ie_matvec_noalloc: ") + why;
        if (dim >= 2 && dim <= 3 && n >= 2 && std::string(why).find("exceeds") != std::string::npos)
            msg += " (" + std::to_string((long long)IE_NOALLOC_MAX_N) + " points)";
        ie_set_error(msg);
        return IE_ERR_ARG;
    }
    double *scratch = nullptr;
    IE_TRY(scratch_for_current_device(&scratch));

    // constants of the collocation matrix (Sec. 2.1), as ie_discretize computes them
    const double pi = 3.14159265358979323846;
    const double h = 1.0 / n;
    const double spacing = grid == IE_GRID_TEXT ? h : 1.0 / (n - 1);
    const double w = dim == 2 ? h * h : h * h * h;
    const double diag = (dim == 2 ? -(h * h / (4.0 * pi)) * (2.0 * std::log(h / 2.0) + std::log(2.0) - 3.0 + pi / 2.0)
                                  : (h * h / (2.0 * pi)) * (3.0 * std::log(1.0 + std::sqrt(3.0)) - 1.5 * std::log(2.0) - pi / 4.0)) +
                        a_shift;
    const double c_const = -w * std::log(spacing) / (2.0 * pi);
    const double c_log2 = -w / (4.0 * pi) * std::log(2.0);
    const double c_r = w / (4.0 * pi * spacing);

    double *red = scratch;                  // kRedBlocksNA partial sums
    double *xsum = scratch + kRedBlocksNA;  // 1 value
    double *partial = scratch + kReserve;   // [split][N]
    const int ntiles = (int)((N + kThreadsNA - 1) / kThreadsNA);
    const int rt = (int)((N + kThreadsNA * kRowsNA - 1) / (kThreadsNA * kRowsNA));
    int sms = 0;
    IE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long want = ((long long)sms * 6 * 8 + rt - 1) / rt;
    const long long cap = (kScratchDoubles - kReserve) / N;
    long long S = want < 1 ? 1 : want;
    if (S > cap) S = cap;
    if (S > ntiles) S = ntiles;
    const int tps = (int)((ntiles + S - 1) / S);
    const int Se = (ntiles + tps - 1) / tps;

    if (dim == 2) {
        colsum_partial<<<kRedBlocksNA, kThreadsNA, 0, s>>>(x, N, red);
        IE_LAUNCHED();
        colsum_final<<<1, 32, 0, s>>>(red, xsum);
        IE_LAUNCHED();
        k1na_matvec_f32<2><<<dim3(rt, Se), kThreadsNA, 0, s>>>(x, n, N, tps, ntiles, partial);
        IE_LAUNCHED();
    } else {
        k1na_matvec_f32<3><<<dim3(rt, Se), kThreadsNA, 0, s>>>(x, n, N, tps, ntiles, partial);
        IE_LAUNCHED();
    }
    combine_na<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(partial, Se, x, y, N, dim, diag, c_const,
                                                          dim == 2 ? c_log2 : c_r, xsum);
    IE_LAUNCHED();
    return IE_OK;
}
