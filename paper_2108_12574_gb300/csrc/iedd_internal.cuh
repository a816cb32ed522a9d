// Internal declarations shared by the translation units of libiedd (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <exception>
#include <mutex>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "iedd.h"

// ---------------------------------------------------------------------------------------------
// Errors: every entry point returns an ie_status; the message goes to a thread-local string.
// ---------------------------------------------------------------------------------------------
void ie_set_error(const std::string &msg);

#define IE_TRY_CUDA(call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            ie_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
            return e_ == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;                 \
        }                                                                                      \
    } while (0)

#define IE_CHECK_LAUNCH() IE_TRY_CUDA(cudaGetLastError())

// Kernel-launch accounting (ie_kernel_launches): every launch site is followed by IE_LAUNCHED(),
// which counts the launch unless the thread is capturing a graph (graph replays add the number
// of kernel nodes of the graph instead) and checks the launch error.
void ie_count_launches(long long k);
bool ie_capturing();
void ie_set_capturing(bool on);
#define IE_LAUNCHED()                                                                          \
    do {                                                                                       \
        if (!ie_capturing()) ie_count_launches(1);                                             \
        IE_CHECK_LAUNCH();                                                                     \
    } while (0)

#define IE_TRY(expr)                                                                           \
    do {                                                                                       \
        int s_ = (expr);                                                                       \
        if (s_ != IE_OK) return s_;                                                            \
    } while (0)

// ---------------------------------------------------------------------------------------------
// Host threads
// ---------------------------------------------------------------------------------------------
// f(b0, b1) over [0, n) in contiguous ranges, on up to hardware_concurrency host threads of at
// least `grain` items each; a range whose thread cannot be started runs on the caller.  The first
// exception a range throws is rethrown here once every thread has ended.
template <class F> void host_ranges(long long n, long long grain, const F &f) {
    const long long hc = std::max(1u, std::thread::hardware_concurrency());
    const long long nth = std::max(1LL, std::min(hc, n / std::max(grain, 1LL)));
    std::exception_ptr first;
    std::mutex mu;
    auto guarded = [&](long long b0, long long b1) {
        try {
            f(b0, b1);
        } catch (...) {
            std::lock_guard<std::mutex> g(mu);
            if (!first) first = std::current_exception();
        }
    };
    std::vector<std::thread> pool;
    long long spawned = 1;  // ranges [0, spawned) run on threads (range 0 here); the rest below
    for (long long t = 1; t < nth; ++t) {
        try {
            pool.emplace_back(guarded, n * t / nth, n * (t + 1) / nth);
            spawned = t + 1;
        } catch (const std::system_error &) {
            break;
        }
    }
    guarded(0LL, n / nth);
    for (long long t = spawned; t < nth; ++t) guarded(n * t / nth, n * (t + 1) / nth);
    for (auto &th : pool) th.join();
    if (first) std::rethrow_exception(first);
}

// Scoped device context: makes `dev` current and restores the previous device on exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------------------------
struct ie_problem {
    int dim = 0, n = 0, grid = 0, device = 0;
    long long N = 0;
    double h = 0, spacing = 0, weight = 0, diag = 0, a_shift = 0;
    // Off-diagonal entries in terms of the integer lattice offset D = i - j (r2 = |D|^2 >= 1):
    //   2D: A_ij = c_const + c_ln * ln(r2) = c_const + c_log2 * log2(r2)
    //   3D: A_ij = c_r * rsqrt(r2)
    double c_const = 0, c_ln = 0, c_log2 = 0, c_r = 0;
    float4 *d_coord = nullptr;     // integer lattice coordinates of every point (x, y, z, 0)
    float2 *d_table = nullptr;     // entry per |offset| (n^dim), split hi + lo; [0] = A_ii
    double *d_table64 = nullptr;   // same table in FP64
    float *d_stored = nullptr;     // optional dense FP32 copy of A (zero diagonal), ie_store_matrix
    int *d_err = nullptr;          // device error word of the tensor-core matvec (bounded waits)
    uint2 *d_table_tc = nullptr;   // per |offset|: the entry split into TF32 high / low words (0 at 0)
    void *d_tc_strip = nullptr;    // the batched tensor-core matvec's strip table (built on first use)
    int sm_count = 0;
    // FFT matvec (built on first use): periodic grid of L = 2^fft_lg points per axis, twiddles
    // exp(-2 pi i k / L) (k < L / 2) and the kernel's spectrum (FP64, L^d, forward-pass order)
    int fft_lg = 0;
    double2 *d_fft_tw = nullptr;
    double *d_fft_chat = nullptr;
    int fft_cfg = 4;               // autotuned launch shape of the FFT passes (see fft.cu)
    // exact tensor-core matvec (built on first use): the window table of the six BF16 digit planes
    // of the per-offset table (192 n^2 bytes) and the bits of max |t| (its power-of-two scale)
    void *d_zt_win = nullptr;
    unsigned long long *d_zt_max = nullptr;
    int zt_F = 0;                  // fraction bits of the int64 sums (units 2^-F of a level-0 product)
};

struct dd_partition_t {
    const ie_problem *prob = nullptr;
    int device = 0;
    int kind = 0, m = 0, delta = 0;
    int nblocks = 0, max_block = 0;
    long long total = 0;
    std::vector<long long> offs;   // CSR offsets, nblocks + 1
    std::vector<int> idx;          // ascending global indices per block
    // device copies
    long long *d_offs = nullptr;
    int *d_idx = nullptr;
    // inverse map for the deterministic overlap sum: for point p the positions (into idx) of
    // every occurrence, in increasing block order
    long long *d_inv_ptr = nullptr;  // N + 1
    long long *d_inv_pos = nullptr;  // total
};

struct RSFactor;  // rs.cu: recursive-skeletonization factors of the CBD subdomains

struct dd_factor_t {
    const ie_problem *prob = nullptr;
    int device = 0;
    const dd_partition_t *part = nullptr;
    int precision = 0;             // IE_FP64 or IE_MIXED
    int nblocks = 0, max_pad = 0;
    long long *d_loff = nullptr;   // offset (elements) of each padded block in the pool
    int *d_npad = nullptr;         // padded (multiple of 32) size of each block
    int *d_n = nullptr;            // true size of each block
    int *d_order = nullptr;        // schedule order: blocks by decreasing size
    void *d_pool = nullptr;        // padded row-major lower factors (float or double), or the
                                   // symmetric inverses M_i = A_i^{-1} when inverse != 0
    long long pool_elems = 0;
    int *d_info = nullptr;         // per-block first bad pivot (-1 ok)
    int inverse = 0;               // FP32 explicit inverses in d_pool (IE_MIXED, max_pad <= kInvMaxPad)
    long long *d_xoff = nullptr;   // per block: offset of its padded slice of the apply's split x
    long long xtotal = 0;          // sum of the padded block sizes
    // apply work items, one table per candidate row count kApplyRowOpts[k]: (block, first row)
    int nchunks[3] = {0, 0, 0};
    int2 *d_chunks[3] = {nullptr, nullptr, nullptr};
    // blocks padded above kApplyColFrom: single-column work items (block, first row, first
    // column, column chunk) of kApplyColRows rows x kApplyColChunk columns; maxcol = chunks of the
    // largest block
    int ncitems = 0, maxcol = 0;
    int4 *d_citems = nullptr;
    // autotuned apply configuration per class (kApplyE1, kApplyE4, kApplyF8): variant * 3 + row option
    int apply_cfg[3] = {1, 1, 1};
    // tensor-core batched apply: per block the first of its 128-row tiles (prefix sums)
    long long *d_tile_off = nullptr;
    int ntiles = 0;
    // dd_factor_rs: the RS factors (then nblocks == 0 and none of the dense fields is used)
    RSFactor *rs = nullptr;
};

// Classes of the explicit-inverse apply: double-float single column, double-float 4-column
// batches (2D), FP32 8-column batches (3D); candidate row counts per work item.
constexpr int kApplyE1 = 0, kApplyE4 = 1, kApplyF8 = 2;
constexpr int kApplyRowOpts[3] = {32, 64, 128};
// The column-chunked apply for large blocks (CBD colour blocks): x staged per 4096 columns
constexpr int kApplyColFrom = 8192, kApplyColChunk = 4096, kApplyColRows = 64;
// 3D batches of at least this many right-hand sides take the tensor-core apply (launch_apply_tc)
constexpr int kApplyTensorFrom = 32;

// Largest padded block applied through its explicit inverse: the apply stages the block's split x
// (8 bytes per point and right-hand side) in one CTA's shared memory.
constexpr int kInvMaxPad = 25600;
// Largest block of an FP64 factor (one CTA per block factors it on CUDA cores).
constexpr int kFp64MaxBlock = 8192;


// ---------------------------------------------------------------------------------------------
// Device vector helpers: host / device pointer detection and staging
// ---------------------------------------------------------------------------------------------
bool ie_is_device_ptr(const void *p);

// RAII stream-ordered device buffer.
struct DevBuf {
    void *ptr = nullptr;
    cudaStream_t s = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    int alloc(size_t b, cudaStream_t st);
    ~DevBuf();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// ---------------------------------------------------------------------------------------------
// Kernel launchers (matvec.cu, factor.cu, apply.cu, pcg.cu)
// ---------------------------------------------------------------------------------------------
// Internal matvec mode: the accurate (double-float) sum for an x whose entries are exactly
// representable in FP32 (PCG rounds its search directions so), which saves one FFMA per pair.
constexpr int IE_ACCURATE_X32 = 4;
// Internal matvec modes of the exact kernel for the PCG inner product q = A p: the low word is
// renormalised every 4 (mode 7) or 16 (mode 8) source steps instead of every step.  The error
// stays many orders below what slows PCG; the true residual always uses IE_ACCURATE.
constexpr int IE_ACCURATE_R4 = 7;
constexpr int IE_ACCURATE_R16 = 8;

// y = A x for device FP64 x (leading dimension ldx) and y (ldy), nrhs columns.
// precision: IE_FP64, IE_MIXED, IE_ACCURATE or IE_ACCURATE_X32.
int launch_matvec(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy,
                  int nrhs, int precision, cudaStream_t s);
// As launch_matvec, and, if dot_out != nullptr, dot_out[k] = x_k^T y_k (FP64, deterministic).
int launch_matvec_dot(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy,
                      int nrhs, int precision, double *dot_out, cudaStream_t s);
int build_problem_tables(ie_problem *p);
int launch_matvec_tc(const ie_problem *p, const double *x, long long ldx, int nrhs, double *partial, int S, int cps,
                     int nchunks, int *d_err, cudaStream_t s);
int prepare_tc();
int build_tc_table(ie_problem *p);
bool tc_toeplitz(const ie_problem *p);  // the tensor-core matvec reads its tiles from the strip table
int prepare_tc_strip(const ie_problem *p);  // builds the strip table (synchronizes; not under capture)
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (nullptr if absent)
void *tensor_map_encode_fn();
int tc_splits_toeplitz(long long tiles, int nchunks, int sms);  // source splits of that kernel
int tc_chunk();
int tc_rows();
int tc_block_rows();  // target rows per CTA of the strip-fed kernel (tc_toeplitz)
int tc_cols();
int launch_matvec_stored(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy, int nrhs,
                         cudaStream_t s);

// FFT matvec (fft.cu): prepare_fft builds the plan once per problem (synchronizes; not inside a
// stream capture); launch_matvec_fft then computes y = A x for nrhs columns.
int prepare_fft(const ie_problem *p);
// 1 if the FFT matvec handles this problem (else 0 and, if why != nullptr, the reason)
int fft_supported(const ie_problem *p, std::string *why);
int launch_matvec_fft(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy, int nrhs,
                      cudaStream_t s);
// Exact tensor-core 2D matvec (tc_exact.cu): prepare_tc_exact builds the digit table once per
// problem (synchronizes; not inside a stream capture).
bool tc_exact_supported(const ie_problem *p);
int prepare_tc_exact(const ie_problem *p);
int launch_matvec_tc_exact(const ie_problem *p, const double *x, long long ldx, double *y, long long ldy, int nrhs,
                           cudaStream_t s);

int launch_factor(dd_factor_t *f, cudaStream_t s);
// apply.cu: time the candidate apply configurations of an explicit-inverse factor (outside any
// capture; cached per partition shape) and record the fastest in f->apply_cfg.
int tune_apply(dd_factor_t *f, cudaStream_t s);

// Autotuning switch and process-wide cache of measured choices (api.cu).
bool autotune_enabled();
bool tune_get(const std::string &key, int *choice);
void tune_put(const std::string &key, int choice, const std::string &detail);
// tc_factor.cu: Cholesky and explicit inverse of the gathered FP32 blocks in f->d_pool (M_i
// replaces the block), bulk on the tensor cores; synchronizes.  f->d_info must hold -1 per block.
int launch_factor_tc(dd_factor_t *f, const std::vector<int> &npad, const std::vector<long long> &loff,
                     cudaStream_t s);
// tc_factor.cu: z_i = M_i (R_i r) for a batch of right-hand sides as GEMM tasks of the persistent
// kernel on the tensor cores (FP32-accurate products, FP32 sums); xh, xe as apply_split<false>
// writes them; results into zbuf [rhs][sum n_i]
int launch_apply_tc(const dd_factor_t *f, const float *xh, const int *xe, int nrhs, double *zbuf, cudaStream_t s);
int prepare_apply(const dd_factor_t *f);
// rs.cu: z = T^{-1} r through the RS factors of f->rs; rs_destroy frees them.
int launch_apply_rs(const dd_factor_t *f, const double *r, long long ldr, double *z, long long ldz, int nrhs,
                    cudaStream_t s);
void rs_destroy(RSFactor *rs);
// z = T^{-1} r for device FP64 r (ldr) and z (ldz).
int launch_apply(const dd_factor_t *f, const double *r, long long ldr, double *z, long long ldz,
                 int nrhs, cudaStream_t s);

// Deterministic FP64 column dot products: out[k] = sum_i a[k*lda+i] * b[k*ldb+i] (device).
int launch_dots(const double *a, long long lda, const double *b, long long ldb, long long N,
                int nrhs, double *out, cudaStream_t s);
