// C-ABI entry points of libiedd: handles, argument checks, host/device staging, and the
// host-side domain decomposition (Sec. 2.2-2.3).  The compute steps live in matvec.cu,
// factor.cu, apply.cu and pcg.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <cstdlib>
#include <mutex>
#include <map>
#include <memory>
#include <vector>

#include "iedd_internal.cuh"

#include <atomic>

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;

void ie_count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
bool ie_capturing() { return g_capturing; }
void ie_set_capturing(bool on) { g_capturing = on; }

extern "C" long long ie_kernel_launches(int reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

void ie_set_error(const std::string &msg) { g_last_error = msg; }

extern "C" const char *ie_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *ie_version(void) { return "iedd-gb300 0.1 (sm_103a)"; }

bool ie_is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear: an unknown pointer is host memory
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The library's scratch and factor pools come from the device's default memory pool
// (cudaMallocAsync).  A pool returns freed memory to the driver at every synchronization unless
// its release threshold says otherwise, and the solver frees and re-allocates the same large
// buffers every step; so the first problem on a device raises this process's threshold to keep
// up to 16 GB cached (a larger threshold set by the caller is left as it is).
void keep_pool_cached(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return;
    done.push_back(device);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return;
    uint64_t cur = 0, want = 16ULL << 30;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < want)
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
}

int DevBuf::alloc(size_t b, cudaStream_t st) {
    s = st;
    bytes = b;
    if (b == 0) return IE_OK;
    IE_TRY_CUDA(cudaMallocAsync(&ptr, b, st));
    return IE_OK;
}

DevBuf::~DevBuf() {
    if (ptr) cudaFreeAsync(ptr, s);
}

// ---------------------------------------------------------------------------------------------
// Autotuning: measured choices of launch shapes, cached per problem shape for the process
// ---------------------------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, std::string>> g_tune;
int g_tune_on = -1;  // -1: not read yet (IEDD_AUTOTUNE=0 disables)
bool tune_on_locked() {
    if (g_tune_on < 0) {
        const char *e = std::getenv("IEDD_AUTOTUNE");
        g_tune_on = (e && e[0] == '0') ? 0 : 1;
    }
    return g_tune_on == 1;
}
}  // namespace

bool autotune_enabled() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return tune_on_locked();
}

bool tune_get(const std::string &key, int *choice) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *choice = it->second.first;
    return true;
}

void tune_put(const std::string &key, int choice, const std::string &detail) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {choice, detail};
}

extern "C" int ie_autotune(int mode) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int prev = tune_on_locked() ? 1 : 0;
    if (mode == 0 || mode == 1) g_tune_on = mode;
    if (mode == 2) g_tune.clear();
    return prev;
}

extern "C" const char *ie_autotune_report(void) {
    static thread_local std::string out;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    out.clear();
    for (const auto &kv : g_tune)
        out += kv.first + " -> " + std::to_string(kv.second.first) + " (" + kv.second.second + ")\n";
    return out.c_str();
}

// ---------------------------------------------------------------------------------------------
// Problem (Sec. 2.1)
// ---------------------------------------------------------------------------------------------
static double self_cell_integral(int dim, double h) {
    const double pi = 3.14159265358979323846;
    if (dim == 2) {
        // -(h^2/(4 pi)) (2 ln(h/2) + int_{[0,1]^2} ln(s^2+t^2)),  the integral = ln 2 - 3 + pi/2
        return -(h * h / (4.0 * pi)) * (2.0 * std::log(h / 2.0) + std::log(2.0) - 3.0 + pi / 2.0);
    }
    // (h^2/(2 pi)) int_{[0,1]^3} 1/|x|,  the integral = 3 ln(1+sqrt 3) - 1.5 ln 2 - pi/4
    return (h * h / (2.0 * pi)) *
           (3.0 * std::log(1.0 + std::sqrt(3.0)) - 1.5 * std::log(2.0) - pi / 4.0);
}

extern "C" int ie_discretize(int dim, int n, double a_shift, int grid, int device, ie_problem **out) {
    if (!out) { ie_set_error("ie_discretize: out is NULL"); return IE_ERR_ARG; }
    *out = nullptr;
    if (dim != 2 && dim != 3) { ie_set_error("ie_discretize: dim must be 2 or 3"); return IE_ERR_ARG; }
    if (n < 2) { ie_set_error("ie_discretize: n must be >= 2"); return IE_ERR_ARG; }
    long long N = 1;
    for (int d = 0; d < dim; ++d) N *= n;
    if (N > (1LL << 26)) { ie_set_error("ie_discretize: N = n^dim exceeds 2^26"); return IE_ERR_ARG; }
    if (!std::isfinite(a_shift)) {
        ie_set_error("ie_discretize: a_shift must be finite"); return IE_ERR_ARG;
    }
    if (grid != IE_GRID_TEXT && grid != IE_GRID_TABLE) {
        ie_set_error("ie_discretize: unknown grid convention"); return IE_ERR_ARG;
    }
    int ndev = 0;
    IE_TRY_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) { ie_set_error("ie_discretize: bad device ordinal"); return IE_ERR_ARG; }
    DeviceGuard g(device);

    keep_pool_cached(device);
    ie_problem *p = new (std::nothrow) ie_problem();
    if (!p) { ie_set_error("ie_discretize: out of host memory"); return IE_ERR_OOM; }
    const double pi = 3.14159265358979323846;
    p->dim = dim; p->n = n; p->N = N; p->grid = grid; p->device = device; p->a_shift = a_shift;
    p->h = 1.0 / n;
    p->spacing = grid == IE_GRID_TEXT ? p->h : 1.0 / (n - 1);
    p->weight = dim == 2 ? p->h * p->h : p->h * p->h * p->h;
    p->diag = self_cell_integral(dim, p->h) + a_shift;
    // A_ij = w K(s D): 2D  -w/(2 pi) (ln s + ln(r2)/2);  3D  w / (4 pi s sqrt(r2))
    p->c_const = -p->weight * std::log(p->spacing) / (2.0 * pi);
    p->c_ln = -p->weight / (4.0 * pi);
    p->c_log2 = p->c_ln * std::log(2.0);
    p->c_r = p->weight / (4.0 * pi * p->spacing);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete p; ie_set_error("cudaGetDeviceProperties failed"); return IE_ERR_CUDA; }
    p->sm_count = prop.multiProcessorCount;
    int st = build_problem_tables(p);
    if (st != IE_OK) { ie_destroy(p); return st; }
    *out = p;
    return IE_OK;
}

extern "C" int ie_problem_info(const ie_problem *p, int *dim, int *n, long long *N, double *h, double *diag) {
    if (!p) { ie_set_error("ie_problem_info: NULL problem"); return IE_ERR_ARG; }
    if (dim) *dim = p->dim;
    if (n) *n = p->n;
    if (N) *N = p->N;
    if (h) *h = p->h;
    if (diag) *diag = p->diag;
    return IE_OK;
}

extern "C" void ie_destroy(ie_problem *p) {
    if (!p) return;
    DeviceGuard g(p->device);
    cudaFree(p->d_coord);
    cudaFree(p->d_table);
    cudaFree(p->d_table64);
    cudaFree(p->d_stored);
    cudaFree(p->d_err);
    cudaFree(p->d_table_tc);
    cudaFree(p->d_tc_strip);
    cudaFree(p->d_fft_tw);
    cudaFree(p->d_fft_chat);
    cudaFree(p->d_zt_win);
    cudaFree(p->d_zt_max);
    delete p;
}

// ---------------------------------------------------------------------------------------------
// Staging of host vectors
// ---------------------------------------------------------------------------------------------
namespace {
struct Staged {
    const double *dev = nullptr;   // device view of the vector
    long long ld = 0;
    DevBuf buf;
};

int stage_in(const double *x, long long N, int nrhs, long long ld, bool copy, cudaStream_t s,
             Staged &st) {
    if (ie_is_device_ptr(x)) { st.dev = x; st.ld = ld; return IE_OK; }
    IE_TRY(st.buf.alloc(sizeof(double) * N * nrhs, s));
    if (copy)
        IE_TRY_CUDA(cudaMemcpy2DAsync(st.buf.ptr, sizeof(double) * N, x, sizeof(double) * ld,
                                      sizeof(double) * N, nrhs, cudaMemcpyHostToDevice, s));
    st.dev = st.buf.as<double>();
    st.ld = N;
    return IE_OK;
}

int stage_out(double *y, const Staged &st, long long N, int nrhs, long long ld, cudaStream_t s) {
    if (st.buf.ptr == nullptr) return IE_OK;
    IE_TRY_CUDA(cudaMemcpy2DAsync(y, sizeof(double) * ld, st.buf.ptr, sizeof(double) * N,
                                  sizeof(double) * N, nrhs, cudaMemcpyDeviceToHost, s));
    return IE_OK;
}

int check_vec_args(const char *who, const ie_problem *p, const void *a, const void *b, int nrhs,
                   long long ld) {
    if (!p) { ie_set_error(std::string(who) + ": NULL problem"); return IE_ERR_ARG; }
    if (!a || !b) { ie_set_error(std::string(who) + ": NULL vector"); return IE_ERR_ARG; }
    if (nrhs < 1) { ie_set_error(std::string(who) + ": nrhs must be >= 1"); return IE_ERR_ARG; }
    if (ld < p->N) { ie_set_error(std::string(who) + ": ld must be >= N"); return IE_ERR_ARG; }
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    size_t span = sizeof(double) * (size_t)(ld * (nrhs - 1) + p->N);
    if (pa < pb + span && pb < pa + span) {
        ie_set_error(std::string(who) + ": input and output overlap"); return IE_ERR_ARG;
    }
    return IE_OK;
}
}  // namespace

extern "C" int ie_matvec(const ie_problem *p, const double *x, double *y, int nrhs, long long ld,
                         int precision, void *stream) {
    IE_TRY(check_vec_args("ie_matvec", p, x, y, nrhs, ld));
    if (precision != IE_FP64 && precision != IE_MIXED && precision != IE_ACCURATE && precision != IE_STORED &&
        precision != IE_TENSOR && precision != IE_FFT && precision != IE_TENSOR_EXACT) {
        ie_set_error("ie_matvec: unknown precision"); return IE_ERR_ARG;
    }
    if (precision == IE_TENSOR_EXACT && !tc_exact_supported(p)) {
        ie_set_error("ie_matvec: IE_TENSOR_EXACT needs a 2D grid with n a multiple of 128 and n <= 4096");
        return IE_ERR_ARG;
    }
    if (precision == IE_STORED && !p->d_stored) {
        ie_set_error("ie_matvec: IE_STORED needs ie_store_matrix first"); return IE_ERR_ARG;
    }
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == IE_FFT && !p->d_fft_chat) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        IE_TRY_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            ie_set_error("ie_matvec: the first IE_FFT call on a problem builds its FFT plan and must not be captured");
            return IE_ERR_ARG;
        }
        IE_TRY(prepare_fft(p));
    }
    if (precision == IE_TENSOR_EXACT && !p->d_zt_win) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        IE_TRY_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            ie_set_error("ie_matvec: the first IE_TENSOR_EXACT call on a problem builds its digit window table and must not "
                         "be captured");
            return IE_ERR_ARG;
        }
        IE_TRY(prepare_tc_exact(p));
    }
    if (precision == IE_TENSOR || precision == IE_TENSOR_EXACT)
        IE_TRY_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), s));
    Staged sx, sy;
    IE_TRY(stage_in(x, p->N, nrhs, ld, true, s, sx));
    IE_TRY(stage_in(y, p->N, nrhs, ld, false, s, sy));
    if (precision == IE_STORED)
        IE_TRY(launch_matvec_stored(p, sx.dev, sx.ld, const_cast<double *>(sy.dev), sy.ld, nrhs, s));
    else
        IE_TRY(launch_matvec(p, sx.dev, sx.ld, const_cast<double *>(sy.dev), sy.ld, nrhs, precision, s));
    IE_TRY(stage_out(y, sy, p->N, nrhs, ld, s));
    if (precision == IE_TENSOR || precision == IE_TENSOR_EXACT) {
        // the tensor-core kernels report a CTA that gave up waiting for its MMAs
        int err = 0;
        IE_TRY_CUDA(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        IE_TRY_CUDA(cudaStreamSynchronize(s));
        if (err) { ie_set_error("ie_matvec: tensor-core matvec timed out waiting for its MMAs"); return IE_ERR_TIMEOUT; }
    }
    if (sx.buf.ptr || sy.buf.ptr) IE_TRY_CUDA(cudaStreamSynchronize(s));
    return IE_OK;
}

// ---------------------------------------------------------------------------------------------
// Domain decomposition (Sec. 2.2-2.3; Eqs. e:dd, e:first, e:cbd; Table t:dd)
// ---------------------------------------------------------------------------------------------
static const int kMaxBlock = kInvMaxPad;  // the largest block the mixed factor and apply take

static int partition_impl(const ie_problem *p, int m, int delta, int kind, dd_partition_t **out);

extern "C" int dd_partition(const ie_problem *p, int m, int delta, int kind, dd_partition_t **out) {
    // host containers and threads may throw; nothing may cross the C ABI
    try {
        return partition_impl(p, m, delta, kind, out);
    } catch (const std::bad_alloc &) {
        ie_set_error("dd_partition: out of host memory");
        return IE_ERR_OOM;
    } catch (const std::exception &e) {
        ie_set_error(std::string("dd_partition: ") + e.what());
        return IE_ERR_ARG;
    }
}

static int partition_impl(const ie_problem *p, int m, int delta, int kind, dd_partition_t **out) {
    if (!out) { ie_set_error("dd_partition: out is NULL"); return IE_ERR_ARG; }
    *out = nullptr;
    if (!p) { ie_set_error("dd_partition: NULL problem"); return IE_ERR_ARG; }
    if (m < 1 || p->n % m != 0) { ie_set_error("dd_partition: n must be a positive multiple of m"); return IE_ERR_ARG; }
    if (delta < 0) { ie_set_error("dd_partition: delta must be >= 0"); return IE_ERR_ARG; }
    if (kind != DD_JACOBI && kind != DD_SCHWARZ && kind != DD_CBD) {
        ie_set_error("dd_partition: unknown kind"); return IE_ERR_ARG;
    }
    const int dim = p->dim, n = p->n, w = n / m;
    const int ext = kind == DD_JACOBI ? 0 : std::min(delta, n);
    long long M = 1;
    for (int d = 0; d < dim; ++d) M *= m;

    dd_partition_t *s = new (std::nothrow) dd_partition_t();
    if (!s) { ie_set_error("dd_partition: out of host memory"); return IE_ERR_OOM; }
    s->prob = p; s->device = p->device; s->kind = kind; s->m = m; s->delta = ext;
    // inverse map (point -> positions of its occurrences, in increasing block order)
    std::unique_ptr<long long[]> inv_ptr, inv_pos;
    if (kind == DD_CBD) {
        // A colour's boxes are the product of one parity per axis, so their union is the product of
        // the per-axis unions of the extended intervals [k w - ext, (k + 1) w + ext), k of that
        // parity: its points in grid order (ascending, no duplicates).  rank[d][par][x] is the
        // index of coordinate x in axis d's union for that parity, or -1.
        std::vector<int> axis[3][2], rank[3][2];
        for (int d = 0; d < 3; ++d)
            for (int par = 0; par < 2; ++par) {
                if (d >= dim) {  // a missing axis: the single coordinate 0
                    axis[d][par].assign(1, 0);
                    rank[d][par].assign(1, 0);
                    continue;
                }
                std::vector<char> in((size_t)n, 0);
                for (int k = par; k < m; k += 2)
                    for (int x = std::max(k * w - ext, 0); x < std::min((k + 1) * w + ext, n); ++x) in[(size_t)x] = 1;
                rank[d][par].assign((size_t)n, -1);
                for (int x = 0; x < n; ++x)
                    if (in[(size_t)x]) {
                        rank[d][par][(size_t)x] = (int)axis[d][par].size();
                        axis[d][par].push_back(x);
                    }
            }
        // the colours with points, in colour order: one block each
        struct Colour {
            int par[3];
            long long len[3], off;
        };
        std::vector<Colour> cols;
        long long total = 0;
        for (int c = 0; c < (1 << dim); ++c) {
            Colour k{};
            long long size = 1;
            for (int d = 0; d < 3; ++d) {
                k.par[d] = d < dim ? (c >> (dim - 1 - d)) & 1 : 0;
                k.len[d] = (long long)axis[d][k.par[d]].size();
                size *= k.len[d];
            }
            if (size == 0) continue;
            k.off = total;
            total += size;
            cols.push_back(k);
        }
        s->nblocks = (int)cols.size();
        s->offs.assign(cols.size() + 1, 0);
        for (size_t b = 0; b < cols.size(); ++b) {
            s->offs[b + 1] = cols[b].off + cols[b].len[0] * cols[b].len[1] * cols[b].len[2];
            s->max_block = std::max(s->max_block, (int)(s->offs[b + 1] - s->offs[b]));
        }
        s->total = total;
        // the blocks' points, one (block, axis-0 coordinate) line per item, on host threads
        s->idx.resize((size_t)total);
        std::vector<std::pair<int, int>> lines;
        for (size_t b = 0; b < cols.size(); ++b)
            for (int r0 = 0; r0 < (int)cols[b].len[0]; ++r0) lines.emplace_back((int)b, r0);
        const long long per_line = std::max<long long>(total / std::max<long long>((long long)lines.size(), 1), 1);
        host_ranges((long long)lines.size(), std::max<long long>(1, (1 << 16) / per_line), [&](long long l0, long long l1) {
            for (long long l = l0; l < l1; ++l) {
                const Colour &k = cols[(size_t)lines[(size_t)l].first];
                const int r0 = lines[(size_t)l].second, i = axis[0][k.par[0]][(size_t)r0];
                long long q = k.off + (long long)r0 * k.len[1] * k.len[2];
                for (int j : axis[1][k.par[1]])
                    for (int x : axis[2][k.par[2]]) s->idx[(size_t)q++] = dim == 2 ? i * n + j : (i * n + j) * n + x;
            }
        });
        // the inverse map in closed form: point (x_0, .., x_{dim-1}) sits in every colour whose
        // unions hold all its coordinates, at the colour's offset plus its row-major rank there;
        // counted per chunk of points, scanned, then filled chunk by chunk on host threads
        const long long N = p->N;
        inv_ptr.reset(new long long[(size_t)N + 1]);
        inv_pos.reset(new long long[(size_t)std::max<long long>(total, 1)]);
        long long *ip = inv_ptr.get(), *pp = inv_pos.get();
        auto occurrences = [&](long long i, long long *out) {  // writes the positions, returns their count
            int x[3] = {0, 0, 0};
            for (int d = dim - 1; d >= 0; --d) { x[d] = (int)(i % n); i /= n; }
            int cnt = 0;
            for (const Colour &k : cols) {
                long long pos = 0;
                bool inside = true;
                for (int d = 0; d < 3 && inside; ++d) {
                    const int r = rank[d][k.par[d]][(size_t)x[d]];
                    inside = r >= 0;
                    pos = pos * k.len[d] + r;
                }
                if (!inside) continue;
                if (out) out[cnt] = k.off + pos;
                ++cnt;
            }
            return cnt;
        };
        const long long nchunk = std::max<long long>(1, std::min<long long>(N >> 14, 1024));  // >= 16K points each
        std::vector<long long> csum((size_t)nchunk + 1, 0);
        host_ranges(nchunk, 1, [&](long long c0, long long c1) {
            for (long long c = c0; c < c1; ++c) {
                long long acc = 0;
                for (long long i = N * c / nchunk; i < N * (c + 1) / nchunk; ++i) acc += occurrences(i, nullptr);
                csum[(size_t)c + 1] = acc;
            }
        });
        for (long long c = 0; c < nchunk; ++c) csum[(size_t)c + 1] += csum[(size_t)c];
        ip[0] = 0;
        host_ranges(nchunk, 1, [&](long long c0, long long c1) {
            for (long long c = c0; c < c1; ++c) {
                long long acc = csum[(size_t)c];
                for (long long i = N * c / nchunk; i < N * (c + 1) / nchunk; ++i) {
                    acc += occurrences(i, pp + acc);
                    ip[i + 1] = acc;
                }
            }
        });
    } else {
        // every extended box, enumerated row-major so its indices come out ascending
        s->nblocks = (int)M;
        s->offs.assign((size_t)M + 1, 0);
        for (long long b = 0; b < M; ++b) {
            int k[3] = {0, 0, 0};
            long long t = b;
            for (int d = dim - 1; d >= 0; --d) { k[d] = (int)(t % m); t /= m; }
            int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
            for (int d = 0; d < dim; ++d) {
                lo[d] = std::max(k[d] * w - ext, 0);
                hi[d] = std::min((k[d] + 1) * w + ext, n);
            }
            for (int i = lo[0]; i < hi[0]; ++i)
                for (int j = lo[1]; j < hi[1]; ++j)
                    for (int l = lo[2]; l < hi[2]; ++l) s->idx.push_back(dim == 2 ? i * n + j : (i * n + j) * n + l);
            s->offs[(size_t)b + 1] = (long long)s->idx.size();
            s->max_block = std::max(s->max_block, (int)(s->offs[(size_t)b + 1] - s->offs[(size_t)b]));
        }
        s->total = s->offs.back();
        if (s->max_block > kMaxBlock) {
            delete s;
            ie_set_error("dd_partition: a subdomain has more than " + std::to_string(kMaxBlock) + " points");
            return IE_ERR_ARG;
        }
        inv_ptr.reset(new long long[(size_t)p->N + 1]());
        inv_pos.reset(new long long[(size_t)std::max<long long>(s->total, 1)]);
        long long *ip = inv_ptr.get(), *pp = inv_pos.get();
        for (long long q = 0; q < s->total; ++q) ip[(size_t)s->idx[(size_t)q] + 1]++;
        for (long long i = 0; i < p->N; ++i) ip[i + 1] += ip[i];
        std::vector<long long> fill(ip, ip + p->N);
        for (long long q = 0; q < s->total; ++q) pp[fill[(size_t)s->idx[(size_t)q]]++] = q;
    }

    DeviceGuard g(p->device);
    auto fail = [&](cudaError_t e) {
        ie_set_error(std::string("dd_partition: ") + cudaGetErrorString(e));
        dd_partition_destroy(s);
        return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&s->d_offs, sizeof(long long) * s->offs.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&s->d_idx, sizeof(int) * std::max<long long>(s->total, 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&s->d_inv_ptr, sizeof(long long) * ((size_t)p->N + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&s->d_inv_pos, sizeof(long long) * std::max<long long>(s->total, 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(s->d_offs, s->offs.data(), sizeof(long long) * s->offs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(s->d_idx, s->idx.data(), sizeof(int) * s->total, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(s->d_inv_ptr, inv_ptr.get(), sizeof(long long) * ((size_t)p->N + 1), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(s->d_inv_pos, inv_pos.get(), sizeof(long long) * s->total, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    *out = s;
    return IE_OK;
}

extern "C" int dd_partition_info(const dd_partition_t *s, int *nblocks, long long *total, int *max_block) {
    if (!s) { ie_set_error("dd_partition_info: NULL partition"); return IE_ERR_ARG; }
    if (nblocks) *nblocks = s->nblocks;
    if (total) *total = s->total;
    if (max_block) *max_block = s->max_block;
    return IE_OK;
}

extern "C" int dd_partition_export(const dd_partition_t *s, long long *offsets, int *index) {
    if (!s) { ie_set_error("dd_partition_export: NULL partition"); return IE_ERR_ARG; }
    if (offsets) std::memcpy(offsets, s->offs.data(), sizeof(long long) * s->offs.size());
    if (index) std::memcpy(index, s->idx.data(), sizeof(int) * s->idx.size());
    return IE_OK;
}

extern "C" void dd_partition_destroy(dd_partition_t *s) {
    if (!s) return;
    DeviceGuard g(s->device);
    cudaFree(s->d_offs);
    cudaFree(s->d_idx);
    cudaFree(s->d_inv_ptr);
    cudaFree(s->d_inv_pos);
    delete s;
}

// ---------------------------------------------------------------------------------------------
// Factor and apply (Sec. 3, Eqs. e:ai, e:ad; exact Cholesky subdomain solver of Sec. 4.3)
// ---------------------------------------------------------------------------------------------
extern "C" int dd_factor(const ie_problem *p, const dd_partition_t *s, int precision, dd_factor_t **out,
                         int *info, void *stream) {
    if (!out) { ie_set_error("dd_factor: out is NULL"); return IE_ERR_ARG; }
    *out = nullptr;
    if (info) *info = -1;
    if (!p || !s) { ie_set_error("dd_factor: NULL problem or partition"); return IE_ERR_ARG; }
    if (s->prob != p) { ie_set_error("dd_factor: partition belongs to another problem"); return IE_ERR_ARG; }
    if (precision != IE_FP64 && precision != IE_MIXED) { ie_set_error("dd_factor: unknown precision"); return IE_ERR_ARG; }
    if (s->max_block > kMaxBlock) {
        ie_set_error("dd_factor: a subdomain has more than " + std::to_string(kMaxBlock) +
                     " points (dense factors); large CBD subdomains take dd_factor_rs");
        return IE_ERR_ARG;
    }
    if (precision == IE_FP64 && s->max_block > kFp64MaxBlock) {
        ie_set_error("dd_factor: IE_FP64 factors take blocks of at most " + std::to_string(kFp64MaxBlock) +
                     " points (one CTA per block); use IE_MIXED");
        return IE_ERR_ARG;
    }
    DeviceGuard g(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dd_factor_t *f = new (std::nothrow) dd_factor_t();
    if (!f) { ie_set_error("dd_factor: out of host memory"); return IE_ERR_OOM; }
    f->prob = p; f->device = p->device; f->part = s; f->precision = precision; f->nblocks = s->nblocks;

    std::vector<long long> loff((size_t)s->nblocks + 1, 0);
    std::vector<int> npad((size_t)s->nblocks), nb((size_t)s->nblocks), order((size_t)s->nblocks);
    for (int i = 0; i < s->nblocks; ++i) {
        nb[(size_t)i] = (int)(s->offs[(size_t)i + 1] - s->offs[(size_t)i]);
        npad[(size_t)i] = (nb[(size_t)i] + 31) / 32 * 32;
        if (npad[(size_t)i] == 0) npad[(size_t)i] = 32;
        f->max_pad = std::max(f->max_pad, npad[(size_t)i]);
        loff[(size_t)i + 1] = loff[(size_t)i] + (long long)npad[(size_t)i] * npad[(size_t)i];
        order[(size_t)i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nb[(size_t)a] > nb[(size_t)b]; });
    f->pool_elems = loff.back();
    size_t esz = precision == IE_FP64 ? sizeof(double) : sizeof(float);
    auto fail = [&](cudaError_t e) {
        ie_set_error(std::string("dd_factor: ") + cudaGetErrorString(e));
        dd_factor_destroy(f);
        return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&f->d_loff, sizeof(long long) * loff.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&f->d_npad, sizeof(int) * npad.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&f->d_n, sizeof(int) * nb.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&f->d_order, sizeof(int) * order.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&f->d_info, sizeof(int) * nb.size())) != cudaSuccess) return fail(e);
    // the pool of blocks comes from the cached memory pool (freed after a device synchronize)
    if ((e = cudaMallocAsync(&f->d_pool, esz * (size_t)f->pool_elems, st)) != cudaSuccess) return fail(e);
    f->inverse = precision == IE_MIXED && f->max_pad <= kInvMaxPad;
    if (f->inverse) {
        std::vector<long long> xoff((size_t)s->nblocks + 1, 0);
        for (int i = 0; i < s->nblocks; ++i) xoff[(size_t)i + 1] = xoff[(size_t)i] + npad[(size_t)i];
        f->xtotal = xoff.back();
        if ((e = cudaMalloc(&f->d_xoff, sizeof(long long) * xoff.size())) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(f->d_xoff, xoff.data(), sizeof(long long) * xoff.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        // the tensor-core batched apply: per block the first of its 128-row tiles
        std::vector<long long> toff((size_t)s->nblocks + 1, 0);
        for (int i = 0; i < s->nblocks; ++i) toff[(size_t)i + 1] = toff[(size_t)i] + (nb[(size_t)i] + 127) / 128;
        f->ntiles = (int)toff.back();
        if ((e = cudaMalloc(&f->d_tile_off, sizeof(long long) * toff.size())) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(f->d_tile_off, toff.data(), sizeof(long long) * toff.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        for (int k = 0; k < 3; ++k) {  // work items of kApplyRowOpts[k] rows, largest blocks first
            std::vector<int2> chunks;
            for (int i : order)
                for (int r0 = 0; r0 < nb[(size_t)i]; r0 += kApplyRowOpts[k]) chunks.push_back(make_int2(i, r0));
            f->nchunks[k] = (int)chunks.size();
            if ((e = cudaMalloc(&f->d_chunks[k], sizeof(int2) * std::max<size_t>(chunks.size(), 1))) != cudaSuccess) return fail(e);
            if (!chunks.empty() && (e = cudaMemcpy(f->d_chunks[k], chunks.data(), sizeof(int2) * chunks.size(),
                                                   cudaMemcpyHostToDevice)) != cudaSuccess)
                return fail(e);
        }
        if (f->max_pad > kApplyColFrom) {  // large blocks: column-chunked single-column work items
            std::vector<int4> items;
            for (int i : order)
                for (int r0 = 0; r0 < nb[(size_t)i]; r0 += kApplyColRows)
                    for (int c0 = 0; c0 < npad[(size_t)i]; c0 += kApplyColChunk)
                        items.push_back(make_int4(i, r0, c0, c0 / kApplyColChunk));
            f->ncitems = (int)items.size();
            f->maxcol = (f->max_pad + kApplyColChunk - 1) / kApplyColChunk;
            if ((e = cudaMalloc(&f->d_citems, sizeof(int4) * items.size())) != cudaSuccess) return fail(e);
            if ((e = cudaMemcpy(f->d_citems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return fail(e);
        }
    }
    if ((e = cudaMemcpy(f->d_loff, loff.data(), sizeof(long long) * loff.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(f->d_npad, npad.data(), sizeof(int) * npad.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(f->d_n, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(f->d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);

    if ((e = cudaMemsetAsync(f->d_info, 0xFF, sizeof(int) * nb.size(), st)) != cudaSuccess) return fail(e);
    int stl = launch_factor(f, st);
    if (stl == IE_OK && f->inverse) stl = launch_factor_tc(f, npad, loff, st);
    if (stl == IE_OK) stl = prepare_apply(f);
    if (stl == IE_OK && f->inverse) {
        // the tuning applies need the factor finished and every block SPD
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        std::vector<int> hinfo0((size_t)s->nblocks);
        if ((e = cudaMemcpy(hinfo0.data(), f->d_info, sizeof(int) * hinfo0.size(), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e);
        bool spd = true;
        for (int v : hinfo0) spd = spd && v < 0;
        if (spd) stl = tune_apply(f, st);
    }
    if (stl != IE_OK) { dd_factor_destroy(f); return stl; }
    std::vector<int> hinfo((size_t)s->nblocks);
    if ((e = cudaMemcpyAsync(hinfo.data(), f->d_info, sizeof(int) * hinfo.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    *out = f;
    for (int i = 0; i < s->nblocks; ++i) {
        if (hinfo[(size_t)i] >= 0) {
            if (info) *info = i;
            ie_set_error("dd_factor: block " + std::to_string(i) + " is not SPD (pivot " +
                         std::to_string(hinfo[(size_t)i]) + ")");
            return IE_ERR_NOT_SPD;
        }
    }
    return IE_OK;
}

extern "C" void dd_factor_destroy(dd_factor_t *f) {
    if (!f) return;
    DeviceGuard g(f->device);
    cudaFree(f->d_loff);
    cudaFree(f->d_npad);
    cudaFree(f->d_tile_off);
    cudaFree(f->d_n);
    cudaFree(f->d_order);
    cudaFree(f->d_info);
    if (f->d_pool) {  // from cudaMallocAsync: every use on any stream has finished after the synchronize
        cudaDeviceSynchronize();
        cudaFreeAsync(f->d_pool, nullptr);
    }
    cudaFree(f->d_xoff);
    for (int k = 0; k < 3; ++k) cudaFree(f->d_chunks[k]);
    cudaFree(f->d_citems);
    if (f->rs) {  // its buffers may still be read by work in flight on any stream
        cudaDeviceSynchronize();
        rs_destroy(f->rs);
    }
    delete f;
}

extern "C" int dd_apply(const dd_factor_t *f, const double *r, double *z, int nrhs, long long ld, void *stream) {
    if (!f) { ie_set_error("dd_apply: NULL factor"); return IE_ERR_ARG; }
    IE_TRY(check_vec_args("dd_apply", f->prob, r, z, nrhs, ld));
    const ie_problem *p = f->prob;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staged sr, sz;
    IE_TRY(stage_in(r, p->N, nrhs, ld, true, s, sr));
    IE_TRY(stage_in(z, p->N, nrhs, ld, false, s, sz));
    IE_TRY(launch_apply(f, sr.dev, sr.ld, const_cast<double *>(sz.dev), sz.ld, nrhs, s));
    IE_TRY(stage_out(z, sz, p->N, nrhs, ld, s));
    if (sr.buf.ptr || sz.buf.ptr) IE_TRY_CUDA(cudaStreamSynchronize(s));
    return IE_OK;
}
