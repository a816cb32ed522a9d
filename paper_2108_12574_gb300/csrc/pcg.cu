// pcg_solve: preconditioned conjugate gradient on A u = f with T^{-1} of Eq. e:ad (Sec. 6 solves
// with PCG).  nrhs independent recurrences share every kernel launch; each column has its own
// scalars and is frozen once it stops.
//
// K7  vector kernels: FP64 axpy updates and deterministic column dot products; the scalars
//     (alpha, beta, rho, residual norms, per-column state) live on the device, so an iteration
//     needs no host round trip.
// K8  driver: one PCG iteration is captured as CUDA graphs (head: q = A p, alpha, u/r update,
//     residual check; tail: z = T^{-1} r, beta, p update).  IE_FP64 launches check_every
//     iterations back to back between host checks.  IE_MIXED checks after each head so that
//     the accurate residual f - A u (FP64-class, ie_matvec IE_ACCURATE) can replace r between
//     head and tail (residual replacement: when the recursive residual has dropped by
//     a set factor since the last replacement, every replace_every iterations, and when it
//     reaches tol -- a column is done only when the replaced (true) residual meets tol).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "iedd_internal.cuh"

namespace {

// Replace r by the accurate residual when the recursive residual fell by this factor since the
// last replacement (FP32 inner matvecs only).  The gap an FP32 matvec opens per cycle is about
// its error times cond(A): 1e-3 in 2D (cond ~1e5) needs a replacement every 1e3 of decrease;
// in 3D (cond ~1e3) every 1e4 suffices.
constexpr double kReplaceDrop2D = 1e-3;
constexpr double kReplaceDrop3D = 1e-4;

struct PcgCol {
    double ff;       // ||f||^2
    double rr;       // ||r||^2 (recurrence)
    double rz;       // r^T z
    double alpha, beta;
    double true_relres;
    int active;      // 1: iterating, 0: frozen
    int flag;        // 0 running, 1 recursive residual met tol, 2 done, < 0 ie_status
    int it;
    int replacements;
};

__global__ void k_init_state(PcgCol *st, const double *ff, const double *rr, double tol2, int nrhs) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    PcgCol c;
    c.ff = ff[k]; c.rr = rr[k]; c.rz = 0; c.alpha = 0; c.beta = 0; c.true_relres = -1;
    c.it = 0; c.replacements = 0;
    if (!(c.ff > 0.0)) {  // f = 0: u = 0 is exact
        c.flag = isfinite(c.ff) ? 2 : IE_ERR_BREAKDOWN;
        c.active = 0;
        c.true_relres = 0.0;
    } else if (!isfinite(c.rr)) {
        c.flag = IE_ERR_BREAKDOWN; c.active = 0;
    } else if (c.rr <= tol2 * c.ff) {
        c.flag = 1; c.active = 0;
    } else {
        c.flag = 0; c.active = 1;
    }
    st[k] = c;
}

__global__ void k_alpha(PcgCol *st, const double *pq, int nrhs) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs || st[k].active != 1) return;
    double v = pq[k];
    if (!(v > 0.0) || !isfinite(v)) {
        st[k].flag = IE_ERR_BREAKDOWN; st[k].active = 0; st[k].alpha = 0.0;
    } else {
        st[k].alpha = st[k].rz / v;
    }
}

// u += alpha p, r -= alpha q  (active columns)
__global__ void k_update(double *u, double *r, const double *p, const double *q, long long N, const PcgCol *st) {
    const int k = blockIdx.y;
    if (st[k].active != 1) return;
    const double a = st[k].alpha;
    const long long off = (long long)k * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        u[off + i] = fma(a, p[off + i], u[off + i]);
        r[off + i] = fma(-a, q[off + i], r[off + i]);
    }
}

__global__ void k_check(PcgCol *st, const double *rr, double tol2, int max_it, int nrhs) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs || st[k].active != 1) return;
    PcgCol c = st[k];
    c.it += 1;
    c.rr = rr[k];
    if (!isfinite(c.rr)) { c.flag = IE_ERR_BREAKDOWN; c.active = 0; }
    else if (c.rr <= tol2 * c.ff) { c.flag = 1; c.active = 0; }
    else if (c.it >= max_it) { c.flag = IE_ERR_MAXIT; c.active = 0; }
    st[k] = c;
}

// beta = rz_new / rz, rz = rz_new (active columns); first = 1 sets beta = 0 (p = z)
__global__ void k_beta(PcgCol *st, const double *rz_new, int nrhs, int first) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs || st[k].active != 1) return;
    double v = rz_new[k];
    if (!(v > 0.0) || !isfinite(v)) {
        st[k].flag = IE_ERR_BREAKDOWN; st[k].active = 0; return;
    }
    st[k].beta = first ? 0.0 : v / st[k].rz;
    st[k].rz = v;
}

// p = z + beta p  (active columns); first: p = z.  round32: the direction is rounded to FP32
// (the exact double-float inner matvec then needs no low word for it; a rounded search
// direction is still a valid direction for the u and r updates, which stay in FP64).
__global__ void k_pupdate(double *p, const double *z, long long N, const PcgCol *st, int first, int round32) {
    const int k = blockIdx.y;
    if (st[k].active != 1) return;
    const double b = st[k].beta;
    const long long off = (long long)k * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double v = first ? z[off + i] : fma(b, p[off + i], z[off + i]);
        p[off + i] = round32 ? (double)__double2float_rn(v) : v;
    }
}

// Warm-start fallback: a column whose initial residual is not below ||f|| restarts from u = 0
// (r = f).  rr and ff hold the squared norms of r and f per column.
__global__ void k_fallback(double *u, double *r, const double *f, double *rr, const double *ff, long long N,
                           int *used) {
    const int k = blockIdx.y;
    const bool bad = !(rr[k] < ff[k]);
    const long long off = (long long)k * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (bad) { u[off + i] = 0.0; r[off + i] = f[off + i]; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        used[k] = bad ? 0 : 1;
        if (bad) rr[k] = ff[k];
    }
}

// r = f - q for one column (or all columns when k < 0)
__global__ void k_residual(double *r, const double *f, const double *q, long long N) {
    const long long off = (long long)blockIdx.y * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        r[off + i] = f[off + i] - q[off + i];
}

// A private non-blocking stream for one solve (stream capture is not allowed on the legacy
// default stream, which is what callers often pass); it first waits for the caller's stream.
struct PrivateStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    int init(cudaStream_t user) {
        IE_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        IE_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        IE_TRY_CUDA(cudaEventRecord(ev, user));
        IE_TRY_CUDA(cudaStreamWaitEvent(s, ev, 0));
        return IE_OK;
    }
    ~PrivateStream() {
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
        if (ev) cudaEventDestroy(ev);
    }
};

struct Graph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t g = nullptr;
    long long kernels = 0;  // kernel nodes, for the launch accounting
    ~Graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
    }
};

}  // namespace

extern "C" void pcg_default_opts(pcg_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->max_it = 1000;
    o->precision = IE_MIXED;
    o->replace_every = 50;
    o->use_x0 = 0;
    o->timeout_s = 0;
    o->check_every = 8;
    o->verify = 1;
    o->inner = 0;
}

namespace {

struct Solver {
    const ie_problem *p;
    const dd_factor_t *fac;
    int nrhs;
    long long N;
    pcg_opts o;
    cudaStream_t s;
    int vgrid;
    DevBuf bf, bu, br, bz, bp, bq, bst, bsc;
    double *f, *u, *r, *z, *pp, *q;
    PcgCol *st;
    double *pq, *rr, *rz, *ff;

    // CUDA events around every inner matvec / apply / accurate matvec; recorded as external
    // event nodes inside graphs, read after the host synchronizes
    std::vector<cudaEvent_t> ev_mv, ev_ap;
    cudaEvent_t ev_acc[2] = {nullptr, nullptr};
    int n_mv = 0, n_ap = 0, n_acc = 0;
    double t_mv = 0, t_ap = 0, t_acc = 0;
    int pend_mv = 0, pend_ap = 0;  // recorded pairs not yet read
    ~Solver() {
        for (auto e : ev_mv) cudaEventDestroy(e);
        for (auto e : ev_ap) cudaEventDestroy(e);
        for (auto e : ev_acc) if (e) cudaEventDestroy(e);
    }
    int make_events(int pairs) {
        ev_mv.resize(2 * pairs);
        ev_ap.resize(2 * pairs);
        for (auto &e : ev_mv) IE_TRY_CUDA(cudaEventCreate(&e));
        for (auto &e : ev_ap) IE_TRY_CUDA(cudaEventCreate(&e));
        for (auto &e : ev_acc) IE_TRY_CUDA(cudaEventCreate(&e));
        return IE_OK;
    }
    int record(cudaEvent_t e) {
        if (ie_capturing()) IE_TRY_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
        else IE_TRY_CUDA(cudaEventRecord(e, s));
        return IE_OK;
    }
    // after a synchronize: add the device time of the pending recorded pairs
    void harvest() {
        for (int i = 0; i < pend_mv; ++i) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev_mv[2 * i], ev_mv[2 * i + 1]) == cudaSuccess) t_mv += ms;
        }
        for (int i = 0; i < pend_ap; ++i) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev_ap[2 * i], ev_ap[2 * i + 1]) == cudaSuccess) t_ap += ms;
        }
        cudaGetLastError();
        n_mv += pend_mv;
        n_ap += pend_ap;
        pend_mv = pend_ap = 0;
    }

    int alloc() {
        size_t v = sizeof(double) * (size_t)N * nrhs;
        IE_TRY(bf.alloc(v, s)); IE_TRY(bu.alloc(v, s)); IE_TRY(br.alloc(v, s));
        IE_TRY(bz.alloc(v, s)); IE_TRY(bp.alloc(v, s)); IE_TRY(bq.alloc(v, s));
        IE_TRY(bst.alloc(sizeof(PcgCol) * nrhs, s));
        IE_TRY(bsc.alloc(sizeof(double) * 4 * nrhs, s));
        f = bf.as<double>(); u = bu.as<double>(); r = br.as<double>(); z = bz.as<double>();
        pp = bp.as<double>(); q = bq.as<double>(); st = bst.as<PcgCol>();
        pq = bsc.as<double>(); rr = pq + nrhs; rz = rr + nrhs; ff = rz + nrhs;
        vgrid = (int)std::min<long long>((N + 255) / 256, (long long)p->sm_count * 8);
        return IE_OK;
    }
    int mv_precision() const {
        if (o.inner == IE_FP64 + 16) return IE_FP64;
        if (o.inner == IE_MIXED || o.inner == IE_ACCURATE || o.inner == IE_ACCURATE_X32 || o.inner == IE_TENSOR ||
            o.inner == IE_ACCURATE_R4 || o.inner == IE_ACCURATE_R16 || o.inner == IE_FFT || o.inner == IE_TENSOR_EXACT)
            return o.inner;
        if (o.precision == IE_FP64) return IE_FP64;
        if (p->dim == 2) return tc_exact_supported(p) ? IE_TENSOR_EXACT : IE_ACCURATE;
        return nrhs >= 16 ? IE_TENSOR : IE_MIXED;  // 3D batches: the tcgen05 kernel
    }
    bool exact_inner() const { return mv_precision() != IE_MIXED && mv_precision() != IE_TENSOR; }
    // the accurate residual (replacements, verification, r0 from x0): by default the FP64 FFT
    // matvec where it is supported (the paper's matvec, FP64-class and far cheaper than an FP64
    // or double-float regenerated sum); else the regenerated FP64 / double-float sum
    int acc_precision() const {
        if (o.residual == IE_FP64 + 16) return IE_FP64;
        if (o.residual) return o.residual;
        if (o.inner == IE_FFT || fft_supported(p, nullptr)) return IE_FFT;
        return o.precision == IE_FP64 ? IE_FP64 : IE_ACCURATE;
    }
    dim3 vg() const { return dim3(vgrid, nrhs); }

    int head(int slot) {
        IE_TRY(record(ev_mv[2 * slot]));
        IE_TRY(launch_matvec_dot(p, pp, N, q, N, nrhs, mv_precision(), pq, s));
        IE_TRY(record(ev_mv[2 * slot + 1]));
        k_alpha<<<(nrhs + 63) / 64, 64, 0, s>>>(st, pq, nrhs);
        IE_LAUNCHED();
        k_update<<<vg(), 256, 0, s>>>(u, r, pp, q, N, st);
        IE_LAUNCHED();
        IE_TRY(launch_dots(r, N, r, N, N, nrhs, rr, s));
        k_check<<<(nrhs + 63) / 64, 64, 0, s>>>(st, rr, o.tol * o.tol, o.max_it, nrhs);
        IE_LAUNCHED();
        return IE_OK;
    }
    int tail(int first, int slot) {
        IE_TRY(record(ev_ap[2 * slot]));
        IE_TRY(launch_apply(fac, r, N, z, N, nrhs, s));
        IE_TRY(record(ev_ap[2 * slot + 1]));
        IE_TRY(launch_dots(r, N, z, N, N, nrhs, rz, s));
        k_beta<<<(nrhs + 63) / 64, 64, 0, s>>>(st, rz, nrhs, first);
        IE_LAUNCHED();
        k_pupdate<<<vg(), 256, 0, s>>>(pp, z, N, st, first, mv_precision() == IE_ACCURATE_X32 ? 1 : 0);
        IE_LAUNCHED();
        return IE_OK;
    }
    // accurate residual of column k into r[:, k]; returns ||r_k||^2 (synchronizes)
    int accurate_residual(int k, double *rr_host) {
        const long long off = (long long)k * N;
        IE_TRY(record(ev_acc[0]));
        IE_TRY(launch_matvec(p, u + off, N, q + off, N, 1, acc_precision(), s));
        IE_TRY(record(ev_acc[1]));
        k_residual<<<dim3(vgrid, 1), 256, 0, s>>>(r + off, f + off, q + off, N);
        IE_LAUNCHED();
        IE_TRY(launch_dots(r + off, N, r + off, N, N, 1, rr + k, s));
        IE_TRY_CUDA(cudaMemcpyAsync(rr_host, rr + k, sizeof(double), cudaMemcpyDeviceToHost, s));
        IE_TRY_CUDA(cudaStreamSynchronize(s));
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ev_acc[0], ev_acc[1]) == cudaSuccess) t_acc += ms;
        cudaGetLastError();
        n_acc += 1;
        return IE_OK;
    }
    int capture(Graph &gr, int which, int reps) {
        IE_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        ie_set_capturing(true);
        int rc = IE_OK;
        for (int i = 0; i < reps && rc == IE_OK; ++i) {
            if (which & 1) rc = head(i);
            if (rc == IE_OK && (which & 2)) rc = tail(0, i);
        }
        ie_set_capturing(false);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc != IE_OK) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) { ie_set_error(std::string("graph capture: ") + cudaGetErrorString(e)); return IE_ERR_CUDA; }
        gr.g = g;
        size_t nn = 0;
        IE_TRY_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        IE_TRY_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) gr.kernels++;
        }
        IE_TRY_CUDA(cudaGraphInstantiate(&gr.exec, g, 0));
        return IE_OK;
    }
    int launch(const Graph &gr, int mv_pairs, int ap_pairs) {
        IE_TRY_CUDA(cudaGraphLaunch(gr.exec, s));
        ie_count_launches(gr.kernels);
        pend_mv += mv_pairs;
        pend_ap += ap_pairs;
        return IE_OK;
    }
};

}  // namespace

extern "C" int pcg_solve(const ie_problem *p, const dd_factor_t *fac, const double *rhs, double *u_out, int nrhs,
                         long long ld, const pcg_opts *opts, pcg_report *rep, void *stream) {
    if (!p || !fac) { ie_set_error("pcg_solve: NULL problem or factor"); return IE_ERR_ARG; }
    if (fac->prob != p) { ie_set_error("pcg_solve: factor belongs to another problem"); return IE_ERR_ARG; }
    if (!rhs || !u_out) { ie_set_error("pcg_solve: NULL vector"); return IE_ERR_ARG; }
    if (nrhs < 1 || ld < p->N) { ie_set_error("pcg_solve: need nrhs >= 1 and ld >= N"); return IE_ERR_ARG; }
    pcg_opts o;
    if (opts) o = *opts; else pcg_default_opts(&o);
    if (!(o.tol >= 0.0) || o.max_it < 1 || (o.precision != IE_FP64 && o.precision != IE_MIXED) ||
        o.replace_every < 0 || o.check_every < 0 || o.use_x0 < 0 || o.use_x0 > 2 ||
        (o.inner != 0 && o.inner != IE_MIXED && o.inner != IE_ACCURATE && o.inner != IE_ACCURATE_X32 &&
         o.inner != IE_TENSOR && o.inner != IE_ACCURATE_R4 && o.inner != IE_ACCURATE_R16 &&
         o.inner != IE_FP64 + 16 && o.inner != IE_FFT && o.inner != IE_TENSOR_EXACT) ||
        (o.residual != 0 && o.residual != IE_ACCURATE && o.residual != IE_FP64 + 16 && o.residual != IE_FFT)) {
        ie_set_error("pcg_solve: invalid options"); return IE_ERR_ARG;
    }
    if (o.check_every < 1) o.check_every = 1;
    const auto t_start = std::chrono::steady_clock::now();
    DeviceGuard g(p->device);
    PrivateStream ps;
    IE_TRY(ps.init(static_cast<cudaStream_t>(stream)));
    Solver S{p, fac, nrhs, p->N, o, ps.s};
    if (S.mv_precision() == IE_FFT || S.acc_precision() == IE_FFT) IE_TRY(prepare_fft(p));  // before any capture
    if (S.mv_precision() == IE_TENSOR_EXACT) {
        if (!tc_exact_supported(p)) {
            ie_set_error("pcg_solve: IE_TENSOR_EXACT needs a 2D grid with n a multiple of 128 and n <= 4096");
            return IE_ERR_ARG;
        }
        IE_TRY(prepare_tc_exact(p));  // before any capture
    }
    if (S.mv_precision() == IE_TENSOR) IE_TRY(prepare_tc_strip(p));  // before any capture
    if (S.mv_precision() == IE_TENSOR || S.mv_precision() == IE_TENSOR_EXACT)
        IE_TRY_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    IE_TRY(S.alloc());
    IE_TRY(S.make_events(std::max(o.check_every, 1)));
    const long long N = p->N;
    const size_t rowb = sizeof(double) * N, ldb = sizeof(double) * ld;
    const cudaMemcpyKind kin = ie_is_device_ptr(rhs) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const bool u_dev = ie_is_device_ptr(u_out);
    cudaStream_t s = S.s;
    IE_TRY_CUDA(cudaMemcpy2DAsync(S.f, rowb, rhs, ldb, rowb, nrhs, kin, s));
    if (o.use_x0) {
        IE_TRY_CUDA(cudaMemcpy2DAsync(S.u, rowb, u_out, ldb, rowb, nrhs,
                                      u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        IE_TRY(launch_matvec(p, S.u, N, S.q, N, nrhs, S.acc_precision(), s));
        k_residual<<<S.vg(), 256, 0, s>>>(S.r, S.f, S.q, N);
        IE_LAUNCHED();
    } else {
        IE_TRY_CUDA(cudaMemsetAsync(S.u, 0, sizeof(double) * N * nrhs, s));
        IE_TRY_CUDA(cudaMemcpyAsync(S.r, S.f, sizeof(double) * N * nrhs, cudaMemcpyDeviceToDevice, s));
    }
    IE_TRY_CUDA(cudaMemsetAsync(S.pp, 0, sizeof(double) * N * nrhs, s));
    IE_TRY(launch_dots(S.f, N, S.f, N, N, nrhs, S.ff, s));
    IE_TRY(launch_dots(S.r, N, S.r, N, N, nrhs, S.rr, s));
    DevBuf used;
    IE_TRY(used.alloc(sizeof(int) * nrhs, s));
    if (o.use_x0 == 2) {
        k_fallback<<<S.vg(), 256, 0, s>>>(S.u, S.r, S.f, S.rr, S.ff, N, used.as<int>());
        IE_LAUNCHED();
    } else {
        IE_TRY_CUDA(cudaMemsetAsync(used.ptr, o.use_x0 ? 0x01 : 0, sizeof(int) * nrhs, s));
    }
    std::vector<int> x0_used((size_t)nrhs, 0);
    k_init_state<<<(nrhs + 63) / 64, 64, 0, s>>>(S.st, S.ff, S.rr, o.tol * o.tol, nrhs);
    IE_LAUNCHED();
    IE_TRY(S.tail(1, 0));
    S.pend_ap = 1;

    std::vector<PcgCol> hs((size_t)nrhs);
    std::vector<double> last_true((size_t)nrhs, INFINITY), relres_at_replace((size_t)nrhs, 1.0);
    auto read_states = [&]() -> int {
        IE_TRY_CUDA(cudaMemcpyAsync(hs.data(), S.st, sizeof(PcgCol) * nrhs, cudaMemcpyDeviceToHost, s));
        IE_TRY_CUDA(cudaStreamSynchronize(s));
        S.harvest();
        return IE_OK;
    };
    auto write_states = [&]() -> int {
        IE_TRY_CUDA(cudaMemcpyAsync(S.st, hs.data(), sizeof(PcgCol) * nrhs, cudaMemcpyHostToDevice, s));
        return IE_OK;
    };
    auto timed_out = [&]() {
        if (o.timeout_s <= 0) return false;
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        return el > o.timeout_s;
    };
    const bool mixed = o.precision == IE_MIXED;
    IE_TRY(read_states());

    if (!mixed) {
        Graph gr;
        IE_TRY(S.capture(gr, 3, o.check_every));
        for (;;) {
            bool any = false;
            for (auto &c : hs) {
                if (c.flag == 1) c.flag = 2;
                any |= c.active == 1;
            }
            if (!any) break;
            if (timed_out()) {
                for (auto &c : hs) if (c.active == 1) { c.active = 0; c.flag = IE_ERR_TIMEOUT; }
                break;
            }
            IE_TRY(S.launch(gr, o.check_every, o.check_every));
            IE_TRY(read_states());
        }
        IE_TRY(write_states());
    } else {
        Graph gh, gt;
        IE_TRY(S.capture(gh, 1, 1));
        IE_TRY(S.capture(gt, 2, 1));
        // Replacement step, run after every head (and once before the first one, for columns
        // whose initial residual already meets tol): r := f - A u with the accurate matvec for
        // columns that met tol on the recurrence, or are due for a periodic replacement.
        auto replace = [&]() -> int {
            bool changed = false;
            for (int k = 0; k < nrhs; ++k) {
                PcgCol &c = hs[(size_t)k];
                double relres = c.ff > 0 ? std::sqrt(c.rr / c.ff) : 0.0;
                bool pending = c.flag == 1;
                bool due = c.active == 1 &&
                           ((o.replace_every > 0 && c.it > 0 && c.it % o.replace_every == 0) ||
                            (!S.exact_inner() &&
                             relres <= (p->dim == 2 ? kReplaceDrop2D : kReplaceDrop3D) * relres_at_replace[(size_t)k]));
                if (!pending && !due) continue;
                double rr_true = 0;
                IE_TRY(S.accurate_residual(k, &rr_true));
                double tr = std::sqrt(rr_true / c.ff);
                c.rr = rr_true;
                c.replacements += 1;
                c.true_relres = tr;
                relres_at_replace[(size_t)k] = tr;
                changed = true;
                if (pending) {
                    if (tr <= o.tol) {
                        c.flag = 2;
                    } else if (tr >= 0.5 * last_true[(size_t)k]) {
                        c.flag = IE_ERR_STAGNATION;
                    } else if (c.it >= o.max_it) {
                        c.flag = IE_ERR_MAXIT;
                    } else {
                        c.flag = 0;
                        c.active = 1;
                    }
                    last_true[(size_t)k] = tr;
                }
            }
            if (changed) IE_TRY(write_states());
            return IE_OK;
        };
        auto any_active = [&]() {
            for (auto &c : hs) if (c.active == 1) return true;
            return false;
        };
        IE_TRY(replace());
        bool need_tail = false;  // the initial tail already ran
        while (any_active()) {
            if (timed_out()) {
                for (auto &c : hs) if (c.active == 1) { c.active = 0; c.flag = IE_ERR_TIMEOUT; }
                IE_TRY(write_states());
                break;
            }
            if (need_tail) IE_TRY(S.launch(gt, 0, 1));  // z = T^{-1} r, beta, p
            IE_TRY(S.launch(gh, 1, 0));                 // q = A p, alpha, u/r, check
            IE_TRY(read_states());
            IE_TRY(replace());
            need_tail = true;
        }
    }
    // true residual for the report
    if (!mixed && o.verify) {
        for (int k = 0; k < nrhs; ++k) {
            double rr_true = 0;
            IE_TRY(S.accurate_residual(k, &rr_true));
            hs[(size_t)k].true_relres = hs[(size_t)k].ff > 0 ? std::sqrt(rr_true / hs[(size_t)k].ff) : 0.0;
        }
    }
    IE_TRY_CUDA(cudaMemcpy2DAsync(u_out, ldb, S.u, rowb, rowb, nrhs,
                                  u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    IE_TRY_CUDA(cudaMemcpyAsync(x0_used.data(), used.ptr, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    int tc_err = 0;
    if (S.mv_precision() == IE_TENSOR || S.mv_precision() == IE_TENSOR_EXACT)  // a CTA gave up waiting for its MMAs
        IE_TRY_CUDA(cudaMemcpyAsync(&tc_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IE_TRY_CUDA(cudaStreamSynchronize(s));
    int ret = IE_OK;
    if (tc_err) {
        ret = IE_ERR_TIMEOUT;
        ie_set_error("pcg_solve: the tensor-core matvec timed out waiting for its MMAs");
    }
    for (int k = 0; k < nrhs; ++k) {
        const PcgCol &c = hs[(size_t)k];
        int stk = tc_err ? IE_ERR_TIMEOUT : c.flag == 2 ? IE_OK : (c.flag < 0 ? c.flag : IE_ERR_MAXIT);
        if (stk != IE_OK && ret == IE_OK) {
            ret = stk;
            ie_set_error("pcg_solve: column " + std::to_string(k) + " stopped with status " + std::to_string(stk));
        }
        if (rep) {
            rep[k].iterations = c.it;
            rep[k].replacements = c.replacements;
            rep[k].status = stk;
            rep[k].x0_used = o.use_x0 == 2 ? (x0_used[(size_t)k] != 0) : (o.use_x0 ? 1 : 0);
            rep[k].recursive_relres = c.ff > 0 ? std::sqrt(c.rr / c.ff) : 0.0;
            rep[k].true_relres = c.true_relres;
            rep[k].matvecs = S.n_mv;
            rep[k].applies = S.n_ap;
            rep[k].matvec_ms = S.t_mv;
            rep[k].apply_ms = S.t_ap;
            rep[k].accurate_matvecs = S.n_acc;
            rep[k].accurate_mode = S.acc_precision();
            rep[k].accurate_ms = S.t_acc;
        }
    }
    return ret;
}
