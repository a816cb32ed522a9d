/*
 * iedd.h -- C ABI of the GB300 (sm_103a) library for preconditioned conjugate gradient on the
 * dense SPD collocation system of the first-kind Laplace volume integral equation, with the
 * additive overlapping domain-decomposition preconditioner of Chen & Biros, "Overlapping
 * Domain Decomposition Preconditioner for Integral Equations" (arXiv 2108.12574).
 *
 * The problem (Sec. 2.1, Eqs. e:ie, e:k):   int_Omega K(x - y) u(y) dy = f(x),  Omega = [0,1]^d,
 *   K(r) = -(1/2pi) log|r| (d = 2),  K(r) = 1/(4 pi |r|) (d = 3),
 * discretized by piecewise-constant collocation on an n^d grid into A u = f (Eq. e:dis) with
 *   A_ij = h^d K(x_i - x_j) for i != j and A_ii = the integral of K over the h^d self cell
 *   (Eqs. e:a_2d, e:a_3d), h = 1/n,  plus an optional second-kind shift a on the diagonal
 *   (the a u term of Eq. e:int).
 * The preconditioner (Sec. 3, Eqs. e:ai, e:ad):  T^{-1} = sum_i R_i^T A_i^{-1} R_i,
 *   A_i = R_i A R_i^T, over the subdomains of Table t:dd (block Jacobi, Schwarz, CBD).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Grid index: row-major, last coordinate fastest (2D: i = i1 * n + i2).
 *  - Vectors are FP64.  A batch of nrhs vectors is column-major: entry (i, k) at x[k * ld + i],
 *    ld >= N.  A vector pointer may be device memory or host memory (pageable or pinned); the
 *    library detects which with cudaPointerGetAttributes and, for host memory, stages through
 *    device memory itself (the copies are enqueued on the caller's stream and the call
 *    synchronizes that stream before returning).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  All
 *    device work is enqueued on it.  Calls that return data to the host (dd_factor's info,
 *    pcg_solve's report, any call given host vectors) synchronize the stream.
 *  - Handles are opaque, owned by the library, created by the call that returns them and freed
 *    by the matching *_destroy (which accepts NULL).  A handle may be used from one host thread
 *    at a time.
 *  - No call aborts or exits.  Every call returns an ie_status; on failure ie_last_error()
 *    returns a message for the calling thread.  A CUDA error inside a call is reported as
 *    IE_ERR_CUDA and leaves output buffers unspecified.
 */
#ifndef IEDD_H
#define IEDD_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define IEDD_API __attribute__((visibility("default")))
#else
#define IEDD_API
#endif

typedef enum {
    IE_OK = 0,
    IE_ERR_ARG = -1,         /* invalid argument (sizes, pointers, modes)                      */
    IE_ERR_CUDA = -2,        /* a CUDA runtime call failed                                     */
    IE_ERR_OOM = -3,         /* device allocation failed                                       */
    IE_ERR_NOT_SPD = -4,     /* a subdomain block had a non-positive Cholesky pivot            */
    IE_ERR_BREAKDOWN = -5,   /* PCG met p^T A p <= 0, r^T z <= 0 or a NaN                      */
    IE_ERR_MAXIT = -6,       /* PCG reached max_it before the tolerance                        */
    IE_ERR_STAGNATION = -7,  /* the true residual stopped decreasing                            */
    IE_ERR_TIMEOUT = -8      /* the wall-clock budget of pcg_opts.timeout_s ran out            */
} ie_status;

typedef enum {
    IE_FP64 = 0,   /* every step in FP64: entries regenerated in FP64, FP64 factors            */
    IE_MIXED = 1   /* FP32 matvec and FP32 factors; FP64 CG scalars, FP64 residual replacement */
} ie_precision;

typedef enum { DD_JACOBI = 0, DD_SCHWARZ = 1, DD_CBD = 2 } dd_kind;

typedef enum {
    IE_GRID_TEXT = 0,  /* x_j = h (j - 1/2), j = 1..n: the cell-centred grid of Sec. 2.1          */
    IE_GRID_TABLE = 1  /* x_j = (j - 1)/(n - 1) with weight (1/n)^d: the spacing under which the
                          paper's 2D eigenvalue tables (Sec. 3-4) are reproduced; for checks only */
} ie_grid;

typedef struct ie_problem ie_problem;
typedef struct dd_partition_t dd_partition_t;
typedef struct dd_factor_t dd_factor_t;

/* Thread-local message describing the last failure of a call on this thread ("" if none). */
IEDD_API const char *ie_last_error(void);

/* Library version string. */
IEDD_API const char *ie_version(void);

/*
 * ie_discretize -- the collocation discretization of Sec. 2.1 (Eqs. e:a_2d, e:a_3d).
 *   dim      2 or 3
 *   n        grid points per dimension, 2 <= n; N = n^dim <= 2^26
 *   a_shift  second-kind term a added to the diagonal (0 for the first-kind equation); A stays
 *            SPD for a >= 0, a negative a can make it (and its blocks) indefinite
 *   grid     ie_grid convention
 *   device   CUDA device ordinal used by everything created from this problem
 *   out      receives the new handle
 * Builds the point coordinates and the per-offset entry table (used by the accurate residual)
 * on the device; synchronous.  The diagonal is the closed-form self-cell integral
 *   2D: -(h^2/(4 pi)) (2 ln(h/2) + ln 2 - 3 + pi/2);   3D: (h^2/(2 pi)) (3 ln(1+sqrt 3) - 1.5 ln 2 - pi/4).
 * Errors: IE_ERR_ARG for bad sizes, IE_ERR_OOM, IE_ERR_CUDA.
 */
IEDD_API int ie_discretize(int dim, int n, double a_shift, int grid, int device, ie_problem **out);

/* Sizes and constants of a problem: any output pointer may be NULL.  diag is A_ii. */
IEDD_API int ie_problem_info(const ie_problem *p, int *dim, int *n, long long *N, double *h, double *diag);

IEDD_API void ie_destroy(ie_problem *p);

/*
 * ie_matvec -- y = A x (Eq. e:dis), matrix-free: every entry is regenerated from the point
 * coordinates and the quadrature weight; nothing of A is stored.
 *   x, y       N x nrhs, column-major with leading dimension ld (host or device, FP64);
 *              x and y must not overlap
 *   precision  IE_FP64: entries and sums in FP64.
 *              IE_MIXED: entries h^d K in FP32 through the SFU (log2 / rsqrt), FP32 sums per
 *              tile, combined with the FP64 diagonal term in FP64.  Relative error of order
 *              1e-6 of ||A|| ||x||.
 *              IE_MIXED + 2 (= 3, "accurate"): double-float sums of a per-offset FP64 entry
 *              table; FP64-class result (relative error ~1e-13 of sum |A_ij x_j|).
 * Errors: IE_ERR_ARG (nrhs < 1, ld < N, NULL pointers), IE_ERR_CUDA.
 */
IEDD_API int ie_matvec(const ie_problem *p, const double *x, double *y, int nrhs, long long ld,
              int precision, void *stream);
#define IE_ACCURATE 3
#define IE_STORED 5   /* ie_matvec from the stored FP32 matrix (ie_store_matrix); HBM-bound */
#define IE_TENSOR 6   /* entries contracted with x on the tcgen05 tensor cores (3xTF32 split,
                         FP32 accumulation in tensor memory), 64 right-hand sides per CTA; the
                         entries come from the exact per-offset table for n = 32, 64 or a multiple
                         of 128, else from the FP32 SFU; same accuracy class as IE_MIXED.  Returns IE_ERR_TIMEOUT if a CTA gave
                         up waiting for its MMAs (bounded waits; the call then synchronizes). */
#define IE_FFT 9      /* the paper's FFT matvec (Sec. 6): A is Toeplitz in every coordinate on the
                         uniform grid, so A x is a convolution, computed in FP64 on the periodic
                         grid of L^d points (L the power of two >= 2n - 1; pairs of columns share
                         one complex transform).  FP64-class result.  n <= 4096 (IE_ERR_ARG
                         otherwise).  The first IE_FFT call on a problem builds the kernel's
                         spectrum (8 L^d bytes, kept until ie_destroy) and synchronizes; it must
                         not be inside a stream capture and must not run concurrently with another
                         call on the same problem.  Scratch: 16 L^d bytes per pair of columns. */
#define IE_TENSOR_EXACT 10 /* the 2D direct sum on the tcgen05 tensor cores with an FP64-class
                         result (Ozaki scheme): the per-offset FP64 entries and x are cut into six
                         fixed-point BF16 digits each; the 21 leading digit products are summed
                         exactly (FP32 windows of 128 terms, then 64-bit integers).  Relative
                         error ~1e-16 of sum |A_ij x_j|.  2D with n a multiple of 128, n <= 4096
                         (IE_ERR_ARG otherwise).  The first call on a problem builds the digit
                         window table (192 N bytes, kept until ie_destroy) and synchronizes; it must not
                         be inside a stream capture.  Returns IE_ERR_TIMEOUT if a CTA gave up
                         waiting for its MMAs (bounded waits). */

/*
 * ie_store_matrix -- stored-matrix fallback: materialise the off-diagonal part of A densely in
 * device memory (FP32, row-major N x N, 4 N^2 bytes; entries from the FP64 per-offset table,
 * rounded once) so that ie_matvec(..., IE_STORED, ...) streams it instead of regenerating entries
 * (the diagonal stays FP64).  Returns IE_ERR_OOM when 4 N^2 bytes exceed 90 % of the free device
 * memory (N <= ~2.5e5 on a GB300).  Synchronizes the stream.  ie_release_matrix frees it.
 */
IEDD_API int ie_store_matrix(ie_problem *p, void *stream);
IEDD_API int ie_release_matrix(ie_problem *p);

/*
 * dd_partition -- index sets of the subdomains (Sec. 2.2-2.3, Eqs. e:dd, e:first, e:cbd).
 *   m      partitions per dimension (M = m^dim boxes of w = n/m cells; n % m == 0 required)
 *   delta  overlap: each box is extended by delta grid layers in every direction, clipped to
 *          the grid (ignored for DD_JACOBI)
 *   kind   DD_JACOBI (the boxes), DD_SCHWARZ (the extended boxes, D = M) or DD_CBD (extended
 *          boxes unioned by the parity colour (k_1 mod 2, ..., k_d mod 2), D = 2^dim)
 * Index sets are in ascending global order.  Host-side; the sets are also copied to the device.
 * Errors: IE_ERR_ARG (n % m != 0, delta < 0, a DD_JACOBI or DD_SCHWARZ subdomain larger than 25600
 * points; a larger DD_CBD subdomain is accepted here and refused by dd_factor, dd_factor_rs takes
 * it), IE_ERR_OOM.
 */
IEDD_API int dd_partition(const ie_problem *p, int m, int delta, int kind, dd_partition_t **out);

/* Number of subdomains D, total index count sum_i n_i and the largest n_i. */
IEDD_API int dd_partition_info(const dd_partition_t *s, int *nblocks, long long *total, int *max_block);

/* Copies the CSR form to host arrays: offsets[nblocks + 1] (int64) and index[total] (int32). */
IEDD_API int dd_partition_export(const dd_partition_t *s, long long *offsets, int *index);

IEDD_API void dd_partition_destroy(dd_partition_t *s);

/*
 * dd_factor -- regenerate every A_i = R_i A R_i^T (Eq. e:ai) and factor it, A_i = L_i L_i^T,
 * by dense Cholesky (the exact subdomain solver of Sec. 4.3), all blocks in one launch.
 *   precision  IE_FP64: FP64 entries and factors, one CTA per block on the CUDA cores (blocks of
 *              at most 8192 points, else IE_ERR_ARG).  IE_MIXED: FP32 entries; the Cholesky
 *              factor and the explicit symmetric inverse M_i = A_i^{-1} of every block are
 *              computed on the tcgen05 tensor cores (3xTF32 products, FP32 storage), and dd_apply
 *              multiplies by M_i.
 *   info       (host, may be NULL) receives -1 if every block is SPD, else the first failing
 *              block index; the call then returns IE_ERR_NOT_SPD and *out is still created
 *              (its failing blocks are unusable).  IE_ERR_TIMEOUT if a tensor-core task gave up
 *              waiting for its MMAs (bounded waits).
 * The factor keeps references to p's device data: destroy it before the problem.
 * Synchronizes the stream (to read the per-block status).
 */
IEDD_API int dd_factor(const ie_problem *p, const dd_partition_t *s, int precision, dd_factor_t **out,
              int *info, void *stream);

IEDD_API void dd_factor_destroy(dd_factor_t *f);

/*
 * dd_factor_rs -- the CBD preconditioner with every subdomain factored approximately by recursive
 * skeletonization (Sec. 4.3, "Recursive skeletonization (RS) as subdomain solver": Eqs. e:oi,
 * e:block, e:id, e:id_err, e:al, e:alu, e:b, e:schur), on the device, in FP64.
 *   s     a DD_CBD partition with 2 delta <= n / m (the extended boxes of one colour are then
 *         disjoint: the regions of Eq. e:oi); s and p must outlive the factor
 *   opts  (host, may be NULL: defaults) relative accuracy eps of every ID (Eq. e:id_err; default
 *         1e-3, the paper's), proxy points nproxy (default 64 in 2D, 256 in 3D) and proxy radius
 *         rho in units of a region's longest side (default 1.5, the paper's)
 * For each colour: level 1 takes the colour's extended boxes as regions; at every level each
 * region's DOFs are split by an ID of A_qp (q: the other regions' DOFs of the subdomain) into
 * skeletons s and redundant r with A_qr ~ A_qs T, computed through a proxy circle (2D; plus one
 * constant row for the log kernel's monopole) or sphere (3D) of radius rho * side around the
 * region's box with the DOFs of other regions inside it as explicit rows; the redundant DOFs are
 * eliminated (B_rr = L L^T, B_ss = A_ss - B_sr B_rr^{-1} B_rs), and 2^d neighbouring regions merge
 * into one region of the next level, until one is left, whose Schur complement is factored by
 * dense Cholesky.  Pivots are column-pivoted Gram-Schmidt with a tie window (the lowest-index
 * column within min(top / 2, max(1e-10 top, 1e-13 nu0)) of the largest squared norm), so that
 * the symmetric grid's exact ties break the same way under any rounding.
 * The result is a dd_factor_t that dd_apply and pcg_solve use like any other: z = sum_c R_c^T
 * F_c^{-1} R_c r with the approximate factors F_c ~ A_c (symmetric positive definite).
 * Synchronizes the stream.  Errors: IE_ERR_ARG (not DD_CBD, 2 delta > n / m, bad opts, a region
 * above 4096 DOFs or 16384 ID rows, a last Schur complement above 8192 DOFs), IE_ERR_NOT_SPD (a
 * non-positive pivot of some B_rr; *out stays NULL), IE_ERR_OOM, IE_ERR_CUDA.
 */
typedef struct {
    double eps;   /* 0: 1e-3 */
    int nproxy;   /* 0: 64 (2D) or 256 (3D) */
    double rho;   /* 0: 1.5 */
} rs_opts;

IEDD_API int dd_factor_rs(const ie_problem *p, const dd_partition_t *s, const rs_opts *opts, dd_factor_t **out,
                          void *stream);

/*
 * dd_rs_info -- shape of an RS factor: *ncolours = 2^dim; per colour c, levels[c] compression
 * levels and top[c] DOFs at the last level (S of Sec. 5's tables).  stats[4]: the algorithmic FP64
 * flops of the IDs and of the eliminations (counted from the regions' shapes and ranks), and the
 * summed device time in ms of their kernel launches (CUDA events on the factor's stream).  Arrays
 * hold 2^dim entries; any pointer may be NULL.  IE_ERR_ARG if f is not from dd_factor_rs.
 */
IEDD_API int dd_rs_info(const dd_factor_t *f, int *ncolours, int *levels, int *top, double *stats);

/*
 * dd_rs_export -- the regions of colour `colour` at level `level` (1-based; levels[c] + 1 is the
 * last level): *nreg regions, *total DOFs; offsets[nreg + 1] (int64) into points[total] (int32,
 * global grid indices), each region's DOFs with its skeletons first, in pivot order, then its
 * redundant DOFs; rank[nreg] the skeleton counts (at the last level: the size).  Regions come in
 * row-major order of their colour-grid coordinate.  Call once with NULL arrays for the sizes.
 */
IEDD_API int dd_rs_export(const dd_factor_t *f, int colour, int level, int *nreg, long long *total,
                          long long *offsets, int *points, int *rank);

/*
 * dd_apply -- z = T^{-1} r = sum_i R_i^T A_i^{-1} R_i r (Eq. e:ad), then a plain (unweighted) sum
 * over the overlaps, taken in a fixed order so the result is bitwise reproducible.
 *   r, z  N x nrhs column-major, leading dimension ld (host or device, FP64); must not overlap.
 * IE_FP64 factors: forward and backward triangular solves with L_i in FP64.  IE_MIXED factors:
 * z_i = M_i (R_i r) with the FP32 inverse, products and sums in double-float (FP32 sums for
 * 3D batches of >= 4 columns), so the operator is a fixed symmetric matrix; z is FP64.
 */
IEDD_API int dd_apply(const dd_factor_t *f, const double *r, double *z, int nrhs, long long ld,
             void *stream);

typedef struct {
    double tol;          /* stop when ||f - A u||_2 <= tol ||f||_2 (true residual, see below)     */
    int max_it;          /* iteration cap per right-hand side (products q = A p)                  */
    int precision;       /* IE_FP64 or IE_MIXED (the factor may have either precision)            */
    int replace_every;   /* IE_MIXED: replace r by the accurate f - A u every k iterations (0: off) */
    int use_x0;          /* 1: u holds the initial iterate on entry; 0: start from u = 0;
                            2: as 1, but a column whose initial residual ||f - A u|| is not
                            below ||f|| starts from u = 0 instead (warm-start fallback)          */
    double timeout_s;    /* wall-clock budget (0: none); exceeded -> IE_ERR_TIMEOUT                */
    int check_every;     /* IE_FP64: iterations per CUDA-graph launch between host checks (>= 1)  */
    int verify;          /* IE_FP64: 1 = compute the true residual at the end (one more matvec)    */
    int inner;           /* matvec inside the iteration (q = A p):
                              0            the library's choice: IE_FP64 precision -> the FP64
                                           regenerated matvec; IE_MIXED -> IE_TENSOR_EXACT in
                                           2D where supported (n a multiple of 128, n <= 4096),
                                           else IE_ACCURATE; IE_TENSOR for 3D batches of >= 16
                                           columns, IE_MIXED for fewer
                              IE_MIXED     FP32 SFU entries with compensated FP32 sums
                              IE_ACCURATE  double-float table sums on the FP32 pipes
                              4            as IE_ACCURATE with the search directions rounded to
                                           FP32 (one FFMA less per pair, more iterations)
                              IE_TENSOR    the tcgen05 batched kernel (many right-hand sides)
                              IE_TENSOR_EXACT  the exact 2D tensor-core sum (see ie_matvec)
                              IE_FFT       the FP64 FFT matvec (Sec. 6), also used for the
                                           accurate residual; the first use builds its plan
                              16           the FP64 regenerated matvec in either precision */
    int residual;        /* matvec of the accurate residual f - A u (IE_MIXED replacements, the
                            final verification, r0 from a given x0):
                              0            the library's choice: IE_FFT where supported
                                           (n <= 4096), else IE_FP64 / IE_ACCURATE by precision
                              IE_FFT, IE_ACCURATE   that matvec
                              16           the FP64 regenerated matvec (IE_FP64 is 0, the
                                           library's choice, so it is selected as 16) */
} pcg_opts;

typedef struct {
    int iterations;          /* products q = A p for this right-hand side                       */
    int replacements;        /* accurate residual recomputations (IE_MIXED)                       */
    int status;              /* ie_status of this right-hand side                                 */
    int x0_used;             /* 1 if the column started from the caller's u, 0 if from zero        */
    double recursive_relres; /* ||r_k||_2 / ||f||_2 of the recurrence                             */
    double true_relres;      /* ||f - A u||_2 / ||f||_2 with the accurate matvec (-1 if not run)  */
    /* per-solve device timing (CUDA events around each launch; the same in every column)     */
    int matvecs;             /* inner matvecs q = A p (one launch covers all columns)           */
    int applies;             /* preconditioner applications z = T^{-1} r                        */
    double matvec_ms;        /* summed device time of the inner matvecs                         */
    double apply_ms;         /* summed device time of the applications                          */
    int accurate_matvecs;    /* accurate f - A u evaluations (replacement, verification)        */
    int accurate_mode;       /* ie_matvec mode of those (IE_FFT, IE_FP64 or IE_ACCURATE)         */
    double accurate_ms;      /* summed device time of those                                     */
} pcg_report;

/*
 * ie_matvec_noalloc -- y = A x with the FP32 SFU matvec (the kernel ie_matvec runs for IE_MIXED,
 * same accuracy), for callers that cannot allocate device memory: code that runs where
 * cudaMalloc is forbidden or unsafe (inside an allocator or a memory-capped host framework,
 * or after all memory was reserved up front).  The paper has no counterpart of this call.
 *   dim, n, a_shift, grid   as ie_discretize (no problem handle is needed: the point
 *                           coordinates are derived from the grid index); N = n^dim must be
 *                           <= IE_NOALLOC_MAX_N, else IE_ERR_ARG with a message
 *   x, y                    FP64 vectors of length N (one right-hand side) in the memory of the
 *                           current device (device or managed memory); host pointers and
 *                           another device's memory are rejected with IE_ERR_ARG (staging or
 *                           peer access would allocate or fault), as are overlapping x and y
 *   stream                  cudaStream_t of the current device (NULL: legacy default stream),
 *                           else IE_ERR_ARG; the call is asynchronous
 * It allocates nothing: no cudaMalloc, cudaFree or allocating library routine.  Its scratch is one
 * file-scope device array of IE_NOALLOC_SCRATCH_BYTES.  The array is reserved on a device when
 * the library's device code for this call is loaded there -- lazily by default in CUDA (the
 * first call on that device), eagerly at context creation under CUDA_MODULE_LOADING=EAGER --
 * and it stays until the process exits.  A caller that reserves all free memory up front must
 * therefore make one call on each device first (or load eagerly).  The first call on a device
 * also looks up the array's address (cudaGetSymbolAddress, with that device current) and
 * caches it for the process; make that first call before any stream capture.  The cached
 * address does not survive cudaDeviceReset: do not use this call on a device after resetting
 * it.  All calls share the array and each overwrites what it reads, so nothing carries over
 * from one call to the next; calls whose GPU work overlaps (other streams, other threads)
 * race on the array and must be ordered by the caller.
 */
#define IE_NOALLOC_SCRATCH_BYTES (32LL << 20)
#define IE_NOALLOC_MAX_N (4194304LL - 1024LL)
IEDD_API int ie_matvec_noalloc(int dim, int n, double a_shift, int grid, const double *x, double *y,
                               void *stream);

/*
 * Learned warm start (not in the paper: a production layer on top of the method).  A 4-level
 * U-Net (encoder 12/24/48/96 channels, 2x2 average pooling, nearest upsampling with skip
 * concatenation, ReLU, 1x1 output; 274,213 parameters; NHWC; BF16 weights and activations with
 * FP32 accumulation; FP32 master weights and Adam) maps a 2D right-hand side f to an initial
 * iterate u0 for pcg_solve (use_x0 = 1).  Inputs: f / rms(f) and the normalised 5-point
 * Laplacian of f; output scale rms(Laplacian f) / h^2 (u is close to -Laplace(f) inside the
 * domain).  The grid side must be a multiple of 16.  Parameter vector layout (FP32): for each
 * layer in order, W[Cout][3][3][Cin] (W[Cout][Cin] for the 1x1) followed by b[Cout].
 *
 * ws_create       He-normal initial weights from SplitMix64 (seed), zero biases.
 * ws_get_params / ws_set_params   copy the FP32 master weights (host arrays of ws_num_params).
 * ws_forward_raw  in: [B][n][n][2] FP32 (host or device), out: [B][n][n] FP32; B <= 16.
 * ws_backward_raw gradient of sum(dout * out) with respect to the parameters (FP32, nparams),
 *                 for the input `in`; no update.
 * ws_train_step   one Adam step (lr; beta 0.9 / 0.999) on the MSE between the network output and
 *                 the scaled target u, for `batch` <= 16 device columns of f and u (ld >= N) of a
 *                 2D problem; *loss (host, may be NULL) receives the loss before the step.
 * ws_predict      u0 for nrhs device columns of f (ld >= N).  Asynchronous.
 * The forward 3x3 convolutions run on the tensor cores (BF16 operands, FP32 accumulation); a
 * convolution whose bounded wait for its MMAs ran out leaves a device flag that the next
 * synchronising call (ws_forward_raw, ws_backward_raw, ws_train_step with loss != NULL) reports
 * as IE_ERR_TIMEOUT, clearing it; outputs are then unspecified.
 */
typedef struct ws_model ws_model;
IEDD_API int ws_create(int device, unsigned long long seed, ws_model **out);
IEDD_API void ws_destroy(ws_model *w);
IEDD_API long long ws_num_params(const ws_model *w);
IEDD_API int ws_get_params(const ws_model *w, float *host);
IEDD_API int ws_set_params(ws_model *w, const float *host);
IEDD_API int ws_forward_raw(ws_model *w, const float *in, float *out, int B, int n, void *stream);
IEDD_API int ws_backward_raw(ws_model *w, const float *in, const float *dout, float *grad, int B, int n,
                             void *stream);
IEDD_API int ws_train_step(ws_model *w, const ie_problem *p, const double *f, const double *u, int batch,
                           long long ld, float lr, double *loss, void *stream);
IEDD_API int ws_predict(ws_model *w, const ie_problem *p, const double *f, double *u0, int nrhs, long long ld,
                        void *stream);

/* Instrumentation: number of kernels this library has launched in this process (a CUDA-graph
 * replay counts the kernel nodes of the graph); reset != 0 returns the count and zeroes it. */
IEDD_API long long ie_kernel_launches(int reset);

/*
 * ie_fp64_fma_rate -- instrumentation (not in the paper): the FP64 FMA throughput of `device` in
 * TFLOP/s (2 flops per FMA), measured by a kernel of eight independent FMA chains per thread on
 * every SM (8 CTAs of 256 threads per SM), best of five timed launches after a warm-up (CUDA
 * events).  The denominator for the FP64-bound kernels' roofline (the RS factor).  Synchronous;
 * IE_ERR_ARG for a NULL out, IE_ERR_CUDA on a CUDA failure.
 */
IEDD_API int ie_fp64_fma_rate(int device, double *tflops);

/*
 * ie_autotune -- the library's autotuner (not in the paper): launch shapes of the explicit-inverse
 * apply (rows per work item, rows per warp pass, loads in flight) and of the FFT passes (lines per
 * CTA) are chosen by timing every candidate once per problem shape, at dd_factor and at the first
 * IE_FFT use (both synchronous and outside any stream capture), and cached for the process.  All
 * candidates compute bitwise identical results.  On by default; the environment variable
 * IEDD_AUTOTUNE=0 starts with it off.
 *   mode  -1: query; 0: off; 1: on; 2: forget the cached choices (state unchanged)
 * Returns the state before the call (1 on, 0 off).  Thread-safe.
 */
IEDD_API int ie_autotune(int mode);
/* The cached choices, one line each: "key -> choice (candidate:time ...)"; valid until the next
 * call from the same thread. */
IEDD_API const char *ie_autotune_report(void);

/* Fills *o with the defaults: tol 1e-8, max_it 1000, IE_MIXED, replace_every 50, use_x0 0,
 * timeout_s 0, check_every 8, verify 1. */
IEDD_API void pcg_default_opts(pcg_opts *o);

/*
 * pcg_solve -- preconditioned conjugate gradient (Hestenes-Stiefel, as used in Sec. 6) on
 * A u = f with T^{-1} from dd_factor, nrhs independent recurrences (per-column scalars; a
 * converged column is frozen).
 *   f      N x nrhs right-hand sides (host or device), column-major, leading dimension ld
 *   u      N x nrhs output (host or device); the initial iterate on entry if opts->use_x0
 *   opts   NULL for the defaults
 *   rep    (host, may be NULL) nrhs reports
 * Iteration: r = f - A u0; z = T^{-1} r; p = z; then q = A p, alpha = r^T z / p^T q,
 * u += alpha p, r -= alpha q, z = T^{-1} r, beta = r_new^T z_new / r^T z, p = z + beta p.
 * IE_MIXED: q = A p by the inner matvec (pcg_opts.inner), T^{-1} in the factor's precision,
 * vectors and scalars in FP64.  When the recursive residual reaches tol (and every
 * replace_every iterations) r is replaced by the accurate f - A u (the FP64-class matvec chosen
 * by pcg_opts.residual); a column is done only when that true residual is <= tol.  IE_FP64:
 * stops on the recursive residual; with verify = 1 the true residual is reported.  A
 * tensor-core inner matvec that timed out (bounded waits) makes every column IE_ERR_TIMEOUT.
 * Returns IE_OK if every column converged, else the first failing column's status.
 * Synchronizes the stream.
 */
IEDD_API int pcg_solve(const ie_problem *p, const dd_factor_t *f, const double *rhs, double *u, int nrhs,
              long long ld, const pcg_opts *opts, pcg_report *rep, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IEDD_H */
